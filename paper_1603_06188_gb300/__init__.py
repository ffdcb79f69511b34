"""GB300-native APIC / explicit MPM hot path (Jiang, Schroeder & Teran, arXiv:1603.06188).

The compute path is the CUDA library ``libapic.so`` built from ``csrc/`` for sm_103a; the
C-ABI is declared in ``include/apic.h``.  ``apic`` is a thin ctypes binding with the same
entry-point names (argument marshalling only).  ``scenes`` holds the seeded synthetic
inputs.  Nothing here falls back to CPU arithmetic: calling the binding without the
built library raises.
"""
__all__ = ["scenes"]
