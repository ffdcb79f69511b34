"""Thin ctypes binding of the C ABI in include/apic.h (argument marshalling only).

Module-level functions carry the C entry points' names; :class:`Sim` bundles them with a
torch-allocated device workspace (PyTorch provides device memory and the stream; every
step of the method runs in libapic.so's kernels).  Loading fails loudly when the library
has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

APIC_OK, APIC_ERR_ARG, APIC_ERR_OOM, APIC_ERR_CUDA, APIC_ERR_TIMEOUT, APIC_ERR_NUMERIC, APIC_ERR_UNSUPPORTED = range(7)
TRANSFER = {"apic": 0, "pic": 1, "flip": 2}
BOUNDARY = {"none": 0, "sticky": 1, "slip": 2}
MODEL = {"none": 0, "fcr": 1, "fixed_corotated": 1, "nh": 2, "neohookean": 2}
WHERE_PARTICLES, WHERE_GRID = 0, 1
GRID_MOMENTUM, GRID_VELOCITY = 0, 1
STATUS_NAMES = {0: "APIC_OK", 1: "APIC_ERR_ARG", 2: "APIC_ERR_OOM", 3: "APIC_ERR_CUDA", 4: "APIC_ERR_TIMEOUT",
                5: "APIC_ERR_NUMERIC", 6: "APIC_ERR_UNSUPPORTED"}


class ApicError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    """Mirror of ``apic_config``."""

    _fields_ = [
        ("dim", C.c_int), ("order", C.c_int), ("precision", C.c_int), ("transfer", C.c_int),
        ("res", C.c_int * 3), ("dx", C.c_double), ("origin", C.c_double * 3),
        ("dt", C.c_double), ("gravity", C.c_double * 3),
        ("boundary", C.c_int), ("wall", C.c_int), ("model", C.c_int),
        ("E", C.c_double), ("nu", C.c_double),
        ("particle_mass", C.c_double), ("particle_volume", C.c_double),
        ("tile_particles", C.c_int), ("p2g_kernel", C.c_int), ("flip_alpha", C.c_double),
        ("p2g_group", C.c_int), ("integrator", C.c_int), ("newton_max", C.c_int), ("cg_max", C.c_int),
        ("solve_tol", C.c_double),
    ]


def make_config(dim=3, order=2, precision=32, transfer="apic", res=(64, 64, 64), dx=1 / 64, origin=(0, 0, 0),
                dt=0.0, gravity=(0, 0, 0), boundary="none", wall=0, model="none", E=0.0, nu=0.0,
                particle_mass=1.0, particle_volume=1.0, tile_particles=0, p2g_kernel=0, flip_alpha=1.0,
                p2g_group=0, integrator=0, newton_max=0, cg_max=0, solve_tol=0.0) -> Config:
    """integrator: 0 = lambda = 0 (symplectic Euler), 1 = the explicit member lambda = 1,
    2 = the implicit midpoint rule (newton_max, cg_max, solve_tol: 0 = the library's defaults)."""
    c = Config()
    c.integrator = integrator
    c.newton_max, c.cg_max, c.solve_tol = newton_max, cg_max, solve_tol
    c.p2g_group = p2g_group
    c.flip_alpha = flip_alpha
    c.dim, c.order, c.precision = dim, order, precision
    c.transfer = TRANSFER[transfer] if isinstance(transfer, str) else transfer
    r = list(res) + [1] * (3 - len(res))
    c.res = (C.c_int * 3)(*r)
    c.dx = dx
    c.origin = (C.c_double * 3)(*(list(origin) + [0.0] * (3 - len(origin))))
    c.dt = dt
    c.gravity = (C.c_double * 3)(*(list(gravity) + [0.0] * (3 - len(gravity))))
    c.boundary = BOUNDARY[boundary] if isinstance(boundary, str) else boundary
    c.wall = wall
    c.model = MODEL[model] if isinstance(model, str) else model
    c.E, c.nu = E, nu
    c.particle_mass, c.particle_volume = particle_mass, particle_volume
    c.tile_particles = tile_particles
    c.p2g_kernel = p2g_kernel
    return c


class BatchConfig(C.Structure):
    """Mirror of ``apic_batch_config``."""

    _fields_ = [
        ("dim", C.c_int), ("order", C.c_int), ("precision", C.c_int), ("max_sims", C.c_int),
        ("max_particles", C.c_int64), ("max_blocks", C.c_int64),
        ("tile_particles", C.c_int), ("group", C.c_int), ("use_graph", C.c_int),
    ]


_lib = None
SIGNATURES = {
    "apic_workspace_size": (C.c_int, [C.POINTER(Config), C.c_int64, C.POINTER(C.c_size_t)]),
    "apic_create": (C.c_int, [C.POINTER(Config), C.c_int64, C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]),
    "apic_destroy": (C.c_int, [C.c_void_p]),
    "apic_upload": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "apic_upload_materials": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int]),
    "apic_upload_mass_volume": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int]),
    "apic_download": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "apic_download_positions": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "apic_p2g": (C.c_int, [C.c_void_p]),
    "apic_grid_update": (C.c_int, [C.c_void_p]),
    "apic_g2p": (C.c_int, [C.c_void_p]),
    "apic_step": (C.c_int, [C.c_void_p, C.c_int]),
    "apic_step_adaptive": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_double)]),
    "apic_momentum": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "apic_momentum_async": (C.c_int, [C.c_void_p, C.c_void_p]),
    "apic_momentum_wait": (C.c_int, [C.c_void_p]),
    "apic_cfl": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "apic_grid_download": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "apic_keys_download": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "apic_grid_occupancy": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "apic_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "apic_last_error": (C.c_char_p, [C.c_void_p]),
    "apic_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "apic_batch_workspace_size": (C.c_int, [C.POINTER(BatchConfig), C.POINTER(C.c_size_t)]),
    "apic_batch_create": (C.c_int, [C.POINTER(BatchConfig), C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]),
    "apic_batch_destroy": (C.c_int, [C.c_void_p]),
    "apic_batch_add": (C.c_int, [C.c_void_p, C.c_void_p]),
    "apic_batch_remove": (C.c_int, [C.c_void_p, C.c_void_p]),
    "apic_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "apic_batch_set_tuning": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "apic_batch_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "apic_batch_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "apic_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "apic_sort_keys_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "apic_profile_read": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "apic_set_wait_limit": (C.c_int, [C.c_void_p, C.c_uint]),
    "apic_batch_admit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_int64]),
    "apic_batch_run": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_int),
                                 C.POINTER(C.c_int)]),
    "apic_batch_resident_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "apic_solve_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
}
PHASES = ["keys", "sort", "tiles", "p2g", "grid_update", "g2p"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libapic.so (optionally building it first).  Raises if it is not there."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libapic.so is not built ({path}); run __graft_entry__.build() or "
                               "python -m paper_1603_06188_gb300.build")
        _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st: int, sim=None):
    if st != APIC_OK:
        msg = load().apic_last_error(sim).decode() if sim else ""
        raise ApicError(st, msg)


def _ptr(a) -> C.c_void_p | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())


# ----------------------------------------------------------------------- C entry points
def apic_workspace_size(cfg: Config, max_particles: int) -> int:
    out = C.c_size_t(0)
    _check(load().apic_workspace_size(C.byref(cfg), max_particles, C.byref(out)))
    return out.value


def apic_create(cfg: Config, max_particles: int, workspace_ptr: int, workspace_bytes: int, stream_ptr: int):
    h = C.c_void_p()
    _check(load().apic_create(C.byref(cfg), max_particles, C.c_void_p(workspace_ptr), workspace_bytes,
                              C.c_void_p(stream_ptr), C.byref(h)))
    return h


def apic_destroy(sim):
    _check(load().apic_destroy(sim))


def apic_upload(sim, n, x, v=None, B=None, F=None, on_device=0):
    _check(load().apic_upload(sim, n, _ptr(x), _ptr(v), _ptr(B), _ptr(F), on_device), sim)


def apic_upload_materials(sim, n, E, nu, on_device=0):
    _check(load().apic_upload_materials(sim, n, _ptr(E), _ptr(nu), on_device), sim)


def apic_upload_mass_volume(sim, n, mass, vol, on_device=0):
    _check(load().apic_upload_mass_volume(sim, n, _ptr(mass), _ptr(vol), on_device), sim)


# dimension of each simulation handle made through Sim, so that the host-array wrappers can
# check an output array holds what the library will write into it
_DIMS: dict = {}


def _check_host_outputs(sim, arrays):
    """Raise APIC_ERR_ARG if a host output array is smaller than the library's particle count
    times its per-particle entries (the library writes that many)."""
    d = _DIMS.get(sim if isinstance(sim, int) else getattr(sim, "value", sim))
    if d is None:
        return
    n = int(apic_stats(sim)[0])
    for a, per in arrays:
        if isinstance(a, np.ndarray) and a.size < n * per(d):
            raise ApicError(APIC_ERR_ARG, f"host array of {a.size} entries for {n} particles")


def apic_download(sim, x=None, v=None, B=None, F=None, on_device=0):
    if not on_device:
        _check_host_outputs(sim, [(x, lambda d: d), (v, lambda d: d), (B, lambda d: d * d), (F, lambda d: d * d)])
    _check(load().apic_download(sim, _ptr(x), _ptr(v), _ptr(B), _ptr(F), on_device), sim)


def apic_download_positions(sim, cell, offset):
    _check_host_outputs(sim, [(cell, lambda d: d), (offset, lambda d: d)])
    _check(load().apic_download_positions(sim, _ptr(cell), _ptr(offset)), sim)


def apic_p2g(sim):
    _check(load().apic_p2g(sim), sim)


def apic_grid_update(sim):
    _check(load().apic_grid_update(sim), sim)


def apic_g2p(sim):
    _check(load().apic_g2p(sim), sim)


def apic_step(sim, n: int):
    _check(load().apic_step(sim, n), sim)


def apic_momentum(sim, where: int):
    p = np.zeros(3)
    l = np.zeros(3)
    _check(load().apic_momentum(sim, where, _ptr(p), _ptr(l)), sim)
    return p, l


def apic_momentum_async(sim, out):
    """Queue the particle momentum of the current state into out[0:6] = (p, l) without
    synchronising.  `out` is a C-contiguous float64 numpy array or torch tensor of at least 6
    entries (pinned host or CUDA memory for the call to return at once); the caller keeps it
    alive until apic_momentum_wait."""
    if isinstance(out, np.ndarray):
        ok = out.dtype == np.float64 and out.flags.c_contiguous and out.size >= 6
    else:
        import torch

        ok = out.dtype == torch.float64 and out.is_contiguous() and out.numel() >= 6
    if not ok:
        raise ApicError(APIC_ERR_ARG, "momentum output must be 6 contiguous float64 values")
    _check(load().apic_momentum_async(sim, _ptr(out)), sim)


def apic_momentum_wait(sim):
    _check(load().apic_momentum_wait(sim), sim)


def apic_step_adaptive(sim, n: int, nu: float, dt_max: float) -> float:
    out = C.c_double(0.0)
    _check(load().apic_step_adaptive(sim, n, nu, dt_max, C.byref(out)), sim)
    return out.value


def apic_cfl(sim) -> float:
    out = C.c_double(0.0)
    _check(load().apic_cfl(sim, C.byref(out)), sim)
    return out.value


def apic_grid_download(sim, which: int, m, mv):
    _check(load().apic_grid_download(sim, which, _ptr(m), _ptr(mv)), sim)


def apic_keys_download(sim, keys, perm):
    _check(load().apic_keys_download(sim, _ptr(keys), _ptr(perm)), sim)


def apic_grid_occupancy(sim, out, n_blocks: int):
    _check(load().apic_grid_occupancy(sim, _ptr(out), n_blocks), sim)


def apic_stats(sim):
    out = np.zeros(5, dtype=np.int64)
    _check(load().apic_stats(sim, _ptr(out)), sim)
    return out


def apic_solve_stats(sim):
    out = np.zeros(3)
    _check(load().apic_solve_stats(sim, _ptr(out)), sim)
    return out


def apic_set_wait_limit(sim, polls: int):
    _check(load().apic_set_wait_limit(sim, polls), sim)


def apic_last_error(sim) -> str:
    return load().apic_last_error(sim).decode()


APIC_SORT_NOALLOC_MAX_KEYS = 1 << 20
APIC_BATCH_SPLIT = 16


def apic_sort_keys_noalloc(keys, n: int, key_bits: int, sorted_keys, perm, stream_ptr: int = 0) -> int:
    """Stable key sort with no device allocation (static scratch inside the library).

    For callers that cannot allocate device memory; all four pointers are device memory
    the caller owns.  Returns the apic_status code (0 = APIC_OK) without raising, so a
    caller can branch on APIC_ERR_OOM for n above APIC_SORT_NOALLOC_MAX_KEYS."""
    return load().apic_sort_keys_noalloc(_ptr(keys), n, key_bits, _ptr(sorted_keys), _ptr(perm),
                                         C.c_void_p(stream_ptr))


def apic_profile(sim, enable: int):
    _check(load().apic_profile(sim, enable), sim)


def apic_profile_read(sim):
    ms = np.zeros(len(PHASES))
    launches = np.zeros(len(PHASES), dtype=np.int64)
    _check(load().apic_profile_read(sim, _ptr(ms), _ptr(launches)), sim)
    return ms, launches


def _bcheck(st: int, batch=None):
    if st != APIC_OK:
        msg = load().apic_batch_last_error(batch).decode() if batch else ""
        raise ApicError(st, msg)


def apic_batch_workspace_size(cfg: BatchConfig) -> int:
    out = C.c_size_t(0)
    _bcheck(load().apic_batch_workspace_size(C.byref(cfg), C.byref(out)))
    return out.value


def apic_batch_create(cfg: BatchConfig, workspace_ptr: int, workspace_bytes: int, stream_ptr: int):
    h = C.c_void_p()
    _bcheck(load().apic_batch_create(C.byref(cfg), C.c_void_p(workspace_ptr), workspace_bytes, C.c_void_p(stream_ptr),
                                     C.byref(h)))
    return h


def apic_batch_destroy(batch):
    _bcheck(load().apic_batch_destroy(batch))


def apic_batch_add(batch, sim):
    _bcheck(load().apic_batch_add(batch, sim), batch)


def apic_batch_remove(batch, sim):
    _bcheck(load().apic_batch_remove(batch, sim), batch)


def apic_batch_step(batch, n: int):
    _bcheck(load().apic_batch_step(batch, n), batch)


def apic_batch_admit(batch, sim, steps: int, footprint_bytes: int, budget_bytes: int):
    _bcheck(load().apic_batch_admit(batch, sim, steps, footprint_bytes, budget_bytes), batch)


def apic_batch_run(batch, max_steps: int, max_finished: int):
    """Returns (handles of the finished members, steps taken)."""
    cap = max(int(max_finished), 1)
    out = (C.c_void_p * cap)()
    n = C.c_int(0)
    done = C.c_int(0)
    _bcheck(load().apic_batch_run(batch, max_steps, out, cap, C.byref(n), C.byref(done)), batch)
    return [out[i] for i in range(n.value)], done.value


def apic_batch_resident_bytes(batch) -> int:
    out = C.c_int64(0)
    _bcheck(load().apic_batch_resident_bytes(batch, C.byref(out)))
    return out.value


def apic_batch_set_tuning(batch, tile_particles: int, group: int):
    _bcheck(load().apic_batch_set_tuning(batch, tile_particles, group), batch)


def apic_batch_autotune(batch, steps: int, force: int = 0):
    t = C.c_int(0)
    g = C.c_int(0)
    _bcheck(load().apic_batch_autotune(batch, steps, force, C.byref(t), C.byref(g)), batch)
    return t.value, g.value


def apic_batch_stats(batch):
    out = np.zeros(5, dtype=np.int64)
    _bcheck(load().apic_batch_stats(batch, _ptr(out)), batch)
    return out


def apic_batch_last_error(batch) -> str:
    return load().apic_batch_last_error(batch).decode()


# ----------------------------------------------------------------------- convenience
class Sim:
    """One simulation: config + torch-owned device workspace + the library handle."""

    def __init__(self, cfg: Config, max_particles: int, device=None, stream=None):
        import torch

        self.cfg = cfg
        self.dim = cfg.dim
        self.capacity = max_particles
        self.device = torch.device(device or "cuda")
        nbytes = apic_workspace_size(cfg, max_particles)
        # torch's caching allocator returns 512-byte aligned blocks
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.handle = apic_create(cfg, max_particles, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)
        _DIMS[self.handle.value] = self.dim
        self.n = 0

    @property
    def res(self):
        return tuple(self.cfg.res[a] for a in range(self.dim))

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.res))

    @property
    def n_blocks(self) -> int:
        return int(np.prod([(r + 3) // 4 for r in self.res]))

    def upload_materials(self, E, nu):
        """Young's modulus and Poisson's ratio per particle (upload order); scalars broadcast."""
        E = np.ascontiguousarray(np.broadcast_to(np.asarray(E, dtype=np.float64), (self.n,)))
        nu = np.ascontiguousarray(np.broadcast_to(np.asarray(nu, dtype=np.float64), (self.n,)))
        apic_upload_materials(self.handle, self.n, E, nu, on_device=0)

    def upload_mass_volume(self, mass, vol):
        """Mass m_p and volume V_p per particle (upload order); scalars broadcast."""
        mass = np.ascontiguousarray(np.broadcast_to(np.asarray(mass, dtype=np.float64), (self.n,)))
        vol = np.ascontiguousarray(np.broadcast_to(np.asarray(vol, dtype=np.float64), (self.n,)))
        apic_upload_mass_volume(self.handle, self.n, mass, vol, on_device=0)

    def upload(self, x, v=None, B=None, F=None):
        """Host numpy arrays (float64) or CUDA float64 tensors."""
        n = len(x)
        self.n = n
        try:
            if isinstance(x, np.ndarray):
                arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (x, v, B, F)]
                apic_upload(self.handle, n, *arrs, on_device=0)
            else:
                arrs = [None if a is None else a.contiguous() for a in (x, v, B, F)]
                apic_upload(self.handle, n, *arrs, on_device=1)
                self._keep = arrs
        except ApicError:
            # a range error keeps the (clamped) particles; a rejected upload keeps none
            self.n = int(apic_stats(self.handle)[0])
            raise

    def count(self) -> int:
        """The library's particle count (also after an upload through the plain entry point)."""
        self.n = int(apic_stats(self.handle)[0])
        return self.n

    def download(self):
        d, n = self.dim, self.count()
        x = np.zeros((n, d)); v = np.zeros((n, d)); B = np.zeros((n, d, d)); F = np.zeros((n, d, d))
        apic_download(self.handle, x, v, B, F, on_device=0)
        return x, v, B, F

    def download_positions(self):
        self.count()
        cell = np.zeros((self.n, self.dim), dtype=np.int32)
        off = np.zeros((self.n, self.dim))
        apic_download_positions(self.handle, cell, off)
        return cell, off

    def p2g(self):
        apic_p2g(self.handle)

    def grid_update(self):
        apic_grid_update(self.handle)

    def g2p(self):
        apic_g2p(self.handle)

    def step(self, n: int = 1):
        apic_step(self.handle, n)

    def step_adaptive(self, n: int, nu: float, dt_max: float) -> float:
        """n steps at dt = min(dt_max, nu dx / max speed) (Sec. 4.3); returns the simulated time."""
        return apic_step_adaptive(self.handle, n, nu, dt_max)

    def momentum(self, where: str = "particles"):
        return apic_momentum(self.handle, WHERE_PARTICLES if where == "particles" else WHERE_GRID)

    def momentum_async(self, out):
        """Queue the particle momentum (p, l) of the current state into out[0:6]; see
        apic_momentum_async.  Read `out` after momentum_wait()."""
        apic_momentum_async(self.handle, out)

    def momentum_wait(self):
        apic_momentum_wait(self.handle)

    def cfl_speed(self) -> float:
        """max_p(|v_p| + 6 sqrt(d)/dx |B_p|_F); dt <= nu dx / this (Sec. 4.3)."""
        return apic_cfl(self.handle)

    def grid(self, which: str = "momentum"):
        m = np.zeros(self.n_nodes)
        mv = np.zeros((self.n_nodes, self.dim))
        apic_grid_download(self.handle, GRID_MOMENTUM if which == "momentum" else GRID_VELOCITY, m, mv)
        return m, mv

    def keys(self):
        self.count()
        k = np.zeros(self.n, dtype=np.uint32)
        p = np.zeros(self.n, dtype=np.uint32)
        apic_keys_download(self.handle, k, p)
        return k, p

    def occupancy(self):
        out = np.zeros(self.n_blocks, dtype=np.uint8)
        apic_grid_occupancy(self.handle, out, self.n_blocks)
        return out

    def stats(self) -> dict:
        s = apic_stats(self.handle)
        return {"particles": int(s[0]), "blocks": int(s[1]), "tiles": int(s[2]), "polar_fp64_fallbacks": int(s[3]),
                "kernel_launches": int(s[4])}

    def solve_stats(self) -> dict:
        s = apic_solve_stats(self.handle)
        return {"newton": int(s[0]), "cg": int(s[1]), "residual": float(s[2])}

    def profile(self, enable: bool = True):
        apic_profile(self.handle, 1 if enable else 0)

    def profile_read(self) -> dict:
        ms, launches = apic_profile_read(self.handle)
        return {name: {"ms": float(ms[i]), "launches": int(launches[i])} for i, name in enumerate(PHASES)}

    def close(self):
        if getattr(self, "handle", None):
            _DIMS.pop(self.handle.value, None)
            apic_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many simulations stepped together (one persistent launch per phase).

    Uses its own CUDA stream (so steps can be captured in a CUDA graph) and a torch-owned
    workspace for the shared work lists; members keep their own workspaces."""

    def __init__(self, dim: int, order: int, precision: int = 32, max_sims: int = 64, max_particles: int = 1 << 22,
                 max_blocks: int = 1 << 20, tile_particles: int = 0, group: int = 0, use_graph: bool = True,
                 device=None):
        import torch

        self.cfg = BatchConfig()
        self.cfg.dim, self.cfg.order, self.cfg.precision = dim, order, precision
        self.cfg.max_sims, self.cfg.max_particles, self.cfg.max_blocks = max_sims, max_particles, max_blocks
        self.cfg.tile_particles, self.cfg.group, self.cfg.use_graph = tile_particles, group, 1 if use_graph else 0
        self.device = torch.device(device or "cuda")
        nbytes = apic_batch_workspace_size(self.cfg)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = torch.cuda.Stream(self.device)
        self.handle = apic_batch_create(self.cfg, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)
        self.members = []

    def add(self, sim: "Sim"):
        apic_batch_add(self.handle, sim.handle)
        self.members.append(sim)

    def remove(self, sim: "Sim"):
        apic_batch_remove(self.handle, sim.handle)
        self.members.remove(sim)

    def step(self, n: int = 1):
        apic_batch_step(self.handle, n)

    def admit(self, sim: "Sim", steps: int, footprint_bytes: int, budget_bytes: int):
        """Join the batch for `steps` steps if its footprint fits the budget (else ApicError
        with status APIC_ERR_OOM and nothing changes)."""
        apic_batch_admit(self.handle, sim.handle, steps, footprint_bytes, budget_bytes)
        self.members.append(sim)

    def run(self, max_steps: int):
        """Steps to the nearest completion (at most max_steps); returns (the Sims that
        finished and left the batch, steps taken)."""
        handles, done = apic_batch_run(self.handle, max_steps, len(self.members))
        by_handle = {s.handle.value: s for s in self.members}
        fin = [by_handle[h] for h in handles]
        for sim in fin:
            self.members.remove(sim)
        return fin, done

    def resident_bytes(self) -> int:
        return apic_batch_resident_bytes(self.handle)

    def set_tuning(self, tile_particles: int = 0, group: int = 0):
        apic_batch_set_tuning(self.handle, tile_particles, group)

    def autotune(self, steps: int = 3, force: bool = False):
        return apic_batch_autotune(self.handle, steps, 1 if force else 0)

    def stats(self) -> dict:
        s = apic_batch_stats(self.handle)
        return {"members": int(s[0]), "particles": int(s[1]), "steps": int(s[2]), "kernel_launches": int(s[3]),
                "tiles": int(s[4])}

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "handle", None):
            apic_batch_destroy(self.handle)
            self.handle = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
