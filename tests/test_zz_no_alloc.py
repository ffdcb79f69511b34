"""apic_sort_keys_noalloc, the key sort for callers that cannot allocate device memory
(a host framework that owns all device memory, or a loop that must not call cudaMalloc
after start-up): it is called through the C ABI with caller-owned inputs and outputs only,
and must give exactly the sort that apic_p2g runs (keys and permutation are integer work,
so the bar is bit-exact), call after call, even though every call reuses the same static
scratch array inside the library.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

from paper_1603_06188_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06188_gb300 import apic

    apic.load(build_if_missing=True)
    return torch, apic


def key_bits(res: int, dim: int = 3) -> int:
    """Bits of the cell key: block index (4^dim nodes per block) above the in-block node."""
    nblocks = ((res + 3) // 4) ** dim
    return 2 * dim + int(np.ceil(np.log2(nblocks)))


def reference_sort(apic, res: int, side: float, ppc: int, seed: int):
    """The sort apic_p2g runs, observed through apic_keys_download."""
    sc = scenes.falling_cube_3d(res=res, side=side, ppc=ppc, seed=seed)
    cfg = apic.make_config(dim=3, order=2, res=(res,) * 3, dx=sc.dx, dt=1e-4, particle_mass=1.0,
                           particle_volume=sc.dx ** 3 / ppc)
    sim = apic.Sim(cfg, sc.n)
    sim.upload(sc.x, sc.v)
    sim.p2g()
    sorted_keys, perm = sim.keys()
    sim.close()
    unsorted = np.empty_like(sorted_keys)
    unsorted[perm] = sorted_keys            # the keys in the order the sort received them
    return unsorted, sorted_keys, perm


def run_noalloc(torch, apic, unsorted: np.ndarray, bits: int):
    n = len(unsorted)
    dk = torch.from_numpy(unsorted.view(np.int32).copy()).cuda()
    out_k = torch.full_like(dk, -1)
    out_p = torch.full_like(dk, -1)
    stream = torch.cuda.current_stream()
    st = apic.apic_sort_keys_noalloc(dk, n, bits, out_k, out_p, stream.cuda_stream)
    torch.cuda.synchronize()
    return st, out_k.cpu().numpy().view(np.uint32), out_p.cpu().numpy().view(np.uint32)


def test_noalloc_sort_equals_the_step_sort_on_consecutive_calls(env):
    torch, apic = env
    # two grids: 15-bit keys (two radix passes) and 21-bit keys (three passes), so the
    # result lands in the caller's buffers for both parities of the ping-pong
    cases = [(32, 0.5, 8, 0), (128, 0.35, 8, 1), (32, 0.5, 8, 0)]
    for res, side, ppc, seed in cases:
        unsorted, ref_keys, ref_perm = reference_sort(apic, res, side, ppc, seed)
        assert len(unsorted) <= apic.APIC_SORT_NOALLOC_MAX_KEYS
        st, got_keys, got_perm = run_noalloc(torch, apic, unsorted, key_bits(res))
        assert st == apic.APIC_OK
        np.testing.assert_array_equal(got_keys, ref_keys)
        np.testing.assert_array_equal(got_perm, ref_perm)


def test_noalloc_sort_rejects_too_many_keys(env):
    torch, apic = env
    dk = torch.zeros(16, dtype=torch.int32, device="cuda")
    st = apic.apic_sort_keys_noalloc(dk, apic.APIC_SORT_NOALLOC_MAX_KEYS + 1, 21, dk, dk, 0)
    assert st == apic.APIC_ERR_OOM
    assert apic.apic_sort_keys_noalloc(dk, 16, 0, dk, dk, 0) == apic.APIC_ERR_ARG
    assert apic.apic_sort_keys_noalloc(dk, 0, 21, dk, dk, 0) == apic.APIC_OK
