"""apic_sort_keys_noalloc, the key sort for callers that cannot allocate device memory
(a host framework that owns all device memory and gives plug-ins no allocator, or a loop
that must not call cudaMalloc after start-up): it is called through the C ABI with
caller-owned inputs and outputs only.  Keys and permutation are integer work, so the bar is
bit-exact: against the oracle's stable sort of the same keys, and against the sort that
apic_p2g runs, call after call, even though every call reuses the same static scratch
array inside the library.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

import oracle
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


def step_sort(apic, res: int, side: float, ppc: int, seed: int):
    """Cell keys of a scene in upload order, from the oracle's key rule applied to the
    positions the library holds, and the sort apic_p2g runs on them (apic_keys_download)."""
    sc = scenes.falling_cube_3d(res=res, side=side, ppc=ppc, seed=seed)
    cfg = apic.make_config(dim=3, order=2, res=(res,) * 3, dx=sc.dx, dt=1e-4, particle_mass=1.0,
                           particle_volume=sc.dx ** 3 / ppc)
    sim = apic.Sim(cfg, sc.n)
    sim.upload(sc.x, sc.v)
    cell, off = sim.download_positions()
    sim.p2g()
    sorted_keys, perm = sim.keys()
    sim.close()
    oc = oracle.make_cfg(dim=3, order=2, res=(res,) * 3, dx=sc.dx)
    return oracle.keys(oc, 4, cell, off), sorted_keys, perm


def run_noalloc(torch, apic, keys: np.ndarray, bits: int):
    n = len(keys)
    dk = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    out_k = torch.full_like(dk, -1)
    out_p = torch.full_like(dk, -1)
    stream = torch.cuda.current_stream()
    st = apic.apic_sort_keys_noalloc(dk, n, bits, out_k, out_p, stream.cuda_stream)
    torch.cuda.synchronize()
    return st, out_k.cpu().numpy().view(np.uint32), out_p.cpu().numpy().view(np.uint32)


def test_noalloc_sort_matches_oracle_and_step_sort_on_consecutive_calls(env):
    torch, apic = env
    # two grids: 15-bit keys (two radix passes) and 21-bit keys (three passes), so the
    # result lands in the caller's buffers for both parities of the ping-pong; the first
    # case runs again last, after the array holds another call's contents
    cases = [(32, 0.5, 8, 0), (128, 0.35, 8, 1), (32, 0.5, 8, 0)]
    for res, side, ppc, seed in cases:
        keys, step_keys, step_perm = step_sort(apic, res, side, ppc, seed)
        assert len(keys) <= apic.APIC_SORT_NOALLOC_MAX_KEYS
        ref_perm = oracle.stable_sort(keys)
        st, got_keys, got_perm = run_noalloc(torch, apic, keys, key_bits(res))
        assert st == apic.APIC_OK
        np.testing.assert_array_equal(got_perm.astype(np.int64), ref_perm)
        np.testing.assert_array_equal(got_keys, keys[ref_perm])
        # the same result as the step's own sort of these keys
        np.testing.assert_array_equal(got_keys, step_keys)
        np.testing.assert_array_equal(got_perm, step_perm)


def test_noalloc_sort_many_equal_keys_and_full_width(env):
    """Random keys with many repeats (stability decides most of the permutation), every bit
    count from one digit to four, against the oracle's stable sort, two calls in a row."""
    torch, apic = env
    rng = np.random.default_rng(5)
    for bits, n in ((8, 1000), (13, 70001), (24, 300000), (32, 1 << 20), (13, 70001)):
        hi = (1 << bits) - 1
        keys = (rng.integers(0, min(hi, 4096) + 1, size=n, dtype=np.uint64) * (hi // max(min(hi, 4096), 1)))
        keys = np.minimum(keys, hi).astype(np.uint32)
        st, got_keys, got_perm = run_noalloc(torch, apic, keys, bits)
        assert st == apic.APIC_OK
        ref = oracle.stable_sort(keys)
        np.testing.assert_array_equal(got_perm.astype(np.int64), ref)
        np.testing.assert_array_equal(got_keys, keys[ref])


def test_noalloc_sort_rejects_bad_arguments(env):
    torch, apic = env
    dk = torch.zeros(64, dtype=torch.int32, device="cuda")
    a, b = dk[:16], dk[32:48]
    st = apic.apic_sort_keys_noalloc(a, apic.APIC_SORT_NOALLOC_MAX_KEYS + 1, 21, b, dk[48:], 0)
    assert st == apic.APIC_ERR_OOM
    assert apic.apic_sort_keys_noalloc(a, 16, 0, b, dk[48:], 0) == apic.APIC_ERR_ARG
    assert apic.apic_sort_keys_noalloc(a, 0, 21, b, dk[48:], 0) == apic.APIC_OK
    # overlapping buffers are refused before any launch
    assert apic.apic_sort_keys_noalloc(a, 16, 21, a, b, 0) == apic.APIC_ERR_ARG
    assert apic.apic_sort_keys_noalloc(a, 16, 21, b, b, 0) == apic.APIC_ERR_ARG
    assert apic.apic_sort_keys_noalloc(a, 16, 21, dk[8:24], b, 0) == apic.APIC_ERR_ARG
    assert apic.apic_sort_keys_noalloc(a, 16, 21, b, dk[40:56], 0) == apic.APIC_ERR_ARG
    torch.cuda.synchronize()
