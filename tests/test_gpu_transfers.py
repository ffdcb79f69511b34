"""Host uploads and downloads through the C ABI, which move the particles in pieces of about
half a million on a copy stream while the upload and gather kernels run:
- a state of 1.3M particles (three pieces) comes back exactly as uploaded (FP64 host values
  that FP32 stores exactly), and the same after steps that reorder the storage (the download
  gathers in upload order through the inverse of the id lane);
- NULL outputs are skipped and the others are unchanged; NULL v and B upload as zeros and
  NULL F as the identity; the binding refuses a host output too small for the particles;
- host and device uploads of the same state give the same step (to the rounding of the
  grid's global adds, whose order varies between runs)."""
import numpy as np
import pytest

from helpers import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06188_gb300 import apic as mod

    mod.load(build_if_missing=True)
    return mod


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _state(n, res, seed):
    """Positions on cell centres plus FP32-exact offsets, and FP32-exact v, B, F."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    cells = rng.integers(8, res - 8, size=(n, 3))
    off = _f32(rng.integers(0, 1 << 12, size=(n, 3)) / float(1 << 12))
    x = (cells + off) * dx
    v = _f32(rng.normal(size=(n, 3)))
    B = _f32(0.01 * dx * rng.normal(size=(n, 3, 3)))
    F = _f32(np.eye(3) + 0.05 * rng.normal(size=(n, 3, 3)))
    return x, v, B, F, dx


def test_pieces_round_trip_exactly(apic):
    n, res = 1_300_003, 128
    x, v, B, F, dx = _state(n, res, 1)
    gc, _, _, _ = configs(3, 2, (res,) * 3, dx, dt=1e-5, model="fcr")
    sim = apic.Sim(gc, n)
    sim.upload(x, v, B, F)
    gx, gv, gB, gF = sim.download()
    np.testing.assert_allclose(gx, x, rtol=0, atol=4 * np.finfo(np.float64).eps)
    np.testing.assert_array_equal(gv, v)
    np.testing.assert_array_equal(gB, B)
    np.testing.assert_array_equal(gF, F)
    # after steps the storage is in sorted order; the download still returns upload order
    sim.step(2)
    a = sim.download()
    ox, ov, oB, oF = (np.zeros_like(t) for t in (x, v, B, F))
    apic.apic_download(sim.handle, ox, None, None, oF, on_device=0)   # x and F only
    np.testing.assert_array_equal(ox, a[0])
    np.testing.assert_array_equal(oF, a[3])
    assert not ov.any() and not oB.any()
    # each particle comes back as itself: two short steps move it by far less than the
    # distance to another particle and change its F by far less than another particle's F
    # differs (a mix-up in the order would show as O(0.1) differences)
    assert np.abs(a[0] - x).max() < 1e-3
    assert np.abs(a[3] - F).max() < 1e-2
    sim.close()


def test_null_inputs_take_their_defaults(apic):
    n, res = 700_001, 96
    x, _, _, _, dx = _state(n, res, 2)
    gc, _, _, _ = configs(3, 2, (res,) * 3, dx, dt=1e-5, model="none")
    sim = apic.Sim(gc, n)
    apic.apic_upload(sim.handle, n, np.ascontiguousarray(x), None, None, None, on_device=0)
    gx, gv, gB, gF = sim.download()
    np.testing.assert_allclose(gx, x, rtol=0, atol=4 * np.finfo(np.float64).eps)
    assert not gv.any() and not gB.any()
    np.testing.assert_array_equal(gF, np.broadcast_to(np.eye(3), (n, 3, 3)))
    # a host output smaller than the particle count is refused before anything is copied
    with pytest.raises(apic.ApicError) as e:
        apic.apic_download(sim.handle, np.zeros((10, 3)), on_device=0)
    assert e.value.status == apic.APIC_ERR_ARG
    sim.close()


def test_host_and_device_uploads_agree(apic):
    torch = pytest.importorskip("torch")
    n, res = 600_000, 96
    x, v, B, F, dx = _state(n, res, 3)
    gc, _, _, _ = configs(3, 3, (res,) * 3, dx, dt=1e-5, model="fcr")
    out = []
    for on_device in (False, True):
        sim = apic.Sim(gc, n)
        if on_device:
            sim.upload(*(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (x, v, B, F)))
        else:
            sim.upload(x, v, B, F)
        sim.step(1)
        out.append(sim.download())
        sim.close()
    # the same arithmetic; runs differ only by the order of the grid's global adds
    for a, b in zip(*out):
        scale = np.abs(b).max()
        assert np.abs(a - b).max() <= 1e-5 * scale
