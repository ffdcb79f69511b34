"""apic_momentum_async: the particle momentum (p, l) of Sec. 3.1 / 5.3 read without
synchronising, on a stream of its own:
- it equals the synchronising apic_momentum of the same state bit for bit (the same
  reduction, its own scratch), in 3-D FP32 and 2-D FP64, into pinned host, pageable host and
  device memory;
- a read queued before later steps or an upload still returns the state at the time of the
  call (the calls that overwrite the copy it reads wait for it on the device);
- bad outputs and batch members are refused."""
import numpy as np
import pytest

from helpers import configs
from paper_1603_06188_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06188_gb300 import apic as mod

    mod.load(build_if_missing=True)
    return mod


def _sim(apic, dim, order, precision, seed=0, res=48):
    if dim == 3:
        sc = scenes.falling_cube_3d(res=res, side=0.3, ppc=8, omega=(3.0, -2.0, 1.0), v0=(0.2, 0.1, -0.3), seed=seed)
    else:
        sc = scenes.rotating_disk_2d(res=res, radius=0.25, ppc=4, omega=2.0, seed=seed)
    gc, _, _, _ = configs(dim, order, (res,) * dim, sc.dx, precision=precision, dt=2e-4, model="fcr",
                          gravity=(0.0, -9.8, 0.0)[:dim])
    sim = apic.Sim(gc, sc.n)
    sim.upload(sc.x, sc.v, sc.grad_v * (0.25 * sc.dx * sc.dx))
    return sim, sc


def _sync6(sim):
    p, l = sim.momentum()
    return np.concatenate([p, l])


@pytest.mark.parametrize("dim,order,precision", [(3, 2, 32), (2, 3, 64)])
def test_async_equals_sync(apic, dim, order, precision):
    import torch

    sim, _ = _sim(apic, dim, order, precision)
    K = 4
    pinned = torch.zeros((K, 6), dtype=torch.float64).pin_memory()
    ref = []
    for k in range(K):
        sim.step(1)
        sim.momentum_async(pinned[k])
        ref.append(_sync6(sim))
    sim.momentum_wait()
    got = pinned.numpy()
    for k in range(K):
        np.testing.assert_array_equal(got[k], ref[k])
    if dim == 2:
        assert not got[:, [2, 4, 5]].any()
    # pageable host memory (the call returns once the read is done) and device memory
    host = np.full(6, np.nan)
    sim.momentum_async(host)
    dev = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    sim.momentum_async(dev)
    sim.momentum_wait()
    last = _sync6(sim)
    np.testing.assert_array_equal(host, last)
    np.testing.assert_array_equal(dev.cpu().numpy(), last)
    sim.close()


def test_async_read_is_of_the_state_at_the_call(apic):
    import torch

    sim, sc = _sim(apic, 3, 2, 32, seed=3, res=64)
    sim.step(1)
    before = _sync6(sim)
    out = torch.full((3, 6), float("nan"), dtype=torch.float64).pin_memory()
    sim.momentum_async(out[0])
    sim.step(3)   # G2P writes both state copies, the one read first two steps on
    mid = _sync6(sim)
    sim.momentum_async(out[1])
    sim.upload(sc.x, -sc.v)   # a new state overwrites the copy just read
    sim.momentum_async(out[2])
    after = _sync6(sim)
    sim.momentum_wait()
    got = out.numpy()
    np.testing.assert_array_equal(got[0], before)
    np.testing.assert_array_equal(got[1], mid)
    np.testing.assert_array_equal(got[2], after)
    assert np.abs(before - mid).max() > 0 and np.abs(mid - after).max() > 0
    sim.close()


def test_async_arguments(apic):
    sim, _ = _sim(apic, 3, 2, 32, seed=5, res=32)
    sim.momentum_wait()   # nothing queued
    for bad in (np.zeros(6, dtype=np.float32), np.zeros(5), np.zeros((6, 2))[:, 0]):
        with pytest.raises(apic.ApicError) as e:
            sim.momentum_async(bad)
        assert e.value.status == apic.APIC_ERR_ARG
    batch = apic.Batch(dim=3, order=2, max_sims=2, max_particles=sim.count() + 1, max_blocks=100000)
    batch.add(sim)
    with pytest.raises(apic.ApicError) as e:
        sim.momentum_async(np.zeros(6))
    assert e.value.status == apic.APIC_ERR_ARG
    batch.close()
    sim.close()


@pytest.mark.parametrize("integrator", [1, 2])
def test_async_read_with_the_other_integrators(apic, integrator):
    """lambda = 1 and the midpoint rule write the next state copy in their own G2P; a read
    queued before two of their steps still returns the state at the time of the call."""
    import torch

    sc = scenes.falling_cube_3d(res=32, side=0.3, ppc=8, omega=(2.0, 1.0, -1.0), seed=9)
    cfg = apic.make_config(dim=3, order=2, res=(32,) * 3, dx=sc.dx, dt=1e-4, model="fcr", E=1e4, nu=0.3,
                           particle_mass=sc.dx ** 3 / 8, particle_volume=sc.dx ** 3 / 8, integrator=integrator)
    sim = apic.Sim(cfg, sc.n)
    sim.upload(sc.x, sc.v, sc.grad_v * (0.25 * sc.dx * sc.dx))
    sim.step(1)
    before = _sync6(sim)
    out = torch.full((6,), float("nan"), dtype=torch.float64).pin_memory()
    sim.momentum_async(out)
    sim.step(2)
    sim.momentum_wait()
    np.testing.assert_array_equal(out.numpy(), before)
    assert np.abs(_sync6(sim) - before).max() > 0
    sim.close()
