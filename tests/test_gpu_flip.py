"""FLIP and PIC/FLIP blends on the GPU: whole steps against the
oracle's transfer 2 (the FLIP update of Sec. 1 blended with PIC's by flip_alpha) in 3-D FP32
and 2-D cubic FP64, with elastic forces and gravity; FLIP keeps particle velocities when the
grid leaves them unchanged while PIC filters them; batches refuse FLIP simulations; the
blend weight is checked."""
import numpy as np
import pytest

import oracle
from helpers import configs, relerr
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


def _scene(dim, res, ppc, seed):
    if dim == 3:
        return scenes.falling_cube_3d(res=res, side=0.5, ppc=ppc, seed=seed, omega=(0.5, -1.0, 2.0), v0=(0.3, 0.1, -0.2))
    return scenes.rotating_disk_2d(res=res, radius=0.25, ppc=ppc, seed=seed, omega=2.0)


def _flip_configs(apic, dim, order, prec, res, dx, alpha, model="fcr", gravity=None, dt=2e-4):
    g = gravity if gravity is not None else (0.0, -9.8, 0.0)[:dim]
    gc, oc, m, vol = configs(dim, order, (res,) * dim, dx, precision=prec, dt=dt, gravity=g, model=model)
    gc.transfer = 2
    gc.flip_alpha = alpha
    oc.transfer = 2
    oc.flip_alpha = alpha
    return gc, oc, m, vol


@pytest.mark.parametrize("dim,order,prec,res,ppc,alpha", [(3, 2, 32, 32, 8, 1.0), (3, 2, 32, 32, 8, 0.95),
                                                          (2, 3, 64, 64, 4, 1.0), (2, 3, 64, 64, 4, 0.9)])
def test_flip_steps_match_oracle(apic, dim, order, prec, res, ppc, alpha):
    sc = _scene(dim, res, ppc, seed=12)
    rng = np.random.default_rng(12)
    n = sc.n
    v = sc.v + 0.2 * rng.normal(size=(n, dim))          # a noisy field PIC would filter
    F = scenes.random_deformation(rng, n, dim, 0.05)
    gc, oc, m, vol = _flip_configs(apic, dim, order, prec, res, sc.dx, alpha)
    sim = apic.Sim(gc, n)
    sim.upload(sc.x, v, None, F)
    state = sim.download()
    tol = 1e-5 if prec == 32 else 1e-11
    for step in range(3):
        sim.step(1)
        got = sim.download()
        ox, ov, oB, oF, bad = oracle.step(oc, *state, m, vol)
        assert bad == 0
        assert relerr(got[1], ov) <= tol, f"step {step}"
        assert np.all(got[2] == 0)
        assert relerr(got[3], oF) <= tol, f"step {step}"
        assert np.abs(got[0] - ox).max() <= (1e-5 if prec == 32 else 1e-12) * sc.dx
        state = got
    sim.close()


def test_flip_keeps_velocities_pic_filters_them(apic):
    sc = _scene(3, 32, 8, seed=13)
    rng = np.random.default_rng(13)
    v = rng.normal(size=(sc.n, 3))
    out = {}
    for transfer in ("flip", "pic"):
        gc, oc, m, vol = configs(3, 2, (32,) * 3, sc.dx, dt=1e-4, model="none", transfer="pic")
        if transfer == "flip":
            gc.transfer, gc.flip_alpha = 2, 1.0
        sim = apic.Sim(gc, sc.n)
        sim.upload(sc.x, v)
        sim.step(1)
        out[transfer] = sim.download()[1]
        sim.close()
    assert relerr(out["flip"], v) <= 1e-6           # the two grid passes differ only by rounding
    assert relerr(out["pic"], v) > 0.1


def test_flip_is_refused_by_batches_and_alpha_is_checked(apic):
    sc = _scene(3, 32, 8, seed=14)
    gc, oc, m, vol = _flip_configs(apic, 3, 2, 32, 32, sc.dx, 1.0)
    sim = apic.Sim(gc, sc.n)
    sim.upload(sc.x, sc.v)
    batch = apic.Batch(dim=3, order=2, max_sims=2, max_particles=400000, max_blocks=100000)
    with pytest.raises(apic.ApicError):
        batch.add(sim)
    batch.close()
    sim.close()
    gc.flip_alpha = 1.5
    with pytest.raises(Exception):
        apic.Sim(gc, sc.n)
