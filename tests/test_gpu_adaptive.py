"""Steps whose time step follows the Sec. 4.3 bound, dt = min(dt_max, nu dx / max_p(|v_p| +
6 sqrt(d)/dx |B_p|_F)), on the GPU: one step at a time
against the oracle taking its own time step by the same rule (the first maximum of a call
is the library's FP64 reduction of the current state); several steps in one call, where
the maximum comes from G2P's fused FP32 reduction; and a small dt_max, where the run
equals plain steps at dt = dt_max."""
import numpy as np
import pytest

import oracle
from helpers import configs, kappa, relerr
from paper_1603_06188_gb300 import scenes

pytestmark = pytest.mark.gpu
NU = 0.5


@pytest.fixture(scope="module")
def apic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06188_gb300 import apic as mod

    mod.load(build_if_missing=True)
    return mod


def _spinning(prec):
    res = 32
    sc = scenes.falling_cube_3d(res=res, side=0.4, ppc=8, seed=11, omega=(4.0, -6.0, 12.0), v0=(0.5, 0.0, 0.0))
    rng = np.random.default_rng(11)
    B = sc.grad_v * kappa(2) * sc.dx ** 2
    F = scenes.random_deformation(rng, sc.n, 3, 0.02)
    gc, oc, m, vol = configs(3, 2, (res,) * 3, sc.dx, precision=prec, dt=1e-2, model="fcr")
    return sc, B, F, gc, oc, m, vol


@pytest.mark.parametrize("prec", [32, 64])
def test_adaptive_step_by_step_matches_oracle(apic, prec):
    sc, B, F, gc, oc, m, vol = _spinning(prec)
    dt_max = 1e-2
    sim = apic.Sim(gc, sc.n)
    sim.upload(sc.x, sc.v, B, F)
    state = sim.download()
    tol = 1e-5 if prec == 32 else 1e-11
    for step in range(3):
        t = sim.step_adaptive(1, NU, dt_max)
        speed = oracle.cfl_speed(oc, state[1], state[2])
        dt = min(dt_max, NU * sc.dx / speed)
        assert dt < dt_max                      # the bound is active in this scene
        assert t == pytest.approx(dt, rel=1e-6 if prec == 32 else 1e-12)
        oc.dt = t                               # the step the library took (FP32 rounding of dt)
        ox, ov, oB, oF, bad = oracle.step(oc, *state, m, vol)
        assert bad == 0
        got = sim.download()
        assert relerr(got[1], ov) <= tol, f"step {step}"
        assert relerr(got[3], oF) <= tol, f"step {step}"
        assert np.abs(got[0] - ox).max() <= (1e-5 if prec == 32 else 1e-12) * sc.dx
        state = got
    sim.close()


def test_adaptive_many_steps_follow_the_fused_maximum(apic):
    sc, B, F, gc, oc, m, vol = _spinning(32)
    sim = apic.Sim(gc, sc.n)
    sim.upload(sc.x, sc.v, B, F)
    state = sim.download()
    t = sim.step_adaptive(4, NU, 1e-2)
    got = sim.download()
    total = 0.0
    for _ in range(4):
        dt = min(1e-2, NU * sc.dx / oracle.cfl_speed(oc, state[1], state[2]))
        oc.dt = dt
        state = oracle.step(oc, *state, m, vol)[:4]
        total += dt
    assert t == pytest.approx(total, rel=1e-5)
    assert relerr(got[1], state[1]) <= 1e-4
    assert relerr(got[3], state[3]) <= 1e-5
    sim.close()


def test_small_dt_max_equals_plain_steps(apic):
    sc, B, F, gc, oc, m, vol = _spinning(32)
    dt_max = 1e-4
    gc2, *_ = configs(3, 2, (32,) * 3, sc.dx, dt=dt_max, model="fcr")
    a = apic.Sim(gc, sc.n)
    a.upload(sc.x, sc.v, B, F)
    t = a.step_adaptive(5, NU, dt_max)
    b = apic.Sim(gc2, sc.n)
    b.upload(sc.x, sc.v, B, F)
    b.step(5)
    assert t == pytest.approx(5 * np.float32(dt_max), rel=1e-7)
    for u, w in zip(a.download(), b.download()):
        assert relerr(u, w) <= 1e-5
    a.close()
    b.close()


def test_adaptive_arguments_are_checked(apic):
    sc, B, F, gc, oc, m, vol = _spinning(32)
    sim = apic.Sim(gc, sc.n)
    sim.upload(sc.x, sc.v, B, F)
    for nu, dtm in ((0.0, 1e-3), (0.5, 0.0), (-1.0, 1e-3)):
        with pytest.raises(apic.ApicError):
            sim.step_adaptive(1, nu, dtm)
    assert sim.step_adaptive(0, NU, 1e-3) == 0.0
    sim.close()
