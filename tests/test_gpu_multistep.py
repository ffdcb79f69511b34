"""Several consecutive steps at the benchmark's settings (FP32, quadratic, 32 particles per
cell, fixed-corotated, gravity, sticky walls, dt = 2e-5): after every step the state is
downloaded (which reports any latched device error) and compared with one oracle step
from the previous GPU state.  This exercises what a single step does not: the sort of
keys written by G2P, the particles' sorted storage order, and the ping-pong state."""
import numpy as np
import pytest

import oracle
from helpers import configs, kappa, relerr
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


@pytest.mark.parametrize("p2g_kernel,tile", [(0, 0), (0, 256), (0, 1024), (1, 0), (1, 256)])
def test_consecutive_steps_match_oracle(apic, p2g_kernel, tile):
    res, ppc = 32, 32
    sc = scenes.falling_cube_3d(res=res, side=0.5, ppc=ppc, seed=9, omega=(0.0, 0.0, 2.0), v0=(0.3, 0.0, 0.0))
    rng = np.random.default_rng(9)
    B = sc.grad_v * kappa(2) * sc.dx ** 2
    F = scenes.random_deformation(rng, sc.n, 3, 0.02)
    gc, oc, m, vol = configs(3, 2, (res,) * 3, sc.dx, dt=2e-5, gravity=(0.0, -9.8, 0.0), boundary="sticky", wall=3,
                             vol=sc.dx ** 3 / ppc, mass=sc.dx ** 3 / ppc, tile=tile,
                             p2g_kernel=p2g_kernel)
    sim = apic.Sim(gc, sc.n)
    sim.upload(sc.x, sc.v, B, F)
    state = sim.download()
    for step in range(6):
        sim.step(1)
        got = sim.download()                    # raises if a device check latched an error
        x0, v0, B0, F0 = state
        ox, ov, oB, oF, bad = oracle.step(oc, x0, v0, B0, F0, m, vol)
        assert bad == 0
        gx, gv, gB, gF = got
        assert relerr(gv, ov) <= 1e-5, f"step {step}"
        assert relerr(gB, oB) <= 1e-4, f"step {step}"
        assert relerr(gF, oF) <= 1e-5, f"step {step}"
        # the change of F in one step is ~1e-5 of F, so it carries the FP32 rounding of the
        # stored F (half an ulp of |F| ~ 1) on top of the relative error of the velocity gradient
        dF_bound = 1e-5 * np.abs(oF - F0).max() + 2 * np.finfo(np.float32).eps * np.abs(oF).max()
        assert np.abs((gF - F0) - (oF - F0)).max() <= dF_bound, f"step {step}"
        assert np.abs(gx - ox).max() <= 1e-5 * sc.dx, f"step {step}"
        state = got
    sim.close()
