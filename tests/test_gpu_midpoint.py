"""The implicit midpoint rule (lambda = 1/2 of the Sec. 3.3 family) on the GPU, through the C ABI,
against the FP64 oracle: Newton on the grid velocity change with the mass-inner-product
conjugate gradients of Algorithm 1 for each system (Sec. 4.1-4.2), the force and its
derivative product at F^{n+1/2}, and the general transfer to particles at lambda = 1/2.

- the grid solve: the GPU's v~ against oracle.midpoint_solve from the GPU's own P2G grid;
- whole steps against oracle.step_midpoint from the GPU's input;
- p and l kept by converged steps (Sec. 4.2, 5.2, 5.3);
- without a constitutive model the rule is the lambda = 0 step;
- what it does not support is refused.
Both sides solve to tight tolerances, so they agree to the solve's accuracy: 1e-9 (FP64) and
1e-5 (FP32, solved to 1e-6 of |v|_M with heavy particles, whose system is well conditioned)."""
import numpy as np
import pytest

import oracle
from helpers import configs, kappa, relerr, state_for
from paper_1603_06188_gb300 import scenes

pytestmark = pytest.mark.gpu

CASES = [
    # dim, order, precision, res, ppc, model
    (3, 2, 64, 16, 8, "fcr"),
    (3, 2, 64, 16, 8, "nh"),
    (3, 3, 64, 16, 8, "fcr"),
    (2, 2, 64, 32, 4, "fcr"),
    (2, 3, 64, 32, 4, "nh"),
    (3, 2, 32, 16, 8, "fcr"),
    (2, 2, 32, 32, 4, "nh"),
]


def _ids(c):
    return f"d{c[0]}_o{c[1]}_fp{c[2]}_{c[5]}"


@pytest.fixture(scope="module")
def apic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06188_gb300 import apic as mod

    mod.load(build_if_missing=True)
    return mod


def setup(apic, case, seed=0, dt=4e-3, model=None, tol=None):
    dim, order, prec, res, ppc, mdl = case
    if dim == 3:
        sc = scenes.falling_cube_3d(res=res, side=0.5, ppc=ppc, seed=seed, omega=(0.5, -1.0, 2.0), v0=(0.3, 0.1, -0.2))
    else:
        sc = scenes.rotating_disk_2d(res=res, radius=0.25, ppc=ppc, seed=seed, omega=2.0)
    x, v, B, F = state_for(sc, order, seed=seed, Fscale=0.1)
    vol = sc.dx ** dim / 8
    gc, oc, m, vol = configs(dim, order, (res,) * dim, sc.dx, precision=prec, dt=dt, model=model or mdl, mass=1.0,
                             vol=vol)
    gc.integrator = 2
    gc.solve_tol = tol if tol is not None else (1e-13 if prec == 64 else 1e-6)
    gc.newton_max, gc.cg_max = 20, 400
    sim = apic.Sim(gc, len(x))
    sim.upload(x, v, B, F)
    return sim, sc, oc, m, vol


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_midpoint_grid_solve_matches_oracle(apic, case):
    dim, order, prec, res, ppc, mdl = case
    sim, sc, oc, m, vol = setup(apic, case)
    x0, v0, B0, F0 = sim.download()
    sim.p2g()
    m_g, mv_g = sim.grid("momentum")
    # P2G transfers mass and momentum alone (the force enters the solve)
    oc0 = oracle.make_cfg(dim=dim, order=order, res=(res,) * dim, dx=sc.dx, dt=oc.dt)
    gm, gmv, _, _ = oracle.p2g(oc0, x0, v0, B0, F0, m, vol)
    assert relerr(mv_g, gmv) <= (1e-11 if prec == 64 else 1e-5)
    sim.grid_update()
    st = sim.solve_stats()
    _, vt_g = sim.grid("velocity")
    gv = np.where(m_g[:, None] > 0, mv_g / np.where(m_g > 0, m_g, 1.0)[:, None], 0.0)
    dv, it = oracle.midpoint_solve(oc, x0, F0, vol, m_g, gv, newton=20, cg=400, tol=1e-13)
    assert it >= 1 and st["newton"] >= 1 and st["cg"] >= 1
    tol = 1e-9 if prec == 64 else 1e-5
    assert relerr(vt_g, gv + dv) <= tol
    if prec == 64:   # the change alone (in FP32 it is a small difference of rounded velocities)
        assert relerr(vt_g - gv, dv) <= 1e-8
    assert st["residual"] <= (1e-12 if prec == 64 else 1e-5)
    sim.close()


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_midpoint_step_matches_oracle(apic, case):
    dim, order, prec, res, ppc, mdl = case
    sim, sc, oc, m, vol = setup(apic, case, seed=2)
    x0, v0, B0, F0 = sim.download()
    sim.step(1)
    gx, gv, gB, gF = sim.download()
    ox, ov, oB, oF, bad = oracle.step_midpoint(oc, x0, v0, B0, F0, m, vol, newton=20, cg=400, tol=1e-13)
    assert bad == 0
    tol = 1e-9 if prec == 64 else 1e-5
    assert relerr(gv, ov) <= tol
    assert relerr(gB, oB) <= 10 * tol
    assert relerr(gF, oF) <= tol
    eps = np.finfo(np.float32 if prec == 32 else np.float64).eps
    assert np.abs((gx - x0) - (ox - x0)).max() <= tol * np.abs(ox - x0).max() + 2 * eps * sc.dx + 1e-15
    sim.close()


@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[3]], ids=_ids)
def test_midpoint_conserves_momentum(apic, case):
    """Converged midpoint steps keep p and l (the family's conservation, Sec. 5.2 / 5.3, with
    the velocity-like CG iterates of Sec. 4.2)."""
    dim, order, prec, res, ppc, mdl = case
    sim, sc, oc, m, vol = setup(apic, case, seed=4)
    x, v, B, F = sim.download()
    p0, l0 = sim.momentum("particles")
    sim.step(2)
    p1, l1 = sim.momentum("particles")
    sp = m * np.linalg.norm(v, axis=1).sum()
    sl = m * (np.linalg.norm(x, axis=1) * np.linalg.norm(v, axis=1)).sum() + m * np.abs(B).sum()
    assert np.abs(p1 - p0).max() <= 1e-11 * sp
    assert np.abs(l1 - l0).max() <= 1e-10 * sl
    sim.close()


@pytest.mark.parametrize("dim,order", [(3, 2), (2, 3)])
def test_midpoint_without_forces_is_the_lambda0_step(apic, dim, order):
    case = (dim, order, 64, 16 if dim == 3 else 32, 8 if dim == 3 else 4, "none")
    sim2, sc, oc, m, vol = setup(apic, case, seed=6, model="none")
    x, v, B, F = sim2.download()
    gc0, _, _, _ = configs(dim, order, sc.res, sc.dx, precision=64, dt=4e-3, model="none")
    sim0 = apic.Sim(gc0, len(x))
    sim0.upload(x, v, B, F)
    sim2.step(2)
    sim0.step(2)
    assert sim2.solve_stats()["newton"] == 0           # no force: converged before the first system
    for u, w in zip(sim2.download(), sim0.download()):
        assert relerr(u, w) <= 1e-12
    sim2.close()
    sim0.close()


def test_midpoint_rejects_gravity_and_walls(apic):
    base = dict(dim=3, order=2, res=(16,) * 3, dx=1 / 16, integrator=2, model="fcr", E=1e4, nu=0.3)
    for extra in (dict(gravity=(0.0, -9.8, 0.0)), dict(boundary="sticky", wall=3), dict(transfer="flip")):
        with pytest.raises(apic.ApicError) as e:
            apic.Sim(apic.make_config(**base, **extra), 10)
        assert e.value.status == apic.APIC_ERR_UNSUPPORTED
