"""A mass and a volume per particle on the GPU (apic_upload_mass_volume): m_p in the grid
mass and the affine momentum of Sec. 3.2, V_p in the force of Sec. 3.3, against the oracle
given the same per-particle values --
- P2G with both P2G kernels, 2-D and 3-D, quadratic and cubic, FP32 and FP64;
- whole steps;
- the momentum diagnostics (Sec. 5.2, 5.3) against the oracle's sums;
- together with a material per particle (either call first), and the reset by apic_upload;
- a batch member against the oracle;
- the lambda = 1 and midpoint members;
- the argument checks.
The values are drawn in [0.5, 2] times the configuration's and rounded to FP32, so an FP32
simulation stores them exactly and both sides use the same numbers."""
import numpy as np
import pytest

import oracle
from helpers import configs, kappa, nodewise_err, relerr, state_for
from paper_1603_06188_gb300 import scenes

pytestmark = pytest.mark.gpu
TOL = {32: 1e-5, 64: 1e-11}


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


def _mass_volume(n, m, vol, seed):
    rng = np.random.default_rng(1000 + seed)
    mass = (m * rng.uniform(0.5, 2.0, n)).astype(np.float32).astype(np.float64)
    V = (vol * rng.uniform(0.5, 2.0, n)).astype(np.float32).astype(np.float64)
    return mass, V


P2G_CASES = [
    # dim, order, precision, res, ppc, model, p2g_kernel
    (3, 2, 32, 32, 8, "fcr", 2),
    (3, 2, 32, 32, 8, "fcr", 1),
    (3, 3, 32, 32, 8, "nh", 1),
    (3, 3, 32, 32, 8, "fcr", 2),
    (3, 2, 64, 16, 8, "fcr", 0),
    (2, 2, 64, 64, 4, "fcr", 0),
    (2, 3, 32, 64, 4, "nh", 0),
]


def _ids(c):
    return f"d{c[0]}_o{c[1]}_fp{c[2]}_{c[5]}_k{c[6]}"


@pytest.mark.parametrize("case", P2G_CASES, ids=_ids)
def test_p2g_with_particle_mass_and_volume_matches_oracle(apic, case):
    dim, order, prec, res, ppc, model, kern = case
    sc = _scene(dim, res, ppc, seed=3)
    x, v, B, F = state_for(sc, order, seed=3, Fscale=0.1)
    gc, oc, m, vol = configs(dim, order, (res,) * dim, sc.dx, precision=prec, dt=2e-3, model=model, p2g_kernel=kern)
    mass, V = _mass_volume(sc.n, m, vol, 3)
    sim = apic.Sim(gc, sc.n)
    sim.upload(x, v, B, F)
    sim.upload_mass_volume(mass, V)
    x0, v0, B0, F0 = sim.download()
    sim.p2g()
    gm, gp = sim.grid("momentum")
    sim.close()
    om, omv, of, bad = oracle.p2g(oc, x0, v0, B0, F0, mass, V)
    assert bad == 0
    ref = omv + oc.dt * of
    assert relerr(gm, om) <= TOL[prec]
    assert relerr(gp, ref) <= TOL[prec]
    assert nodewise_err(gm[:, None], om[:, None], om) <= 10 * TOL[prec]
    assert nodewise_err(gp, ref, om) <= 10 * TOL[prec]
    # the configuration's uniform values give a different grid: the particle values were used
    om1, omv1, of1, _ = oracle.p2g(oc, x0, v0, B0, F0, m, vol)
    assert relerr(om1, om) > 0.05
    assert relerr(omv1 + oc.dt * of1, ref) > 0.05


STEP_CASES = [(3, 2, 32, 32, 8, "fcr", 0), (3, 3, 32, 32, 8, "nh", 0), (2, 3, 64, 64, 4, "fcr", 0)]


@pytest.mark.parametrize("case", STEP_CASES, ids=_ids)
def test_steps_with_particle_mass_and_volume_match_oracle(apic, case):
    dim, order, prec, res, ppc, model, kern = case
    sc = _scene(dim, res, ppc, seed=4)
    rng = np.random.default_rng(4)
    n = sc.n
    B = sc.grad_v * kappa(order) * sc.dx ** 2
    F = scenes.random_deformation(rng, n, dim, 0.05)
    gc, oc, m, vol = configs(dim, order, (res,) * dim, sc.dx, precision=prec, dt=2e-4, model=model,
                             gravity=(0.0, -9.8, 0.0)[:dim], boundary="sticky", wall=3)
    mass, V = _mass_volume(n, m, vol, 4)
    sim = apic.Sim(gc, n)
    sim.upload(sc.x, sc.v, B, F)
    sim.upload_mass_volume(mass, V)
    state = sim.download()
    for step in range(3):
        sim.step(1)
        got = sim.download()
        ox, ov, oB, oF, bad = oracle.step(oc, *state, mass, V)
        assert bad == 0
        gx, gv, gB, gF = got
        assert relerr(gv, ov) <= TOL[prec], f"step {step}"
        assert relerr(gB, oB) <= (1e-4 if prec == 32 else TOL[prec]), f"step {step}"
        assert relerr(gF, oF) <= TOL[prec], f"step {step}"
        assert np.abs(gx - ox).max() <= (1e-5 if prec == 32 else 1e-12) * sc.dx, f"step {step}"
        state = got
    sim.close()


@pytest.mark.parametrize("dim,order", [(3, 2), (2, 3)])
def test_momentum_diagnostics_use_particle_mass(apic, dim, order):
    """apic_momentum after upload (particles) and after P2G (grid) against the oracle's FP64
    sums with the same per-particle masses (the force is off, so the grid sums equal the
    particle sums, Sec. 5.2, 5.3)."""
    res, ppc = (32, 8) if dim == 3 else (64, 4)
    sc = _scene(dim, res, ppc, seed=5)
    x, v, B, F = state_for(sc, order, seed=5)
    gc, oc, m, vol = configs(dim, order, (res,) * dim, sc.dx, precision=32, dt=1e-3, model="none")
    mass, V = _mass_volume(sc.n, m, vol, 5)
    sim = apic.Sim(gc, sc.n)
    sim.upload(x, v, B, F)
    sim.upload_mass_volume(mass, V)
    x0, v0, B0, _ = sim.download()
    p, l = sim.momentum("particles")
    op, ol = oracle.momentum_particles(oc, x0, v0, B0, mass)
    scale_p = np.sum(mass * np.linalg.norm(v0, axis=1))
    scale_l = np.sum(mass * (np.linalg.norm(x0, axis=1) * np.linalg.norm(v0, axis=1)
                             + np.abs(B0).reshape(len(B0), -1).sum(axis=1)))
    assert np.abs(np.asarray(p) - op).max() <= 1e-12 * scale_p
    assert np.abs(np.asarray(l) - ol).max() <= 1e-12 * scale_l
    sim.p2g()
    pg, lg = sim.momentum("grid")
    assert np.abs(np.asarray(pg) - op).max() <= 1e-5 * scale_p
    assert np.abs(np.asarray(lg) - ol).max() <= 1e-5 * scale_l
    sim.close()


def test_materials_and_mass_volume_combine_in_either_order(apic):
    sc = _scene(3, 32, 8, seed=6)
    x, v, B, F = state_for(sc, 2, seed=6, Fscale=0.1)
    gc, oc, m, vol = configs(3, 2, (32,) * 3, sc.dx, dt=2e-3, model="fcr")
    mass, V = _mass_volume(sc.n, m, vol, 6)
    soft = sc.x[:, 0] < 0.5
    E, nu = np.where(soft, 1e3, 3e4), np.where(soft, 0.3, 0.42)
    mu, lam = oracle.lame(E, nu)
    grids = []
    for first_materials in (True, False):
        sim = apic.Sim(gc, sc.n)
        sim.upload(x, v, B, F)
        if first_materials:
            sim.upload_materials(E, nu)
            sim.upload_mass_volume(mass, V)
        else:
            sim.upload_mass_volume(mass, V)
            sim.upload_materials(E, nu)
        x0, v0, B0, F0 = sim.download()
        sim.p2g()
        grids.append(sim.grid("momentum"))
        sim.close()
    om, omv, of, _ = oracle.p2g(oc, x0, v0, B0, F0, mass, V, mu=mu, lam=lam)
    for gm, gp in grids:
        assert relerr(gm, om) <= 1e-5
        assert relerr(gp, omv + oc.dt * of) <= 2e-5


def test_upload_returns_to_the_configuration(apic):
    sc = _scene(3, 32, 8, seed=7)
    x, v, B, F = state_for(sc, 2, seed=7)
    gc, oc, m, vol = configs(3, 2, (32,) * 3, sc.dx, dt=2e-3, model="fcr")
    mass, V = _mass_volume(sc.n, m, vol, 7)
    sim = apic.Sim(gc, sc.n)
    sim.upload(x, v, B, F)
    sim.upload_mass_volume(mass, V)
    sim.upload(x, v, B, F)
    x0, v0, B0, F0 = sim.download()
    sim.p2g()
    gm, gp = sim.grid("momentum")
    sim.close()
    om, omv, of, _ = oracle.p2g(oc, x0, v0, B0, F0, m, vol)
    assert relerr(gm, om) <= 1e-5
    assert relerr(gp, omv + oc.dt * of) <= 1e-5


@pytest.mark.parametrize("group", [0, 2])
def test_batch_member_with_particle_mass_matches_oracle(apic, group):
    """Two members, one with per-particle mass and volume, stepped together; each against
    the oracle after two batched steps (group 0: the batch's default P2G kernel)."""
    members = []
    for seed in (8, 9):
        sc = _scene(3, 32, 8, seed=seed)
        x, v, B, F = state_for(sc, 2, seed=seed, Fscale=0.05)
        gc, oc, m, vol = configs(3, 2, (32,) * 3, sc.dx, dt=2e-4, model="fcr")
        mv = _mass_volume(sc.n, m, vol, seed) if seed == 8 else (np.full(sc.n, m), np.full(sc.n, vol))
        members.append((gc, oc, sc, (x, v, B, F), mv))
    kw = {} if group == 0 else {"group": group}
    batch = apic.Batch(dim=3, order=2, max_sims=2, max_particles=400000, max_blocks=100000, **kw)
    sims = []
    for (gc, oc, sc, st, (mass, V)), seed in zip(members, (8, 9)):
        sim = apic.Sim(gc, sc.n)
        sim.upload(*st)
        if seed == 8:
            sim.upload_mass_volume(mass, V)
        sims.append((sim, sim.download()))
        batch.add(sim)
    batch.step(2)
    for (sim, st0), (gc, oc, sc, _, (mass, V)) in zip(sims, members):
        got = sim.download()
        ox, ov, oB, oF, bad = oracle.step(oc, *st0, mass, V, nsteps=2)
        assert bad == 0
        assert relerr(got[1], ov) <= 1e-5
        assert relerr(got[3], oF) <= 1e-5
        assert np.abs(got[0] - ox).max() <= 1e-5 * sc.dx
    batch.close()
    for sim, _ in sims:
        sim.close()


@pytest.mark.parametrize("integrator", [1, 2])
def test_lambda1_and_midpoint_with_particle_mass_match_oracle(apic, integrator):
    sc = _scene(3, 16, 8, seed=10)
    x, v, B, F = state_for(sc, 2, seed=10, Fscale=0.1)
    gc, oc, m, vol = configs(3, 2, (16,) * 3, sc.dx, precision=64, dt=2e-3, model="fcr", mass=1.0,
                             vol=sc.dx ** 3 / 8)
    gc.integrator = integrator
    if integrator == 2:
        gc.solve_tol, gc.newton_max, gc.cg_max = 1e-13, 20, 400
    mass, V = _mass_volume(sc.n, m, vol, 10)
    sim = apic.Sim(gc, sc.n)
    sim.upload(x, v, B, F)
    sim.upload_mass_volume(mass, V)
    st0 = sim.download()
    sim.step(1)
    gx, gv, gB, gF = sim.download()
    sim.close()
    if integrator == 1:
        ox, ov, oB, oF, bad = oracle.step_lambda1(oc, *st0, mass, V)
        tol = 1e-11
    else:
        ox, ov, oB, oF, bad = oracle.step_midpoint(oc, *st0, mass, V, newton=20, cg=400, tol=1e-13)
        tol = 1e-9
    assert bad == 0
    assert relerr(gv, ov) <= tol
    assert relerr(gB, oB) <= 10 * tol
    assert relerr(gF, oF) <= tol


def test_mass_volume_argument_checks(apic):
    sc = _scene(3, 16, 8, seed=11)
    gc, _, m, vol = configs(3, 2, (16,) * 3, sc.dx)
    sim = apic.Sim(gc, sc.n)
    sim.upload(sc.x, sc.v)
    n = sc.n
    good = np.full(n, m)
    for mass, V in ((np.full(n, -1.0), np.full(n, vol)), (good, np.zeros(n)),
                    (np.where(np.arange(n) == 3, np.nan, m), np.full(n, vol))):
        with pytest.raises(apic.ApicError) as e:
            apic.apic_upload_mass_volume(sim.handle, n, np.ascontiguousarray(mass), np.ascontiguousarray(V))
        assert e.value.status == apic.APIC_ERR_ARG
    with pytest.raises(apic.ApicError) as e:
        apic.apic_upload_mass_volume(sim.handle, n - 1, good[:-1].copy(), np.full(n - 1, vol))
    assert e.value.status == apic.APIC_ERR_ARG
    sim.p2g()
    with pytest.raises(apic.ApicError) as e:   # between P2G and G2P
        sim.upload_mass_volume(m, vol)
    assert e.value.status == apic.APIC_ERR_ARG
    sim.close()
