"""A material per particle on the GPU: two materials in one
body (soft half, stiff half) against the oracle with per-particle Lame parameters --
the P2G force alone (v = B = 0, so the grid momentum is dt f), then several whole steps --
in 3-D FP32 and 2-D cubic FP64; uniform per-particle values against the configuration's
material; a batch member with materials against the same simulation alone; and the
argument checks."""
import numpy as np
import pytest

import oracle
from helpers import configs, kappa, relerr
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


def _materials(x):
    soft = x[:, 0] < 0.5
    return np.where(soft, 1e3, 3e4), np.where(soft, 0.3, 0.42)


CASES = [(3, 2, 32, 32, 8, "fcr"), (3, 2, 32, 32, 8, "nh"), (2, 3, 64, 64, 4, "fcr")]


@pytest.mark.parametrize("dim,order,prec,res,ppc,model", CASES)
def test_mixed_material_force_matches_oracle(apic, dim, order, prec, res, ppc, model):
    sc = _scene(dim, res, ppc, seed=5)
    rng = np.random.default_rng(5)
    n = sc.n
    F = scenes.random_deformation(rng, n, dim, 0.1)
    gc, oc, m, vol = configs(dim, order, (res,) * dim, sc.dx, precision=prec, dt=2e-3, model=model)
    E, nu = _materials(sc.x)
    sim = apic.Sim(gc, n)
    sim.upload(sc.x, np.zeros((n, dim)), np.zeros((n, dim, dim)), F)
    sim.upload_materials(E, nu)
    x0, _, _, F0 = sim.download()
    sim.p2g()
    gm, gp = sim.grid("momentum")
    sim.close()
    mu, lam = oracle.lame(E, nu)
    om, omv, of, bad = oracle.p2g(oc, x0, np.zeros((n, dim)), np.zeros((n, dim, dim)), F0, m, vol, mu=mu, lam=lam)
    assert bad == 0
    assert relerr(gm, om) <= TOL[prec]
    assert relerr(gp, oc.dt * of) <= (2e-5 if prec == 32 else TOL[prec])
    # with the configuration's single material the force differs: the materials were used
    _, _, of1, _ = oracle.p2g(oc, x0, np.zeros((n, dim)), np.zeros((n, dim, dim)), F0, m, vol)
    assert relerr(oc.dt * of1, oc.dt * of) > 0.1


@pytest.mark.parametrize("dim,order,prec,res,ppc,model", CASES[:1] + CASES[2:])
def test_mixed_material_steps_match_oracle(apic, dim, order, prec, res, ppc, model):
    sc = _scene(dim, res, ppc, seed=6)
    rng = np.random.default_rng(6)
    n = sc.n
    B = sc.grad_v * kappa(order) * sc.dx ** 2
    F = scenes.random_deformation(rng, n, dim, 0.05)
    gc, oc, m, vol = configs(dim, order, (res,) * dim, sc.dx, precision=prec, dt=2e-4, model=model)
    E, nu = _materials(sc.x)
    mu, lam = oracle.lame(E, nu)
    sim = apic.Sim(gc, n)
    sim.upload(sc.x, sc.v, B, F)
    sim.upload_materials(E, nu)
    state = sim.download()
    for step in range(4):
        sim.step(1)
        got = sim.download()
        ox, ov, oB, oF, bad = oracle.step(oc, *state, m, vol, mu=mu, lam=lam)
        assert bad == 0
        gx, gv, gB, gF = got
        assert relerr(gv, ov) <= TOL[prec], f"step {step}"
        assert relerr(gB, oB) <= (1e-4 if prec == 32 else TOL[prec]), f"step {step}"
        assert relerr(gF, oF) <= TOL[prec], f"step {step}"
        assert np.abs(gx - ox).max() <= (1e-5 if prec == 32 else 1e-12) * sc.dx, f"step {step}"
        state = got
    sim.close()


def test_uniform_materials_equal_the_configuration(apic):
    sc = _scene(3, 32, 8, seed=7)
    rng = np.random.default_rng(7)
    n = sc.n
    B = sc.grad_v * kappa(2) * sc.dx ** 2
    F = scenes.random_deformation(rng, n, 3, 0.05)
    gc, oc, m, vol = configs(3, 2, (32,) * 3, sc.dx, dt=2e-4, model="fcr", E=2e3, nu=0.35)
    out = []
    for with_mat in (False, True):
        sim = apic.Sim(gc, n)
        sim.upload(sc.x, sc.v, B, F)
        if with_mat:
            sim.upload_materials(2e3, 0.35)
        sim.step(3)
        out.append(sim.download())
        sim.close()
    # the same arithmetic; runs differ only by the order of the grid's global adds
    for a, b in zip(out[0], out[1]):
        assert relerr(b, a) <= 1e-5


def test_batch_member_with_materials_equals_alone(apic):
    members = []
    for seed in (8, 9):
        sc = _scene(3, 32, 8, seed=seed)
        gc, oc, m, vol = configs(3, 2, (32,) * 3, sc.dx, dt=2e-4, model="fcr")
        members.append((gc, sc))
    alone = []
    for gc, sc in members:
        sim = apic.Sim(gc, sc.n)
        sim.upload(sc.x, sc.v)
        sim.upload_materials(*_materials(sc.x))
        sim.step(3)
        alone.append(sim.download())
        sim.close()
    batch = apic.Batch(dim=3, order=2, max_sims=2, max_particles=400000, max_blocks=100000)
    sims = []
    for gc, sc in members:
        sim = apic.Sim(gc, sc.n)
        sim.upload(sc.x, sc.v)
        sim.upload_materials(*_materials(sc.x))
        batch.add(sim)
        sims.append(sim)
    batch.step(3)
    for sim, ref in zip(sims, alone):
        got = sim.download()
        for g, r in zip(got[1:], ref[1:]):
            assert relerr(g, r) <= 1e-5
        assert np.abs(got[0] - ref[0]).max() <= 1e-6
    batch.close()


def test_material_arguments_are_checked(apic):
    sc = _scene(3, 32, 8, seed=10)
    gc, *_ = configs(3, 2, (32,) * 3, sc.dx, dt=2e-4, model="fcr")
    sim = apic.Sim(gc, sc.n + 10)
    sim.upload(sc.x)
    with pytest.raises(apic.ApicError):
        apic.apic_upload_materials(sim.handle, sc.n + 1, np.full(sc.n + 1, 1e3), np.full(sc.n + 1, 0.3))
    with pytest.raises(apic.ApicError):
        sim.upload_materials(1e3, 0.5)          # nu = 0.5 has no finite lambda
    with pytest.raises(apic.ApicError):
        sim.upload_materials(-1.0, 0.3)
    sim.upload_materials(1e3, 0.3)
    sim.step(1)
    sim.download()
    sim.close()
