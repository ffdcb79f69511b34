"""CUDA path (through the C ABI) against the FP64 oracle, one transfer at a time, the
oracle always fed the GPU's exact input state (FP32 values widened to FP64).

Bars: cell keys, sort permutation and grid occupancy bit-exact; grid momentum, grid
velocity, v_p, B_p, F_p and the displacement within 1e-5 normwise relative
(||gpu - oracle||_inf / ||oracle||_inf) in FP32 and 1e-11 in FP64."""
import numpy as np
import pytest

import oracle
from helpers import (E_DEFAULT, NU_DEFAULT, configs, kappa, nodewise_err, occupancy_rule, particlewise_err, relerr,
                     state_for, stencil_max_speed)
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


def cube_scene(dim, res, ppc, seed=0, side=0.5):
    if dim == 3:
        return scenes.falling_cube_3d(res=res, side=side, ppc=ppc, seed=seed, omega=(0.5, -1.0, 2.0), v0=(0.3, 0.1, -0.2))
    return scenes.rotating_disk_2d(res=res, radius=side / 2, ppc=ppc, seed=seed, omega=2.0)


CASES = [
    # dim, order, precision, res, ppc
    (3, 2, 32, 32, 8),
    (3, 3, 32, 32, 8),
    (2, 2, 32, 64, 4),
    (2, 3, 32, 64, 4),
    (3, 2, 64, 24, 8),
    (3, 3, 64, 24, 8),
    (2, 2, 64, 64, 4),
    (2, 3, 64, 64, 4),
]


def _ids(c):
    return f"d{c[0]}_o{c[1]}_fp{c[2]}_r{c[3]}"


def run_one_step(apic, dim, order, prec, res, ppc, model="fcr", transfer="apic", dt=2e-3, gravity=None,
                 boundary="none", wall=0, tile=0, seed=0, p2g_kernel=0, p2g_group=0):
    sc = cube_scene(dim, res, ppc, seed=seed)
    x, v, B, F = state_for(sc, order, seed=seed)
    g = gravity if gravity is not None else (0.0,) * dim
    gc, oc, m, vol = configs(dim, order, (res,) * dim, sc.dx, precision=prec, transfer=transfer, dt=dt,
                             gravity=g, boundary=boundary, wall=wall, model=model, tile=tile, p2g_kernel=p2g_kernel,
                             p2g_group=p2g_group)
    sim = apic.Sim(gc, len(x) + 7)
    sim.upload(x, v, B, F)
    x0, v0, B0, F0 = sim.download()          # the GPU's exact input state
    cell0, off0 = sim.download_positions()
    out = {"sim": sim, "sc": sc, "oc": oc, "m": m, "vol": vol, "in": (x0, v0, B0, F0), "cell": cell0, "off": off0}
    sim.p2g()
    out["keys"], out["perm"] = sim.keys()
    out["occ"] = sim.occupancy()
    out["grid_p2g"] = sim.grid("momentum")
    out["mom_grid_p2g"] = sim.momentum("grid")
    sim.grid_update()
    out["grid_vel"] = sim.grid("velocity")
    out["mom_grid_vel"] = sim.momentum("grid")
    sim.g2p()
    out["out"] = sim.download()
    out["mom_particles_g2p"] = sim.momentum("particles")
    out["stats"] = sim.stats()
    return out


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_keys_sort_occupancy_bit_exact(apic, case):
    dim, order, prec, res, ppc = case
    r = run_one_step(apic, dim, order, prec, res, ppc)
    oc = r["oc"]
    ref_keys = oracle.keys(oc, 4, r["cell"], r["off"])
    ref_perm = oracle.stable_sort(ref_keys)
    np.testing.assert_array_equal(r["keys"], ref_keys[ref_perm])
    np.testing.assert_array_equal(r["perm"].astype(np.int64), ref_perm)
    np.testing.assert_array_equal(r["occ"], occupancy_rule(ref_keys, dim, (res,) * dim))
    assert r["stats"]["tiles"] >= 2


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_p2g_matches_oracle(apic, case):
    dim, order, prec, res, ppc = case
    r = run_one_step(apic, dim, order, prec, res, ppc)
    x0, v0, B0, F0 = r["in"]
    gm, gmv, gf, bad = oracle.p2g(r["oc"], x0, v0, B0, F0, r["m"], r["vol"])
    assert bad == 0
    m_gpu, p_gpu = r["grid_p2g"]
    ref_p = gmv + r["oc"].dt * gf
    assert relerr(m_gpu, gm) <= TOL[prec]
    assert relerr(p_gpu, ref_p) <= TOL[prec]
    # node occupancy by mass is the same set
    np.testing.assert_array_equal(m_gpu > 0, gm > 0)
    # and node by node against each node's own scale (tighter than normwise where mass is small)
    assert nodewise_err(m_gpu, gm, gm) <= TOL[prec]
    assert nodewise_err(p_gpu, ref_p, gm) <= TOL[prec]


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_grid_update_matches_oracle(apic, case):
    dim, order, prec, res, ppc = case
    r = run_one_step(apic, dim, order, prec, res, ppc, gravity=(0.0, -9.8, 0.0)[:dim], boundary="sticky",
                     wall=order + 1)
    m_gpu, p_gpu = r["grid_p2g"]
    _, vt_ref = oracle.grid_update(r["oc"], m_gpu, p_gpu, np.zeros_like(p_gpu))
    m2, vt_gpu = r["grid_vel"]
    np.testing.assert_array_equal(m2, m_gpu)
    assert relerr(vt_gpu, vt_ref) <= TOL[prec]


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_g2p_matches_oracle(apic, case):
    dim, order, prec, res, ppc = case
    r = run_one_step(apic, dim, order, prec, res, ppc)
    x0, v0, B0, F0 = r["in"]
    _, vt = r["grid_vel"]
    x1, v1, B1, F1, bad = oracle.g2p(r["oc"], x0, F0, vt, vt)
    assert bad == 0
    gx, gv, gB, gF = r["out"]
    tol = TOL[prec]
    assert relerr(gv, v1) <= tol
    assert relerr(gB, B1) <= tol
    assert relerr(gF, F1) <= tol
    assert relerr(gF - F0, F1 - F0) <= 10 * tol
    assert relerr(gx - x0, x1 - x0) <= tol
    # particle by particle against the largest grid speed its stencil sees: v_p and B_p of a
    # particle in a slow region must be as accurate as those in a fast one
    smax = stencil_max_speed(x0, vt, (res,) * dim, r["oc"].dx, order)
    assert particlewise_err(gv, v1, smax) <= tol
    assert particlewise_err(gB, B1, smax * r["oc"].dx) <= tol


@pytest.mark.parametrize("transfer", ["apic", "pic"])
def test_transfer_modes_and_transfer_only(apic, transfer):
    r = run_one_step(apic, 3, 2, 32, 32, 8, model="none", transfer=transfer)
    x0, v0, B0, F0 = r["in"]
    gm, gmv, gf, _ = oracle.p2g(r["oc"], x0, v0, B0, F0, r["m"], r["vol"])
    m_gpu, p_gpu = r["grid_p2g"]
    assert relerr(p_gpu, gmv) <= 1e-5
    _, vt = r["grid_vel"]
    x1, v1, B1, F1, _ = oracle.g2p(r["oc"], x0, F0, vt, vt)
    gx, gv, gB, gF = r["out"]
    assert relerr(gv, v1) <= 1e-5
    if transfer == "pic":
        assert np.all(gB == 0)
    else:
        assert relerr(gB, B1) <= 1e-5


@pytest.mark.parametrize("tile", [256, 1024, 4096])
@pytest.mark.parametrize("p2g_kernel", [0, 1, 2])
@pytest.mark.parametrize("dim,order,prec", [(3, 2, 32), (2, 2, 32), (2, 3, 32), (3, 2, 64), (2, 3, 64), (3, 3, 32),
                                            (3, 3, 64)])
def test_p2g_kernels_and_tile_sizes_agree(apic, tile, p2g_kernel, dim, order, prec):
    """Both P2G kernels (1: component-split, 3-D only; 2: cell-parallel; 0: the default) at
    every tile size, against the oracle's grid."""
    if p2g_kernel == 1 and dim == 2:
        pytest.skip("the component-split kernel is 3-D only")
    r = run_one_step(apic, dim, order, prec, 32 if dim == 3 else 64, 8 if dim == 3 else 4, tile=tile,
                     p2g_kernel=p2g_kernel)
    x0, v0, B0, F0 = r["in"]
    gm, gmv, gf, _ = oracle.p2g(r["oc"], x0, v0, B0, F0, r["m"], r["vol"])
    assert relerr(r["grid_p2g"][0], gm) <= TOL[prec]
    assert relerr(r["grid_p2g"][1], gmv + r["oc"].dt * gf) <= TOL[prec]
    assert nodewise_err(r["grid_p2g"][1], gmv + r["oc"].dt * gf, gm) <= TOL[prec]


@pytest.mark.parametrize("p2g_group", [0, 2, 4])
@pytest.mark.parametrize("ppc", [8, 32])
@pytest.mark.parametrize("dim,order,prec", [(3, 2, 32), (3, 3, 32), (2, 2, 64)])
def test_p2g_lane_groups_agree(apic, p2g_group, ppc, dim, order, prec):
    """The cell-parallel P2G with two or four lanes per base cell, and the choice made from
    the particle density (0), gives the oracle's grid momentum and the same G2P output."""
    if dim == 2:
        ppc = ppc // 2
    r = run_one_step(apic, dim, order, prec, 24 if dim == 3 else 64, ppc, p2g_group=p2g_group, p2g_kernel=2)
    x0, v0, B0, F0 = r["in"]
    gm, gmv, gf, _ = oracle.p2g(r["oc"], x0, v0, B0, F0, r["m"], r["vol"])
    assert relerr(r["grid_p2g"][0], gm) <= TOL[prec]
    assert relerr(r["grid_p2g"][1], gmv + r["oc"].dt * gf) <= TOL[prec]
    _, vt = r["grid_vel"]
    _, v1, B1, _, _ = oracle.g2p(r["oc"], x0, F0, vt, vt)
    gx, gv, gB, gF = r["out"]
    assert relerr(gv, v1) <= TOL[prec]
    assert relerr(gB, B1) <= TOL[prec]


def test_p2g_group_argument_checked(apic):
    with pytest.raises(apic.ApicError):
        apic.Sim(apic.make_config(dim=3, order=2, res=(16,) * 3, dx=1 / 16, p2g_group=3), 10)


def test_gpu_momentum_conservation_fp32(apic):
    """Sec. 5.2 / 5.3 on the GPU: P2G and G2P keep p and l to FP32 rounding (forces on, no
    gravity, no walls); the FP64 reductions see it."""
    sc = scenes.falling_cube_3d(res=48, side=0.5, ppc=8, omega=(0.0, 0.0, 3.0), v0=(0.2, 0.0, 0.0), seed=3)
    x, v, B, F = state_for(sc, 2, seed=3)
    gc, oc, m, vol = configs(3, 2, (48,) * 3, sc.dx, dt=1e-3)
    sim = apic.Sim(gc, len(x))
    sim.upload(x, v, B, F)
    p0, l0 = sim.momentum("particles")
    sim.p2g()
    pg, lg = sim.momentum("grid")
    sim.grid_update()
    sim.g2p()
    p1, l1 = sim.momentum("particles")
    sp = m * np.linalg.norm(v, axis=1).sum()
    sl = m * (np.linalg.norm(x, axis=1) * np.linalg.norm(v, axis=1)).sum() + m * np.abs(B).sum()
    assert np.abs(pg - p0).max() <= 1e-5 * sp
    assert np.abs(lg - l0).max() <= 1e-5 * sl
    assert np.abs(p1 - p0).max() <= 1e-5 * sp
    assert np.abs(l1 - l0).max() <= 1e-5 * sl


def test_gpu_fp64_disk_round_trips_conserve_to_1e12(apic):
    """2-D FP64 rotating disk (64^2, dx = 1/64, 4 ppc, omega = 1, v0 = (0.1, 0)), transfer only,
    100 P2G -> G2P round trips at dt = 5e-3: p and l conserved to 1e-12 relative, and the
    trajectory matches the oracle's.  (Without forces the particles move ballistically, so
    at dt = 1e-2 the disk would leave the unit box before step 100.)"""
    sc = scenes.rotating_disk_2d(res=64, ppc=4, seed=0)
    k = kappa(2) * sc.dx ** 2
    B = sc.grad_v * k
    gc, oc, m, vol = configs(2, 2, (64, 64), sc.dx, precision=64, dt=5e-3, model="none")
    sim = apic.Sim(gc, sc.n)
    sim.upload(sc.x, sc.v, B, None)
    p0, l0 = sim.momentum("particles")
    sim.step(100)
    p1, l1 = sim.momentum("particles")
    sp = np.linalg.norm(sc.v, axis=1).sum()
    sl = (np.linalg.norm(sc.x, axis=1) * np.linalg.norm(sc.v, axis=1)).sum() + np.abs(B).sum()
    assert np.abs(p1 - p0).max() <= 1e-12 * sp
    assert np.abs(l1 - l0).max() <= 1e-12 * sl
    gx, gv, gB, gF = sim.download()
    ox, ov, oB, oF, bad = oracle.step(oc, sc.x, sc.v, B, np.broadcast_to(np.eye(2), (sc.n, 2, 2)), 1.0, vol, nsteps=100)
    assert bad == 0
    assert relerr(gv, ov) <= 1e-9
    assert relerr(gx - sc.x, ox - sc.x) <= 1e-9


def test_gpu_affine_round_trip(apic):
    """Sec. 5.5 on the GPU at dt = 0: v_p = c + C x_p, B_p = C D_p are reproduced."""
    sc = scenes.falling_cube_3d(res=32, side=0.5, ppc=8, seed=4)
    rng = np.random.default_rng(4)
    c = rng.normal(size=3)
    Cm = rng.normal(size=(3, 3))
    v = c + sc.x @ Cm.T
    B = np.broadcast_to(Cm * kappa(2) * sc.dx ** 2, (sc.n, 3, 3)).copy()
    gc, oc, m, vol = configs(3, 2, (32,) * 3, sc.dx, dt=0.0, model="none")
    sim = apic.Sim(gc, sc.n)
    sim.upload(sc.x, v, B)
    sim.step(1)
    gx, gv, gB, gF = sim.download()
    # FP32 bound: the grid velocity carries an absolute rounding error ~eps |v|, and
    # B = dx sum w v~ r^ is smaller than |v| dx by the factor |B| / (|v| dx)
    eps = np.finfo(np.float32).eps
    assert relerr(gv, v) <= 16 * eps
    assert relerr(gB, B) <= 16 * eps * np.abs(v).max() * sc.dx / np.abs(B).max()
    assert np.abs(gx - sc.x).max() <= 1e-6 * sc.dx


def test_gpu_single_particle_stability(apic):
    """Sec. 5.4: one isolated particle keeps v_p and B_p and moves by dt v_p."""
    rng = np.random.default_rng(5)
    x = np.array([[0.43, 0.51, 0.57]])
    v = rng.normal(size=(1, 3))
    B = 1e-4 * rng.normal(size=(1, 3, 3))
    gc, oc, m, vol = configs(3, 3, (32,) * 3, 1 / 32, dt=1e-3, model="none")
    sim = apic.Sim(gc, 1)
    sim.upload(x, v, B)
    sim.step(3)
    gx, gv, gB, gF = sim.download()
    # FP32 bound per step as in the affine test: B is |v| dx / |B| times smaller than the
    # velocities it is summed from
    eps = np.finfo(np.float32).eps
    assert relerr(gv, v) <= 3 * 16 * eps
    assert relerr(gB, B) <= 3 * 16 * eps * np.abs(v).max() / 32 / np.abs(B).max()
    np.testing.assert_allclose(gx, x + 3e-3 * v, atol=1e-6 / 32)


def test_empty_and_single_cell_edge_cases(apic):
    gc, oc, m, vol = configs(3, 2, (16,) * 3, 1 / 16, dt=1e-3)
    sim = apic.Sim(gc, 5000)
    sim.upload(np.zeros((0, 3)))
    sim.step(2)
    p, l = sim.momentum("particles")
    assert np.all(p == 0) and np.all(l == 0)
    # every particle in one cell: a single long segment in P2G
    rng = np.random.default_rng(6)
    x = (8 + rng.random((5000, 3))) / 16
    v = rng.normal(size=(5000, 3))
    sim.upload(x, v)
    x0, v0, B0, F0 = sim.download()
    sim.p2g()
    m_gpu, p_gpu = sim.grid("momentum")
    gm, gmv, gf, _ = oracle.p2g(oc, x0, v0, B0, F0, m, vol)
    assert relerr(m_gpu, gm) <= 1e-5
    assert relerr(p_gpu, gmv + oc.dt * gf) <= 1e-5


def test_out_of_grid_particle_is_reported(apic):
    gc, oc, m, vol = configs(3, 2, (16,) * 3, 1 / 16, dt=1e-3)
    sim = apic.Sim(gc, 10)
    with pytest.raises(apic.ApicError) as e:
        sim.upload(np.array([[0.5, 0.5, 0.5], [1.5, 0.5, 0.5]]))
    assert e.value.status == apic.APIC_ERR_NUMERIC
    # the clamp keeps the step memory-safe; the condition is reported again by the step
    sim.step(1)
    with pytest.raises(apic.ApicError):
        sim.download()


@pytest.mark.parametrize("dim,order,prec", [(3, 2, 32), (3, 3, 32), (2, 2, 64)])
def test_neohookean_and_slip_walls(apic, dim, order, prec):
    """The Neo-Hookean stress in P2G and slip walls in the grid update, one transfer at a time."""
    res = 32 if dim == 3 else 64
    r = run_one_step(apic, dim, order, prec, res, 8 if dim == 3 else 4, model="nh", boundary="slip", wall=order + 1,
                     gravity=(0.0, -9.8, 0.0)[:dim])
    x0, v0, B0, F0 = r["in"]
    gm, gmv, gf, _ = oracle.p2g(r["oc"], x0, v0, B0, F0, r["m"], r["vol"])
    m_gpu, p_gpu = r["grid_p2g"]
    assert relerr(p_gpu, gmv + r["oc"].dt * gf) <= TOL[prec]
    _, vt_ref = oracle.grid_update(r["oc"], m_gpu, p_gpu, np.zeros_like(p_gpu))
    assert relerr(r["grid_vel"][1], vt_ref) <= TOL[prec]
    _, vt = r["grid_vel"]
    x1, v1, B1, F1, _ = oracle.g2p(r["oc"], x0, F0, vt, vt)
    gx, gv, gB, gF = r["out"]
    assert relerr(gv, v1) <= TOL[prec] and relerr(gF, F1) <= TOL[prec]


@pytest.mark.parametrize("dim,order,prec", [(3, 2, 32), (2, 3, 64)])
def test_cfl_speed_matches_oracle(apic, dim, order, prec):
    """Sec. 4.3 bound max_p(|v_p| + 6 sqrt(d)/dx |B_p|_F) from the device reduction."""
    sc = cube_scene(dim, 32 if dim == 3 else 64, 8 if dim == 3 else 4, seed=5)
    x, v, B, F = state_for(sc, order, seed=5)
    gc, oc, m, vol = configs(dim, order, sc.res, sc.dx, precision=prec)
    sim = apic.Sim(gc, sc.n)
    sim.upload(x, v, B, F)
    _, v0, B0, _ = sim.download()
    got = sim.cfl_speed()
    ref = oracle.cfl_speed(oc, v0, B0)
    assert got == pytest.approx(ref, rel=1e-6 if prec == 32 else 1e-12)


MOM_CASES = [(3, 2, 32), (3, 3, 32), (2, 2, 32), (3, 2, 64), (2, 3, 64)]


@pytest.mark.parametrize("dim,order,prec", MOM_CASES, ids=lambda c: str(c))
def test_momentum_reductions_match_oracle(apic, dim, order, prec):
    """apic_momentum against the oracle's momentum of the same state (Sec. 3.1; Sec. 5.3 for
    the particle term m_p (B_p)^T : eps): particles after the upload and after G2P, the grid
    after P2G (sum (m v)_i with the folded force) and after the grid update (sum m_i v~_i).
    Both sides reduce the same FP32 / FP64 values in FP64, so only the order of the sums
    differs: 1e-12 relative to the sum of the terms' magnitudes."""
    res = 24 if dim == 3 else 64
    r = run_one_step(apic, dim, order, prec, res, 8 if dim == 3 else 4, gravity=(0.0, -9.8, 0.0)[:dim])
    oc, m = r["oc"], r["m"]
    x0, v0, B0, F0 = r["in"]
    sim = r["sim"]

    def scales(x, v, B):
        sp = m * np.linalg.norm(v, axis=1).sum()
        sl = m * (np.linalg.norm(x, axis=1) * np.linalg.norm(v, axis=1)).sum() + m * np.abs(B).sum()
        return sp, sl

    # the particles right after an upload of the input state
    gc, _, _, _ = configs(dim, order, (res,) * dim, 1.0 / res, precision=prec, dt=2e-3)
    fresh = apic.Sim(gc, len(x0))
    fresh.upload(x0, v0, B0, F0)
    p_gpu, l_gpu = fresh.momentum("particles")
    p_ref, l_ref = oracle.momentum_particles(oc, x0, v0, B0, m)
    sp, sl = scales(x0, v0, B0)
    assert np.abs(p_gpu - p_ref).max() <= 1e-12 * sp
    assert np.abs(l_gpu - l_ref).max() <= 1e-12 * sl
    fresh.close()
    # the grid after P2G
    m_g, p_g = r["grid_p2g"]
    pg_ref, lg_ref = oracle.momentum_grid(oc, p_g)
    pg_gpu, lg_gpu = r["mom_grid_p2g"]
    # node positions lie in the unit box, so |x_i x (m v)_i| <= 2 |(m v)_i|
    sgp = np.abs(p_g).sum()
    assert np.abs(pg_gpu - pg_ref).max() <= 1e-12 * sgp
    assert np.abs(lg_gpu - lg_ref).max() <= 1e-12 * sgp * 2
    # the grid after the update: sum m_i v~_i
    m_v, vt = r["grid_vel"]
    pv_ref, lv_ref = oracle.momentum_grid(oc, m_v[:, None] * vt)
    pv_gpu, lv_gpu = r["mom_grid_vel"]
    smv = np.abs(m_v[:, None] * vt).sum()
    assert np.abs(pv_gpu - pv_ref).max() <= 1e-12 * smv
    assert np.abs(lv_gpu - lv_ref).max() <= 1e-12 * smv * 2
    # the particles after G2P
    gx, gv, gB, gF = r["out"]
    p1_ref, l1_ref = oracle.momentum_particles(oc, gx, gv, gB, m)
    p1_gpu, l1_gpu = r["mom_particles_g2p"]
    sp, sl = scales(gx, gv, gB)
    assert np.abs(p1_gpu - p1_ref).max() <= 1e-12 * sp
    assert np.abs(l1_gpu - l1_ref).max() <= 1e-12 * sl
    # and the l term of B is there: the same state without B gives a different l
    if prec == 64:
        l_noB = oracle.momentum_particles(oc, gx, gv, np.zeros_like(gB), m)[1]
        assert np.abs(l_noB - l1_ref).max() > 1e3 * 1e-12 * sl


def _rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def stress_edge_cases(rng, per_case: int):
    """Deformation gradients that take every route of the library's polar decomposition:
    exactly repeated singular values (F = I, F = a rotation, F = U diag(a, a, b) V^T), large
    stretch and near-singular F (the Newton polar iteration), inverted F (det F < 0: the
    Jacobi route, its sign convention R = U V^T with det R = +1 and the smallest singular
    value negated), and inverted F whose two smallest singular values nearly coincide (the
    Jacobi route in FP32 fails its residual check and is redone in FP64)."""
    cases = {
        "identity": lambda: np.eye(3),
        "rotation": lambda: _rotation(rng),
        "repeated": lambda: _rotation(rng) @ np.diag([0.9, 0.9, 1.2]) @ _rotation(rng).T,
        "stretch": lambda: _rotation(rng) @ np.diag([3.0, 0.4, 1.3]) @ _rotation(rng).T,
        "near_singular": lambda: _rotation(rng) @ np.diag([1.1, 0.8, 2e-3]) @ _rotation(rng).T,
        "inverted": lambda: _rotation(rng) @ np.diag([1.2, 0.8, -0.6]) @ _rotation(rng).T,
        "inverted_close": lambda: _rotation(rng) @ np.diag([1.1, 0.5 + 2e-5, -0.5]) @ _rotation(rng).T,
    }
    return {name: np.stack([f() for _ in range(per_case)]) for name, f in cases.items()}


@pytest.mark.parametrize("prec", [32, 64])
def test_stress_edge_cases_match_oracle(apic, prec):
    """The elastic force of P2G (the only place the stress enters a step) for F on every
    route of the polar decomposition, against the oracle's one-sided Jacobi SVD in FP64; the
    library's FP64 fallback counter moves where FP32 cannot resolve the rotation."""
    rng = np.random.default_rng(17)
    sets = stress_edge_cases(rng, 40)
    res = 24
    dx = 1.0 / res
    fallbacks = {}
    for name, Fset in sets.items():
        n = len(Fset)
        x = 0.3 + 0.4 * rng.random((n, 3))
        gc, oc, m, vol = configs(3, 2, (res,) * 3, dx, precision=prec, dt=1e-3, model="fcr")
        sim = apic.Sim(gc, n)
        sim.upload(x, np.zeros((n, 3)), np.zeros((n, 3, 3)), Fset)
        fallbacks[name] = sim.stats()["polar_fp64_fallbacks"]
        x0, v0, B0, F0 = sim.download()
        sim.p2g()
        m_gpu, p_gpu = sim.grid("momentum")
        sim.close()
        gm, gmv, gf, bad = oracle.p2g(oc, x0, v0, B0, F0, m, vol)
        assert bad == 0
        # v = 0 and B = 0: the grid momentum is dt f_i alone.  Where the stress vanishes
        # (F a rotation) both sides are rounding noise, so the error is taken against the
        # force a unit strain would give, dt V_p (2 mu + lam) / dx per particle, too
        mu, lam = oracle.lame(E_DEFAULT, NU_DEFAULT)
        unit = oc.dt * vol * (2 * mu + lam) / dx
        ref = oc.dt * gf
        err = np.abs(p_gpu - ref).max() / max(np.abs(ref).max(), unit)
        assert err <= TOL[prec], (name, err)
    if prec == 32:
        assert fallbacks["inverted_close"] > 0
        assert fallbacks["identity"] == 0 and fallbacks["rotation"] == 0 and fallbacks["stretch"] == 0
    else:
        assert all(v == 0 for v in fallbacks.values())
