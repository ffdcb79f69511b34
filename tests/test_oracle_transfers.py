"""Pins of the oracle's transfers and grid update against what the paper proves:
conservation of linear / angular momentum per phase (Sec. 5.2, 5.3), single-particle
stability (Sec. 5.4), the affine round trip (Sec. 5.5), the lambda = 0 reduction
(Sec. 5.7), force = -dPhi/dx~ (Sec. 3.3), and PIC's loss of angular momentum (Sec. 1)."""
import numpy as np
import pytest

import oracle
from paper_1603_06188_gb300 import scenes

E, NU = 1e4, 0.3


def k_of(order, dx):
    return dx * dx * (0.25 if order == 2 else 1.0 / 3.0)


def random_state(dim, order, n=60, res=14, seed=0, Fscale=0.2, model="fcr", dt=1e-3, **kw):
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    cfg = oracle.make_cfg(dim=dim, order=order, res=(res,) * dim, dx=dx, dt=dt, model=model,
                          E=E, nu=NU, **kw)
    x = scenes.random_particles(rng, n, dim, (res,) * dim, dx, margin=order + 1)
    v = rng.normal(size=(n, dim))
    B = 0.05 * rng.normal(size=(n, dim, dim))
    F = scenes.random_deformation(rng, n, dim, Fscale)
    mass = rng.uniform(0.5, 2.0, size=n)
    vol = rng.uniform(0.5, 2.0, size=n) * dx ** dim
    return cfg, x, v, B, F, mass, vol


def scale_p(mass, v):
    return np.sum(mass * np.linalg.norm(v, axis=1))


def scale_l(x, v, B, mass):
    return np.sum(mass * np.linalg.norm(x, axis=1) * np.linalg.norm(v, axis=1)) + \
        np.sum(mass * np.linalg.norm(B.reshape(len(B), -1), axis=1))


CASES = [(d, o) for d in (2, 3) for o in (2, 3)]


@pytest.mark.parametrize("dim,order", CASES)
def test_p2g_conserves_momentum(dim, order):
    cfg, x, v, B, F, m, vol = random_state(dim, order)
    gm, gmv, gf, bad = oracle.p2g(cfg, x, v, B, F, m, vol)
    assert bad == 0
    pP, lP = oracle.momentum_particles(cfg, x, v, B, m)
    pG, lG = oracle.momentum_grid(cfg, gmv)
    assert np.abs(pG - pP).max() <= 1e-12 * scale_p(m, v)
    assert np.abs(lG - lP).max() <= 1e-12 * scale_l(x, v, B, m)
    assert gm.sum() == pytest.approx(m.sum(), rel=1e-13)


@pytest.mark.parametrize("dim,order", CASES)
def test_grid_update_conserves_momentum_with_elastic_force(dim, order):
    cfg, x, v, B, F, m, vol = random_state(dim, order, dt=1e-2)
    gm, gmv, gf, _ = oracle.p2g(cfg, x, v, B, F, m, vol)
    assert np.abs(gf).max() > 0
    gv, gvt = oracle.grid_update(cfg, gm, gmv, gf)
    pG, lG = oracle.momentum_grid(cfg, gmv)
    # Sec. 5.2 / 5.3 with lambda = 0: p~ = p and sum x~_i x m_i v~_i = l with x~ = x + dt v~
    pT, lTx = oracle.momentum_grid(cfg, gm[:, None] * gvt)
    s = scale_p(m, v) + np.abs(gf).sum() * cfg.dt
    assert np.abs(pT - pG).max() <= 1e-12 * s
    # x~_i x m v~ = x_i x m v~ + dt v~ x m v~ = x_i x m v~
    assert np.abs(lTx - lG).max() <= 1e-12 * (scale_l(x, v, B, m) + s)
    # the force itself sums to zero and has no torque (Sec. 5.2, 5.3)
    p_f, l_f = oracle.momentum_grid(cfg, gf)
    assert np.abs(p_f).max() <= 1e-12 * np.abs(gf).sum()
    assert np.abs(l_f).max() <= 1e-12 * np.abs(gf).sum()


@pytest.mark.parametrize("dim,order", CASES)
def test_g2p_conserves_momentum(dim, order):
    cfg, x, v, B, F, m, vol = random_state(dim, order, dt=1e-2)
    gm, gmv, gf, _ = oracle.p2g(cfg, x, v, B, F, m, vol)
    gv, gvt = oracle.grid_update(cfg, gm, gmv, gf)
    x1, v1, B1, F1, bad = oracle.g2p(cfg, x, F, gv, gvt)
    assert bad == 0
    pT, _ = oracle.momentum_grid(cfg, gm[:, None] * gvt)
    # grid angular momentum with moved nodes x~_i = x_i + dt v~_i
    nodes = np.stack(np.meshgrid(*[np.arange(cfg.res[a]) for a in range(dim)], indexing="ij"),
                     -1)
    nodes = nodes.transpose(*reversed(range(dim)), dim).reshape(-1, dim) * cfg.dx
    xt = nodes + cfg.dt * gvt
    mvt = gm[:, None] * gvt
    if dim == 2:
        lT = np.array([np.sum(xt[:, 0] * mvt[:, 1] - xt[:, 1] * mvt[:, 0]), 0, 0])
    else:
        lT = np.cross(xt, mvt).sum(0)
    p1, l1 = oracle.momentum_particles(cfg, x1, v1, B1, m)
    assert np.abs(p1 - pT).max() <= 1e-12 * scale_p(m, v1)
    assert np.abs(l1 - lT).max() <= 1e-12 * scale_l(x1, v1, B1, m)


@pytest.mark.parametrize("dim,order", CASES)
def test_whole_step_conserves_momentum(dim, order):
    cfg, x, v, B, F, m, vol = random_state(dim, order, n=120, dt=5e-3, seed=4)
    p0, l0 = oracle.momentum_particles(cfg, x, v, B, m)
    x1, v1, B1, F1, bad = oracle.step(cfg, x, v, B, F, m, vol, nsteps=3)
    assert bad == 0
    p1, l1 = oracle.momentum_particles(cfg, x1, v1, B1, m)
    assert np.abs(p1 - p0).max() <= 1e-12 * scale_p(m, v)
    assert np.abs(l1 - l0).max() <= 1e-12 * scale_l(x, v, B, m)
    assert np.abs(F1 - F).max() > 0


@pytest.mark.parametrize("dim,order", CASES)
def test_general_g2p_equals_lambda0_form(dim, order):
    """Sec. 5.7: at lambda = 0 the general B / x updates reduce to the original APIC ones."""
    cfg, x, v, B, F, m, vol = random_state(dim, order, dt=1e-2, seed=5)
    gm, gmv, gf, _ = oracle.p2g(cfg, x, v, B, F, m, vol)
    gv, gvt = oracle.grid_update(cfg, gm, gmv, gf)
    a = oracle.g2p(cfg, x, F, gv, gvt)
    b = oracle.g2p_lambda0(cfg, x, F, gvt)
    for u, w in zip(a[:4], b[:4]):
        np.testing.assert_allclose(u, w, rtol=1e-12, atol=1e-13 * max(1.0, np.abs(w).max()))


def test_lambda_one_general_form_differs():
    """Regression guard: with lambda = 1 the general form must NOT match the lambda = 0 one
    (x~ uses v_i, so the B correction term no longer cancels)."""
    cfg, x, v, B, F, m, vol = random_state(3, 2, dt=1e-1, seed=6, lambda_t=1.0)
    gm, gmv, gf, _ = oracle.p2g(cfg, x, v, B, F, m, vol)
    gv, gvt = oracle.grid_update(cfg, gm, gmv, gf)
    a = oracle.g2p(cfg, x, F, gv, gvt)
    b = oracle.g2p_lambda0(cfg, x, F, gvt)
    assert np.abs(a[2] - b[2]).max() > 1e-8


@pytest.mark.parametrize("dim,order", CASES)
def test_single_particle_stability(dim, order):
    """Sec. 5.4: an isolated particle with no force keeps v_p and B_p and moves by dt v_p."""
    cfg, x, v, B, F, m, vol = random_state(dim, order, n=1, dt=1e-3, model="none", seed=7)
    x1, v1, B1, F1, bad = oracle.step(cfg, x, v, B, F, m, vol)
    assert bad == 0
    np.testing.assert_allclose(v1, v, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(B1, B, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(x1, x + cfg.dt * v, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("dim,order", CASES)
def test_affine_round_trip(dim, order):
    """Sec. 5.5: v_p = c + C x_p and B_p = C D_p survive P2G -> G2P at dt = 0, and the grid
    velocity is the same affine field v_i = c + C x_i."""
    res = 14
    cfg, x, _, _, F, m, vol = random_state(dim, order, n=80, res=res, dt=0.0, model="none", seed=8)
    rng = np.random.default_rng(9)
    cvec = rng.normal(size=dim)
    Cm = rng.normal(size=(dim, dim))           # deliberately not symmetric
    v = cvec + x @ Cm.T
    B = np.broadcast_to(Cm * k_of(order, cfg.dx), (len(x), dim, dim)).copy()
    gm, gmv, gf, _ = oracle.p2g(cfg, x, v, B, F, m, vol)
    gv, gvt = oracle.grid_update(cfg, gm, gmv, gf)
    nodes = np.stack(np.meshgrid(*[np.arange(res)] * dim, indexing="ij"), -1)
    nodes = nodes.transpose(*reversed(range(dim)), dim).reshape(-1, dim) * cfg.dx
    occ = gm > 0
    np.testing.assert_allclose(gv[occ], cvec + nodes[occ] @ Cm.T, atol=1e-11)
    x1, v1, B1, F1, _ = oracle.g2p(cfg, x, F, gv, gvt)
    np.testing.assert_allclose(x1, x, atol=1e-14)
    np.testing.assert_allclose(v1, v, atol=1e-11)
    np.testing.assert_allclose(B1, B, atol=1e-13)


@pytest.mark.parametrize("dim,order", [(2, 2), (3, 2), (3, 3)])
def test_force_is_minus_energy_gradient(dim, order):
    """Sec. 3.3: f_i = -dPhi/dx~_i at x~ = x, by central differences of Phi."""
    cfg, x, v, B, F, m, vol = random_state(dim, order, n=6, res=8, dt=1.0, seed=10, Fscale=0.3)
    gm, gmv, gf, _ = oracle.p2g(cfg, x, v, B, F, m, vol)
    nn = gm.shape[0]
    h = 1e-6 * cfg.dx
    rng = np.random.default_rng(11)
    nodes = np.flatnonzero(gm > 0)
    for node in rng.choice(nodes, size=min(12, len(nodes)), replace=False):
        for a in range(dim):
            e = np.zeros((nn, dim)); e[node, a] = h
            fd = (oracle.potential(cfg, x, F, vol, e) - oracle.potential(cfg, x, F, vol, -e)) / (2 * h)
            assert -fd == pytest.approx(gf[node, a], rel=1e-5, abs=1e-7 * np.abs(gf).max())


def test_gravity_changes_momentum_by_dt_g_mass():
    cfg, x, v, B, F, m, vol = random_state(3, 2, dt=1e-3, gravity=(0.0, -9.8, 0.0), seed=12)
    p0, _ = oracle.momentum_particles(cfg, x, v, B, m)
    x1, v1, B1, F1, _ = oracle.step(cfg, x, v, B, F, m, vol)
    p1, _ = oracle.momentum_particles(cfg, x1, v1, B1, m)
    np.testing.assert_allclose(p1 - p0, cfg.dt * np.array([0.0, -9.8, 0.0]) * m.sum(), atol=1e-12 * scale_p(m, v))


def test_sticky_walls_zero_boundary_velocity():
    cfg, x, v, B, F, m, vol = random_state(3, 2, res=10, dt=1e-3, boundary="sticky", wall=3, seed=13)
    gm, gmv, gf, _ = oracle.p2g(cfg, x, v, B, F, m, vol)
    gv, gvt = oracle.grid_update(cfg, gm, gmv, gf)
    idx = np.stack(np.meshgrid(*[np.arange(10)] * 3, indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(-1, 3)
    wall = np.any((idx < 3) | (idx >= 7), axis=1)
    assert np.all(gvt[wall] == 0.0)
    assert np.any(gvt[(~wall) & (gm > 0)] != 0.0)


def test_pic_conserves_linear_but_loses_angular_momentum():
    """Sec. 1: PIC's G2P keeps linear momentum but dissipates angular momentum; APIC keeps both."""
    sc = scenes.rotating_disk_2d(res=32, ppc=4, seed=1)
    n = sc.n
    m = np.ones(n)
    res = {}
    for mode in ("pic", "apic"):
        cfg = oracle.make_cfg(dim=2, order=2, transfer=mode, res=sc.res, dx=sc.dx, dt=1e-2)
        B = sc.grad_v * k_of(2, sc.dx) if mode == "apic" else np.zeros((n, 2, 2))
        p0, l0 = oracle.momentum_particles(cfg, sc.x, sc.v, B, m)
        x1, v1, B1, F1, bad = oracle.step(cfg, sc.x, sc.v, B, np.broadcast_to(np.eye(2), (n, 2, 2)), m, m, nsteps=5)
        p1, l1 = oracle.momentum_particles(cfg, x1, v1, B1, m)
        res[mode] = (p0, l0, p1, l1)
    p0, l0, p1, l1 = res["pic"]
    assert np.abs(p1 - p0).max() < 1e-12 * n
    assert abs(l1[0] - l0[0]) > 1e-3 * abs(l0[0])
    p0, l0, p1, l1 = res["apic"]
    assert np.abs(p1 - p0).max() < 1e-12 * n
    assert abs(l1[0] - l0[0]) < 1e-12 * n


def test_pic_p2g_conserves_angular_momentum_without_B():
    cfg, x, v, B, F, m, vol = random_state(3, 2, transfer="pic", model="none", seed=14)
    gm, gmv, gf, _ = oracle.p2g(cfg, x, v, B, F, m, vol)
    pP, lP = oracle.momentum_particles(cfg, x, v, np.zeros_like(B), m)
    pG, lG = oracle.momentum_grid(cfg, gmv)
    assert np.abs(lG - lP).max() <= 1e-12 * scale_l(x, v, B, m)


@pytest.mark.parametrize("dim,order", CASES)
def test_g2p_of_affine_grid_field(dim, order):
    """A grid velocity field v~_i = c + C x_i is reproduced on particles: v_p = c + C x_p,
    B_p = C D_p, x_p moves by dt v_p and F_p^{n+1} = (I + dt C) F_p^n (Sec. 3.4 with the
    weight identities of Sec. 3.5)."""
    res = 12
    cfg, x, _, _, F, m, vol = random_state(dim, order, n=40, res=res, dt=0.05, model="none", seed=15)
    rng = np.random.default_rng(16)
    cvec = rng.normal(size=dim)
    Cm = rng.normal(size=(dim, dim))
    nodes = np.stack(np.meshgrid(*[np.arange(res)] * dim, indexing="ij"), -1)
    nodes = nodes.transpose(*reversed(range(dim)), dim).reshape(-1, dim) * cfg.dx
    gvt = cvec + nodes @ Cm.T
    x1, v1, B1, F1, bad = oracle.g2p(cfg, x, F, gvt, gvt)
    assert bad == 0
    np.testing.assert_allclose(v1, cvec + x @ Cm.T, atol=1e-12)
    np.testing.assert_allclose(x1, x + cfg.dt * v1, atol=1e-14)
    np.testing.assert_allclose(B1, np.broadcast_to(Cm * k_of(order, cfg.dx), B1.shape), atol=1e-13)
    np.testing.assert_allclose(F1, np.einsum("ab,pbc->pac", np.eye(dim) + cfg.dt * Cm, F), atol=1e-12)
