"""Pins of the oracle's widened parts: Neo-Hookean stress (the model of the paper's
experiments, Sec. 6), slip walls (used by the paper's Sec. 6.2 rebound test), and the
time-step bound of Sec. 4.3."""
import numpy as np
import pytest

import oracle
from paper_1603_06188_gb300 import scenes

MU, LAM = oracle.lame(1e3, 0.3)


def _rot(rng, d):
    Q, _ = np.linalg.qr(rng.normal(size=(d, d)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


@pytest.mark.parametrize("d", [2, 3])
def test_neohookean_stress_is_energy_derivative_and_invariant(d):
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(15):
        F = np.eye(d) + 0.3 * rng.uniform(-1, 1, size=(d, d))
        if np.linalg.det(F) < 0.3:
            continue
        P = oracle.stress_nh(F, MU, LAM)
        fd = np.zeros_like(F)
        for a in range(d):
            for b in range(d):
                E = np.zeros_like(F); E[a, b] = h
                fd[a, b] = (oracle.psi_nh(F + E, MU, LAM) - oracle.psi_nh(F - E, MU, LAM)) / (2 * h)
        np.testing.assert_allclose(P, fd, rtol=1e-6, atol=1e-6 * np.abs(P).max())
        Q = _rot(rng, d)
        np.testing.assert_allclose(oracle.stress_nh(Q, MU, LAM), 0.0, atol=1e-9)
        np.testing.assert_allclose(oracle.stress_nh(Q @ F, MU, LAM), Q @ P, atol=1e-9 * np.abs(P).max())
        tau = P @ F.T
        np.testing.assert_allclose(tau, tau.T, atol=1e-9 * np.abs(tau).max())
        # closed form of the Kirchhoff stress: P F^T = mu (F F^T - I) + lam log(J) I
        np.testing.assert_allclose(tau, MU * (F @ F.T - np.eye(d)) + LAM * np.log(np.linalg.det(F)) * np.eye(d),
                                   atol=1e-9 * np.abs(tau).max())


def test_neohookean_step_conserves_momentum():
    rng = np.random.default_rng(1)
    res = 14
    cfg = oracle.make_cfg(dim=3, order=2, res=(res,) * 3, dx=1 / res, dt=5e-3, model="nh", E=1e3, nu=0.3)
    n = 100
    x = scenes.random_particles(rng, n, 3, (res,) * 3, 1 / res, margin=3)
    v = rng.normal(size=(n, 3))
    B = 0.01 * rng.normal(size=(n, 3, 3))
    F = scenes.random_deformation(rng, n, 3, 0.2)
    m = np.ones(n)
    p0, l0 = oracle.momentum_particles(cfg, x, v, B, m)
    x1, v1, B1, F1, bad = oracle.step(cfg, x, v, B, F, m, np.full(n, 1e-4), nsteps=3)
    p1, l1 = oracle.momentum_particles(cfg, x1, v1, B1, m)
    assert bad == 0
    assert np.abs(p1 - p0).max() <= 1e-12 * np.abs(v).sum()
    assert np.abs(l1 - l0).max() <= 1e-12 * (np.abs(v).sum() + np.abs(B).sum())


def test_neohookean_force_is_minus_energy_gradient():
    rng = np.random.default_rng(2)
    res = 8
    cfg = oracle.make_cfg(dim=3, order=2, res=(res,) * 3, dx=1 / res, dt=1.0, model="nh", E=1e3, nu=0.3)
    n = 5
    x = scenes.random_particles(rng, n, 3, (res,) * 3, 1 / res, margin=3)
    F = scenes.random_deformation(rng, n, 3, 0.2)
    vol = np.full(n, 1e-3)
    gm, gmv, gf, _ = oracle.p2g(cfg, x, np.zeros((n, 3)), np.zeros((n, 3, 3)), F, 1.0, vol)
    h = 1e-6 * cfg.dx
    for node in rng.choice(np.flatnonzero(gm > 0), size=8, replace=False):
        for a in range(3):
            e = np.zeros((len(gm), 3)); e[node, a] = h
            fd = (oracle.potential(cfg, x, F, vol, e) - oracle.potential(cfg, x, F, vol, -e)) / (2 * h)
            assert -fd == pytest.approx(gf[node, a], rel=1e-5, abs=1e-7 * np.abs(gf).max())


def test_slip_walls_zero_only_the_normal_component():
    rng = np.random.default_rng(3)
    res = 10
    cfg = oracle.make_cfg(dim=3, order=2, res=(res,) * 3, dx=1 / res, dt=1e-3, boundary="slip", wall=3)
    n = 300
    x = scenes.random_particles(rng, n, 3, (res,) * 3, 1 / res, margin=3)
    v = rng.normal(size=(n, 3))
    gm, gmv, gf, _ = oracle.p2g(cfg, x, v, np.zeros((n, 3, 3)), np.broadcast_to(np.eye(3), (n, 3, 3)), 1.0, 1.0)
    gv, gvt = oracle.grid_update(cfg, gm, gmv, gf)
    idx = np.stack(np.meshgrid(*[np.arange(res)] * 3, indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(-1, 3)
    inwall = (idx < 3) | (idx >= res - 3)
    occ = (gm > 0)[:, None] & np.ones((1, 3), dtype=bool)
    assert np.all(gvt[occ & inwall] == 0.0)                       # normal components
    np.testing.assert_allclose(gvt[occ & ~inwall], gv[occ & ~inwall], rtol=1e-14)   # tangential kept
    assert np.any(occ & inwall) and np.any(occ & ~inwall & inwall.any(axis=1, keepdims=True))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("order", [2, 3])
def test_cfl_speed_bound(dim, order):
    """Sec. 4.3: (kappa/k) dx = 6 sqrt(d) / dx for both splines, and it bounds
    |D_p^{-1}(x_i - x_p)| over the stencil; the bound on |v_i| holds on the grid."""
    dx = 1 / 16
    cfg = oracle.make_cfg(dim=dim, order=order, res=(16,) * dim, dx=dx, dt=0.0)
    rng = np.random.default_rng(4)
    v = np.zeros((1, dim)); B = np.zeros((1, dim, dim)); B[0, 0, 0] = 1.0
    assert oracle.cfl_speed(cfg, v, B) == pytest.approx(6 * np.sqrt(dim) / dx, rel=1e-14)
    k = (0.25 if order == 2 else 1 / 3) * dx * dx
    worst = 0.0
    for _ in range(200):
        xp = 0.3 + 0.4 * rng.random(dim)
        rc, base, w, dw = oracle.stencil(cfg, xp)
        r = oracle.stencil_nodes(cfg, base) - xp
        worst = max(worst, np.linalg.norm(r, axis=1)[w > 0].max() / k)
    assert worst <= 6 * np.sqrt(dim) / dx
    assert worst >= 0.7 * 6 * np.sqrt(dim) / dx
    # grid velocities obey |v_i| <= max_p(|v_p| + 6 sqrt(d)/dx |B_p|_F)
    n = 200
    x = scenes.random_particles(rng, n, dim, (16,) * dim, dx, margin=order + 1)
    v = rng.normal(size=(n, dim))
    B = 1e-3 * rng.normal(size=(n, dim, dim))
    gm, gmv, gf, _ = oracle.p2g(cfg, x, v, B, np.broadcast_to(np.eye(dim), (n, dim, dim)), 1.0, 1.0)
    gv, _ = oracle.grid_update(cfg, gm, gmv, gf)
    assert np.linalg.norm(gv, axis=1).max() <= oracle.cfl_speed(cfg, v, B) * (1 + 1e-12)
