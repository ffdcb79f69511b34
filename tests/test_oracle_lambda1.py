"""Pins of the oracle's explicit member lambda = 1 of the Sec. 3.3 integrator family (the
other explicit member besides symplectic Euler): the force evaluated at
F^{n+1} = (I + dt sum_i v_i grad w^T) F^n is -dPhi/dx~ at x~ = x + dt v (central
differences of Phi); the whole step conserves linear and angular momentum (the family
proof of Sec. 5.2 / 5.3 holds for every lambda); without forces it coincides with the
lambda = 0 step; with forces it does not."""
import numpy as np
import pytest

import oracle
from test_oracle_transfers import CASES, random_state, scale_l, scale_p


@pytest.mark.parametrize("dim,order", CASES)
def test_force_at_rest_is_the_lambda0_force(dim, order):
    """With no grid displacement the force reduces to the lambda = 0 force of P2G."""
    cfg, x, v, B, F, m, vol = random_state(dim, order, seed=21)
    _, _, gf0, _ = oracle.p2g(cfg, x, v, B, F, m, vol)
    gf1, bad = oracle.force_at(cfg, x, F, vol, np.zeros_like(gf0))
    assert bad == 0
    np.testing.assert_allclose(gf1, gf0, rtol=0, atol=1e-13 * np.abs(gf0).max())


@pytest.mark.parametrize("dim,order", [(2, 2), (3, 2), (3, 3)])
def test_force_at_displaced_grid_is_minus_energy_gradient(dim, order):
    """Sec. 3.3: f_i = -dPhi/dx~_i at x~ = x + dxg, Phi = sum_p V_p Psi(F^_p(x~)), by central
    differences; the displacement is the lambda = 1 one, dt times the grid velocities."""
    cfg, x, v, B, F, m, vol = random_state(dim, order, n=6, res=8, dt=2e-2, seed=22, Fscale=0.3)
    gm, gmv, _, _ = oracle.p2g(cfg, x, v, B, F, m, vol)
    gv, _ = oracle.grid_update(cfg, gm, gmv, np.zeros_like(gmv))
    dxg = cfg.dt * gv
    assert np.abs(dxg).max() > 1e-3 * cfg.dx     # a real displacement, F^ != F
    gf, _ = oracle.force_at(cfg, x, F, vol, dxg)
    h = 1e-6 * cfg.dx
    rng = np.random.default_rng(23)
    nodes = np.flatnonzero(gm > 0)
    for node in rng.choice(nodes, size=min(12, len(nodes)), replace=False):
        for a in range(dim):
            e = np.zeros_like(dxg); e[node, a] = h
            fd = (oracle.potential(cfg, x, F, vol, dxg + e) - oracle.potential(cfg, x, F, vol, dxg - e)) / (2 * h)
            assert -fd == pytest.approx(gf[node, a], rel=1e-5, abs=1e-7 * np.abs(gf).max())


@pytest.mark.parametrize("model", ["fcr", "nh"])
@pytest.mark.parametrize("dim,order", CASES)
def test_lambda1_step_conserves_momentum(dim, order, model):
    """Sec. 5.2 / 5.3 for the family: with elastic forces and no gravity or walls, p and l
    (including m_p (B_p)^T : eps) are kept to rounding by three lambda = 1 steps.  Evaluating
    the force with F^{n+1} in place of F^n in the last factor, or with P(F^n), breaks l."""
    cfg, x, v, B, F, m, vol = random_state(dim, order, dt=2e-3, seed=24, model=model)
    p0, l0 = oracle.momentum_particles(cfg, x, v, B, m)
    x1, v1, B1, F1, bad = oracle.step_lambda1(cfg, x, v, B, F, m, vol, nsteps=3)
    assert bad == 0
    p1, l1 = oracle.momentum_particles(cfg, x1, v1, B1, m)
    assert np.abs(p1 - p0).max() <= 1e-12 * scale_p(m, v)
    assert np.abs(l1 - l0).max() <= 1e-12 * scale_l(x, v, B, m)
    assert not np.allclose(F1, F)


@pytest.mark.parametrize("dim,order", [(2, 2), (3, 3)])
def test_lambda1_without_forces_is_the_lambda0_step(dim, order):
    """With no force and no gravity v~ = v, so x~ is the same for lambda = 0 and 1."""
    cfg, x, v, B, F, m, vol = random_state(dim, order, model="none", dt=1e-2, seed=25)
    a = oracle.step(cfg, x, v, B, F, m, vol)
    b = oracle.step_lambda1(cfg, x, v, B, F, m, vol)
    for u, w in zip(a[:4], b[:4]):
        np.testing.assert_allclose(w, u, rtol=0, atol=1e-14 * max(1.0, np.abs(u).max()))


def test_lambda1_differs_from_lambda0_with_forces():
    cfg, x, v, B, F, m, vol = random_state(3, 2, dt=2e-2, seed=26, Fscale=0.3)
    a = oracle.step(cfg, x, v, B, F, m, vol)
    b = oracle.step_lambda1(cfg, x, v, B, F, m, vol)
    assert np.abs(b[1] - a[1]).max() > 1e-9 * np.abs(a[1]).max()


def test_lambda1_gravity_changes_momentum_by_dt_g_mass():
    cfg, x, v, B, F, m, vol = random_state(3, 2, dt=1e-3, gravity=(0.0, -9.8, 0.0), seed=27)
    p0, _ = oracle.momentum_particles(cfg, x, v, B, m)
    x1, v1, B1, F1, _ = oracle.step_lambda1(cfg, x, v, B, F, m, vol)
    p1, _ = oracle.momentum_particles(cfg, x1, v1, B1, m)
    np.testing.assert_allclose(p1 - p0, cfg.dt * np.array([0.0, -9.8, 0.0]) * m.sum(), atol=1e-12 * scale_p(m, v))
