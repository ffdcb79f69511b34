"""Pins of the oracle's implicit midpoint rule (lambda = 1/2, Sec. 4.1-4.2), the member the
paper itself uses: the stress derivatives dP/dF : dF by central differences of P; the
force-derivative product by central differences of the force (Sec. 3.3); the Newton / CG
grid solve satisfies m_i dv_i = dt f_i(x_i + dt/2 v_i + dt/4 dv_i) and agrees with an
independent root finder; the converged step conserves linear and angular momentum (the
family proof of Sec. 5.2 / 5.3); a truncated solve still conserves linear momentum, because
conjugate gradients in the mass inner product keep every vector velocity-like (Sec. 4.2);
without forces the step is the lambda = 0 step."""
import numpy as np
import pytest

import oracle
from test_oracle_transfers import CASES, random_state, scale_l, scale_p

E, NU = 1e4, 0.3


def rand_F(rng, d, scale=0.25):
    while True:
        F = np.eye(d) + scale * rng.normal(size=(d, d))
        if np.linalg.det(F) > 0.2:
            return F


@pytest.mark.parametrize("model", ["fcr", "nh"])
@pytest.mark.parametrize("d", [2, 3])
def test_dstress_matches_finite_differences(model, d):
    mu, lam = oracle.lame(E, NU)
    stress = oracle.stress_nh if model == "nh" else oracle.stress_fcr
    rng = np.random.default_rng(31 + d)
    h = 1e-6
    for _ in range(8):
        F = rand_F(rng, d)
        dF = rng.normal(size=(d, d))
        fd = (stress(F + h * dF, mu, lam) - stress(F - h * dF, mu, lam)) / (2 * h)
        got = oracle.dstress(model, F, dF, mu, lam)
        np.testing.assert_allclose(got, fd, rtol=0, atol=1e-6 * np.abs(fd).max())


def grid_velocity(cfg, x, v, B, F, m, vol):
    cfg0 = oracle.make_cfg(dim=cfg.dim, order=cfg.order, res=tuple(cfg.res[:cfg.dim]), dx=cfg.dx, dt=cfg.dt)
    gm, gmv, _, _ = oracle.p2g(cfg0, x, v, B, F, m, vol)
    gv = np.where(gm[:, None] > 0, gmv / np.where(gm > 0, gm, 1.0)[:, None], 0.0)
    return gm, gv


@pytest.mark.parametrize("model", ["fcr", "nh"])
@pytest.mark.parametrize("dim,order", [(2, 2), (3, 2), (3, 3)])
def test_force_diff_matches_finite_differences_of_the_force(dim, order, model):
    cfg, x, v, B, F, m, vol = random_state(dim, order, n=8, res=8, dt=2e-2, seed=32, Fscale=0.3, model=model)
    gm, gv = grid_velocity(cfg, x, v, B, F, m, vol)
    dxg = 0.5 * cfg.dt * gv
    rng = np.random.default_rng(33)
    du = rng.normal(size=gv.shape) * (gm[:, None] > 0)
    got, bad = oracle.force_diff_at(cfg, x, F, vol, dxg, du)
    assert bad == 0
    h = 1e-6 * cfg.dx / np.abs(du).max()
    fp, _ = oracle.force_at(cfg, x, F, vol, dxg + h * du)
    fm, _ = oracle.force_at(cfg, x, F, vol, dxg - h * du)
    fd = (fp - fm) / (2 * h)
    np.testing.assert_allclose(got, fd, rtol=0, atol=1e-5 * np.abs(fd).max())


def residual(cfg, x, F, vol, gm, gv, dv):
    f, _ = oracle.force_at(cfg, x, F, vol, 0.5 * cfg.dt * gv + 0.25 * cfg.dt * dv)
    return gm[:, None] * dv - cfg.dt * f


@pytest.mark.parametrize("model", ["fcr", "nh"])
@pytest.mark.parametrize("dim,order", CASES)
def test_grid_solve_satisfies_the_midpoint_system(dim, order, model):
    cfg, x, v, B, F, m, vol = random_state(dim, order, dt=5e-3, seed=34, model=model)
    gm, gv = grid_velocity(cfg, x, v, B, F, m, vol)
    dv, it = oracle.midpoint_solve(cfg, x, F, vol, gm, gv)
    assert 1 <= it < 20
    assert np.abs(dv).max() > 0
    res = residual(cfg, x, F, vol, gm, gv, dv)
    scale = np.abs(gm[:, None] * dv).max()
    assert np.abs(res).max() <= 1e-11 * scale
    assert np.all(dv[gm <= 0] == 0.0)


def test_grid_solve_agrees_with_an_independent_root_finder():
    """The same system solved by MINPACK's hybrid method (scipy) from the same start."""
    optimize = pytest.importorskip("scipy.optimize")
    cfg, x, v, B, F, m, vol = random_state(2, 2, n=10, res=8, dt=1e-2, seed=35, model="fcr")
    gm, gv = grid_velocity(cfg, x, v, B, F, m, vol)
    live = gm > 0
    shape = gv.shape

    def fun(z):
        dv = np.zeros(shape)
        dv[live] = z.reshape(-1, shape[1])
        return residual(cfg, x, F, vol, gm, gv, dv)[live].ravel() / gm[live].repeat(shape[1])

    sol = optimize.root(fun, np.zeros(live.sum() * shape[1]), method="hybr", tol=1e-12)
    assert np.abs(fun(sol.x)).max() <= 1e-10 * np.abs(sol.x).max()
    dv, _ = oracle.midpoint_solve(cfg, x, F, vol, gm, gv)
    np.testing.assert_allclose(dv[live].ravel(), sol.x, rtol=0, atol=1e-9 * np.abs(sol.x).max())


@pytest.mark.parametrize("model", ["fcr", "nh"])
@pytest.mark.parametrize("dim,order", CASES)
def test_converged_midpoint_step_conserves_momentum(dim, order, model):
    cfg, x, v, B, F, m, vol = random_state(dim, order, dt=5e-3, seed=36, model=model)
    p0, l0 = oracle.momentum_particles(cfg, x, v, B, m)
    x1, v1, B1, F1, bad = oracle.step_midpoint(cfg, x, v, B, F, m, vol)
    assert bad == 0
    p1, l1 = oracle.momentum_particles(cfg, x1, v1, B1, m)
    assert np.abs(p1 - p0).max() <= 1e-12 * scale_p(m, v)
    assert np.abs(l1 - l0).max() <= 1e-11 * scale_l(x, v, B, m)


@pytest.mark.parametrize("dim,order", [(2, 2), (3, 2)])
def test_truncated_solve_still_conserves_linear_momentum(dim, order):
    """One Newton step with two CG iterations leaves the system unsolved, yet p is kept to
    rounding: with the mass inner product every CG vector is velocity-like (Sec. 4.2)."""
    cfg, x, v, B, F, m, vol = random_state(dim, order, dt=2e-2, seed=37, Fscale=0.3)
    gm, gv = grid_velocity(cfg, x, v, B, F, m, vol)
    dv, _ = oracle.midpoint_solve(cfg, x, F, vol, gm, gv, newton=1, cg=2)
    res = residual(cfg, x, F, vol, gm, gv, dv)
    assert np.abs(res).max() > 1e-6 * np.abs(gm[:, None] * dv).max()     # not converged
    np.testing.assert_allclose((gm[:, None] * dv).sum(axis=0), 0.0, atol=1e-13 * np.abs(gm[:, None] * dv).sum())
    p0, _ = oracle.momentum_particles(cfg, x, v, B, m)
    x1, v1, B1, F1, _ = oracle.step_midpoint(cfg, x, v, B, F, m, vol, newton=1, cg=2)
    p1, _ = oracle.momentum_particles(cfg, x1, v1, B1, m)
    assert np.abs(p1 - p0).max() <= 1e-12 * scale_p(m, v)


@pytest.mark.parametrize("dim,order", [(2, 3), (3, 2)])
def test_midpoint_without_forces_is_the_lambda0_step(dim, order):
    cfg, x, v, B, F, m, vol = random_state(dim, order, model="none", dt=1e-2, seed=38)
    a = oracle.step(cfg, x, v, B, F, m, vol)
    b = oracle.step_midpoint(cfg, x, v, B, F, m, vol)
    for u, w in zip(a[:4], b[:4]):
        np.testing.assert_allclose(w, u, rtol=0, atol=1e-14 * max(1.0, np.abs(u).max()))


def test_midpoint_differs_from_the_explicit_members_with_forces():
    cfg, x, v, B, F, m, vol = random_state(3, 2, dt=2e-2, seed=39, Fscale=0.3)
    mid = oracle.step_midpoint(cfg, x, v, B, F, m, vol)
    for other in (oracle.step(cfg, x, v, B, F, m, vol), oracle.step_lambda1(cfg, x, v, B, F, m, vol)):
        assert np.abs(mid[1] - other[1]).max() > 1e-9 * np.abs(other[1]).max()


@pytest.mark.parametrize("model", ["fcr", "nh"])
def test_cg_solves_the_newton_system_within_its_size(model):
    """Algorithm 1 with the mass inner product, in which the Newton operator
    I - dt^2/4 M^{-1} df/dx is symmetric, solves one Newton system in at most as many
    iterations as unknowns (Sec. 4.2); the linear residual is checked from outside."""
    cfg, x, v, B, F, m, vol = random_state(2, 2, n=3, res=8, dt=2e-2, seed=40, Fscale=0.3, model=model)
    gm, gv = grid_velocity(cfg, x, v, B, F, m, vol)
    live = gm > 0
    unknowns = int(live.sum()) * cfg.dim
    dv, _ = oracle.midpoint_solve(cfg, x, F, vol, gm, gv, newton=1, cg=unknowns, tol=1e-15)
    dxg0 = 0.5 * cfg.dt * gv
    f0, _ = oracle.force_at(cfg, x, F, vol, dxg0)
    minv = np.where(live, 1.0 / np.where(live, gm, 1.0), 0.0)[:, None]
    r0 = cfg.dt * minv * f0
    kdv, _ = oracle.force_diff_at(cfg, x, F, vol, dxg0, dv)
    r_lin = r0 - (dv - 0.25 * cfg.dt ** 2 * minv * kdv)
    norm_m = lambda u: np.sqrt(np.sum(gm[:, None] * u * u))
    assert norm_m(r_lin) <= 1e-9 * norm_m(r0)
