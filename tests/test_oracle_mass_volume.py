"""Pins of the oracle's per-particle mass and volume (Sec. 3.2: every particle carries its
own constant mass m_p; Sec. 3.3: its own volume V_p in Phi = sum_p V_p Psi_p and in the
force), which the GPU's apic_upload_mass_volume is compared with:
- the grid mass at every node is sum_p m_p N(x_p - x_i), written out here with the textbook
  quadratic and cubic B-spline kernels, on a few particles of different mass;
- P2G of a set is the sum of the P2G of each particle alone with its own scalar m_p and V_p
  (mass, momentum and force), so each per-particle value reaches its own particle and no
  other;
- with unequal masses the transfer still keeps p and l (Sec. 5.2, 5.3):
  sum_i (m v)_i = sum_p m_p v_p and sum_i x_i x (m v)_i = sum_p x_p x m_p v_p + m_p B_p^T : eps;
- the force scales with V_p: doubling every volume doubles the force and leaves mass and
  momentum unchanged."""
import numpy as np
import pytest

import oracle
from paper_1603_06188_gb300 import scenes


def _bspline(order, r):
    """Textbook 1-D B-spline kernels of the grid-unit distance r."""
    a = np.abs(r)
    if order == 2:
        return np.where(a < 0.5, 0.75 - a * a, np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))
    return np.where(a < 1.0, 0.5 * a ** 3 - a * a + 2.0 / 3.0, np.where(a < 2.0, (2.0 - a) ** 3 / 6.0, 0.0))


def _nodes(res, dim, dx):
    idx = np.stack(np.meshgrid(*[np.arange(res)] * dim, indexing="ij"), -1)
    return idx.transpose(*reversed(range(dim)), dim).reshape(-1, dim) * dx


def _state(dim, order, n, res, seed):
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    cfg = oracle.make_cfg(dim=dim, order=order, res=(res,) * dim, dx=dx, dt=1e-3, model="fcr", E=1e4, nu=0.3)
    x = scenes.random_particles(rng, n, dim, (res,) * dim, dx, margin=3)
    v = rng.normal(size=(n, dim))
    B = 0.05 * dx * rng.normal(size=(n, dim, dim))
    F = scenes.random_deformation(rng, n, dim, 0.2)
    mass = rng.uniform(0.2, 3.0, n)
    vol = dx ** dim * rng.uniform(0.05, 0.3, n)
    return cfg, x, v, B, F, mass, vol


@pytest.mark.parametrize("dim,order", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_grid_mass_is_the_weighted_sum_of_particle_masses(dim, order):
    res = 10
    cfg, x, v, B, F, mass, vol = _state(dim, order, 5, res, seed=1)
    gm, _, _, bad = oracle.p2g(cfg, x, v, B, F, mass, vol)
    assert bad == 0
    nodes = _nodes(res, dim, cfg.dx)
    ref = np.zeros(len(nodes))
    for p in range(len(x)):
        w = np.ones(len(nodes))
        for a in range(dim):
            w *= _bspline(order, (x[p, a] - nodes[:, a]) / cfg.dx)
        ref += mass[p] * w
    np.testing.assert_allclose(gm, ref, rtol=0, atol=1e-14 * mass.sum())
    # a permuted mass array moves the grid mass: the values are per particle
    gm2, _, _, _ = oracle.p2g(cfg, x, v, B, F, mass[::-1].copy(), vol)
    assert np.abs(gm2 - gm).max() > 1e-3


@pytest.mark.parametrize("dim,order", [(2, 3), (3, 2), (3, 3)])
def test_p2g_is_the_sum_over_particles_with_their_own_mass_and_volume(dim, order):
    cfg, x, v, B, F, mass, vol = _state(dim, order, 7, 10, seed=2)
    gm, gmv, gf, bad = oracle.p2g(cfg, x, v, B, F, mass, vol)
    assert bad == 0
    sm, smv, sf = np.zeros_like(gm), np.zeros_like(gmv), np.zeros_like(gf)
    for p in range(len(x)):
        a, b, c, _ = oracle.p2g(cfg, x[p:p + 1], v[p:p + 1], B[p:p + 1], F[p:p + 1], float(mass[p]),
                                float(vol[p]))
        sm += a
        smv += b
        sf += c
    for got, ref in ((gm, sm), (gmv, smv), (gf, sf)):
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("dim,order", [(2, 2), (3, 2), (3, 3)])
def test_unequal_masses_keep_momentum_through_the_transfer(dim, order):
    cfg, x, v, B, F, mass, vol = _state(dim, order, 60, 12, seed=3)
    gm, gmv, _, _ = oracle.p2g(cfg, x, v, B, F, mass, vol)
    p_grid, l_grid = oracle.momentum_grid(cfg, gmv)
    p_part, l_part = oracle.momentum_particles(cfg, x, v, B, mass)
    sp = np.sum(mass * np.linalg.norm(v, axis=1))
    sl = np.sum(mass * (np.linalg.norm(x, axis=1) * np.linalg.norm(v, axis=1) + np.abs(B).reshape(len(B), -1).sum(1)))
    assert np.abs(p_grid - p_part).max() <= 1e-12 * sp
    assert np.abs(l_grid - l_part).max() <= 1e-12 * sl
    # the particle sums are those of the per-particle masses (not of their mean)
    p_mean, _ = oracle.momentum_particles(cfg, x, v, B, np.full(len(x), mass.mean()))
    assert np.abs(p_mean - p_part).max() > 1e-6 * sp


def test_force_scales_with_volume():
    cfg, x, v, B, F, mass, vol = _state(3, 2, 20, 10, seed=4)
    gm, gmv, gf, _ = oracle.p2g(cfg, x, v, B, F, mass, vol)
    gm2, gmv2, gf2, _ = oracle.p2g(cfg, x, v, B, F, mass, 2.0 * vol)
    np.testing.assert_array_equal(gm2, gm)
    np.testing.assert_array_equal(gmv2, gmv)
    np.testing.assert_allclose(gf2, 2.0 * gf, rtol=0, atol=1e-14 * np.abs(gf).max())
    assert np.abs(gf).max() > 0
