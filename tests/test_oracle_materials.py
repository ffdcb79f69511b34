"""Pins of the oracle's per-particle materials (a Lame pair per particle): uniform
per-particle values reproduce the configuration's material exactly,
P2G is linear in the particles so a two-material set equals the sum of its two
single-material halves, the force is minus the gradient of the sum of the halves' elastic
energies, and a mixed-material step conserves momentum (Sec. 5.2, 5.3)."""
import numpy as np
import pytest

import oracle
from paper_1603_06188_gb300 import scenes

RES = 12


def _setup(model, seed=0, n=120):
    rng = np.random.default_rng(seed)
    x = scenes.random_particles(rng, n, 3, (RES,) * 3, 1 / RES, margin=3)
    v = rng.normal(size=(n, 3))
    B = 0.01 * rng.normal(size=(n, 3, 3))
    F = scenes.random_deformation(rng, n, 3, 0.2)
    soft = rng.random(n) < 0.5
    E = np.where(soft, 1e3, 4e4)
    nu = np.where(soft, 0.3, 0.42)
    mu, lam = oracle.lame(E, nu)
    cfgs = {e: oracle.make_cfg(dim=3, order=2, res=(RES,) * 3, dx=1 / RES, dt=2e-4, model=model, E=e, nu=p)
            for e, p in ((1e3, 0.3), (4e4, 0.42))}
    return x, v, B, F, soft, mu, lam, cfgs


@pytest.mark.parametrize("model", ["fcr", "nh"])
def test_uniform_materials_equal_the_configuration(model):
    x, v, B, F, _, _, _, cfgs = _setup(model)
    cfg = cfgs[1e3]
    n = len(x)
    mu = np.full(n, cfg.mu); lam = np.full(n, cfg.lam)
    vol = np.full(n, 1e-4)
    a = oracle.p2g(cfg, x, v, B, F, 1.0, vol)
    b = oracle.p2g(cfg, x, v, B, F, 1.0, vol, mu=mu, lam=lam)
    for u, w in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(u, w)
    sa = oracle.step(cfg, x, v, B, F, 1.0, vol, nsteps=2)
    sb = oracle.step(cfg, x, v, B, F, 1.0, vol, nsteps=2, mu=mu, lam=lam)
    for u, w in zip(sa[:4], sb[:4]):
        np.testing.assert_array_equal(u, w)


@pytest.mark.parametrize("model", ["fcr", "nh"])
def test_mixed_p2g_is_the_sum_of_its_single_material_parts(model):
    x, v, B, F, soft, mu, lam, cfgs = _setup(model, seed=1)
    vol = np.full(len(x), 1e-4)
    gm, gmv, gf, bad = oracle.p2g(cfgs[1e3], x, v, B, F, 1.0, vol, mu=mu, lam=lam)
    assert bad == 0
    parts = [oracle.p2g(cfgs[e], x[s], v[s], B[s], F[s], 1.0, vol[s]) for e, s in ((1e3, soft), (4e4, ~soft))]
    np.testing.assert_allclose(gm, parts[0][0] + parts[1][0], rtol=0, atol=1e-12 * gm.max())
    np.testing.assert_allclose(gmv, parts[0][1] + parts[1][1], rtol=0, atol=1e-12 * np.abs(gmv).max())
    np.testing.assert_allclose(gf, parts[0][2] + parts[1][2], rtol=0, atol=1e-12 * np.abs(gf).max())
    # the stiff half really is stiffer: its force differs from the same particles' soft force
    stiff_as_soft = oracle.p2g(cfgs[1e3], x[~soft], v[~soft], B[~soft], F[~soft], 1.0, vol[~soft])[2]
    assert np.abs(parts[1][2] - stiff_as_soft).max() > 0.5 * np.abs(parts[1][2]).max()


def test_mixed_force_is_minus_the_gradient_of_both_energies():
    x, _, _, F, soft, mu, lam, cfgs = _setup("fcr", seed=2, n=8)
    n = len(x)
    vol = np.full(n, 1e-3)
    cfg = oracle.make_cfg(dim=3, order=2, res=(RES,) * 3, dx=1 / RES, dt=1.0, model="fcr", E=1e3, nu=0.3)
    gm, _, gf, _ = oracle.p2g(cfg, x, np.zeros((n, 3)), np.zeros((n, 3, 3)), F, 1.0, vol, mu=mu, lam=lam)
    h = 1e-6 / RES
    rng = np.random.default_rng(3)
    for node in rng.choice(np.flatnonzero(gm > 0), size=6, replace=False):
        for a in range(3):
            e = np.zeros((len(gm), 3)); e[node, a] = h
            phi = lambda d: sum(oracle.potential(cfgs[k], x[s], F[s], vol[s], d)
                                for k, s in ((1e3, soft), (4e4, ~soft)))
            fd = (phi(e) - phi(-e)) / (2 * h)
            assert -fd == pytest.approx(gf[node, a], rel=1e-5, abs=1e-7 * np.abs(gf).max())


def test_mixed_step_conserves_momentum():
    x, v, B, F, _, mu, lam, cfgs = _setup("fcr", seed=4)
    n = len(x)
    cfg = cfgs[1e3]
    m = np.ones(n)
    p0, l0 = oracle.momentum_particles(cfg, x, v, B, m)
    x1, v1, B1, F1, bad = oracle.step(cfg, x, v, B, F, m, np.full(n, 1e-4), nsteps=3, mu=mu, lam=lam)
    p1, l1 = oracle.momentum_particles(cfg, x1, v1, B1, m)
    assert bad == 0
    assert np.abs(p1 - p0).max() <= 1e-12 * np.abs(v).sum()
    assert np.abs(l1 - l0).max() <= 1e-12 * (np.abs(v).sum() + np.abs(B).sum())
