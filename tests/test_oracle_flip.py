"""Pins of the oracle's FLIP transfer and PIC/FLIP blend (the
FLIP update is the one the paper states in Sec. 1, the blend weight is an extension):
alpha = 0 is PIC exactly; with no force and no gravity the grid leaves velocities unchanged,
so FLIP keeps every particle velocity exactly where PIC filters them; gravity alone adds
dt g to every velocity (partition of unity); linear momentum is conserved by every blend
with elastic forces (lumped mass: sum_p m_p sum_i w (v~_i - v_i) = sum_i m_i (v~_i - v_i))."""
import numpy as np
import pytest

import oracle
from paper_1603_06188_gb300 import scenes

RES = 12


def _state(seed, n=150):
    rng = np.random.default_rng(seed)
    x = scenes.random_particles(rng, n, 3, (RES,) * 3, 1 / RES, margin=3)
    v = rng.normal(size=(n, 3))
    B = np.zeros((n, 3, 3))
    F = scenes.random_deformation(rng, n, 3, 0.1)
    return x, v, B, F


def _cfg(transfer, alpha=1.0, model="none", gravity=(0.0, 0.0, 0.0), dt=1e-3):
    return oracle.make_cfg(dim=3, order=2, transfer=transfer, res=(RES,) * 3, dx=1 / RES, dt=dt, gravity=gravity,
                           model=model, E=1e3, nu=0.3, flip_alpha=alpha)


def test_alpha_zero_is_pic():
    x, v, B, F = _state(0)
    a = oracle.step(_cfg("pic", model="fcr"), x, v, B, F, 1.0, 1e-4, nsteps=2)
    b = oracle.step(_cfg("flip", 0.0, model="fcr"), x, v, B, F, 1.0, 1e-4, nsteps=2)
    for u, w in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(u, w)


def test_flip_keeps_velocities_when_the_grid_does_nothing():
    x, v, B, F = _state(1)
    _, vf, Bf, _, bad = oracle.step(_cfg("flip"), x, v, B, F, 1.0, 1e-4)
    assert bad == 0
    np.testing.assert_array_equal(vf, v)
    assert np.all(Bf == 0)
    _, vp, _, _, _ = oracle.step(_cfg("pic"), x, v, B, F, 1.0, 1e-4)
    assert np.abs(vp - v).max() > 0.1          # PIC filters the same random field


@pytest.mark.parametrize("alpha", [1.0, 0.97])
def test_gravity_alone_adds_dt_g(alpha):
    x, v, B, F = _state(2)
    g = (0.0, -9.8, 2.0)
    dt = 1e-3
    _, vf, _, _, _ = oracle.step(_cfg("flip", alpha, gravity=g, dt=dt), x, v, B, F, 1.0, 1e-4)
    _, vpic, _, _, _ = oracle.step(_cfg("pic", gravity=g, dt=dt), x, v, B, F, 1.0, 1e-4)
    expect = alpha * (v + dt * np.array(g)) + (1 - alpha) * vpic
    np.testing.assert_allclose(vf, expect, rtol=0, atol=1e-13)


@pytest.mark.parametrize("alpha", [1.0, 0.95, 0.0])
def test_blends_conserve_linear_momentum(alpha):
    x, v, B, F = _state(3)
    m = np.ones(len(x))
    cfg = _cfg("flip", alpha, model="fcr", dt=5e-3)
    p0 = (m[:, None] * v).sum(axis=0)
    _, v1, _, _, bad = oracle.step(cfg, x, v, B, F, m, 1e-4, nsteps=3)
    assert bad == 0
    p1 = (m[:, None] * v1).sum(axis=0)
    assert np.abs(p1 - p0).max() <= 1e-12 * np.abs(v).sum()
