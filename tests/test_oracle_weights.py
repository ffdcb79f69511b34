"""Pins of the oracle's interpolation weights (Sec. 3.5) against closed forms, the paper's
printed inertia entries (Sec. 5.6) and brute force over every grid node."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bspline_inertia.json")


def _cfg(dim, order, res=12, dx=0.125):
    return oracle.make_cfg(dim=dim, order=order, res=(res,) * dim, dx=dx)


@pytest.mark.parametrize("order", [2, 3])
def test_bspline_knot_values_and_unit_integral(order):
    # textbook values of the cardinal B-splines at the integers / half-integers
    if order == 2:
        pins = {0.0: 0.75, 0.5: 0.5, 1.0: 0.125, 1.5: 0.0, 2.0: 0.0}
    else:
        pins = {0.0: 2.0 / 3.0, 1.0: 1.0 / 6.0, 2.0: 0.0, 0.5: 23.0 / 48.0, 1.5: 1.0 / 48.0}
    for t, val in pins.items():
        assert oracle.N(order, t) == pytest.approx(val, abs=1e-15)
        assert oracle.N(order, -t) == pytest.approx(val, abs=1e-15)
    ts = np.linspace(-3, 3, 600001)
    vals = np.array([oracle.N(order, t) for t in ts[::10]])
    integral = np.trapezoid(vals, ts[::10])
    assert integral == pytest.approx(1.0, abs=1e-8)


@pytest.mark.parametrize("order", [2, 3])
def test_bspline_derivative_matches_finite_difference(order):
    h = 1e-6
    for t in np.linspace(-2.2, 2.2, 97):
        fd = (oracle.N(order, t + h) - oracle.N(order, t - h)) / (2 * h)
        assert oracle.dN(order, t) == pytest.approx(fd, abs=1e-6)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("order", [2, 3])
def test_weight_identities(dim, order):
    """Sec. 3.5: sum w = 1, sum w x_i = x_p, sum w (x_i - x_p) = 0, sum x_i grad w^T = I,
    and sum grad w = 0 (used by the momentum proof of Sec. 5.2)."""
    c = _cfg(dim, order)
    rng = np.random.default_rng(1)
    for _ in range(50):
        xp = 0.4 + rng.random(dim) * 0.6
        rc, base, w, dw = oracle.stencil(c, xp)
        assert rc == 0
        xi = oracle.stencil_nodes(c, base)
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
        np.testing.assert_allclose(w @ xi, xp, atol=1e-14)
        np.testing.assert_allclose(w @ (xi - xp), 0.0, atol=1e-14)
        np.testing.assert_allclose(xi.T @ dw, np.eye(dim), atol=1e-12)
        np.testing.assert_allclose(dw.sum(0), 0.0, atol=1e-12)
        assert np.all(w >= 0)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("order", [2, 3])
def test_inertia_matches_printed_entries(dim, order):
    """D_p = k I with k = dx^2/4 (quadratic), dx^2/3 (cubic); and the quadratic form
    sum_i w_ip |C (x_i - x_p)|^2 over the paper's affine modes gives the printed diagonal
    of b^T M b (Sec. 5.6, per unit mass)."""
    gold = json.load(open(GOLDEN))["quadratic" if order == 2 else "cubic"]
    dx = 0.0625
    c = _cfg(dim, order, res=20, dx=dx)
    rng = np.random.default_rng(2)
    for _ in range(20):
        xp = 0.4 + rng.random(dim) * 0.4
        rc, base, w, dw = oracle.stencil(c, xp)
        r = oracle.stencil_nodes(c, base) - xp
        D = np.einsum("j,ja,jb->ab", w, r, r)
        k = dx * dx * (0.25 if order == 2 else 1.0 / 3.0)
        np.testing.assert_allclose(D, k * np.eye(dim), atol=1e-15)
        if dim == 3:
            modes = []
            E = lambda a, b: np.outer(np.eye(3)[a], np.eye(3)[b])
            for a, b in [(0, 1), (0, 2), (1, 2)]:
                modes.append(E(a, b) - E(b, a))
            for a, b in [(0, 1), (0, 2), (1, 2)]:
                modes.append(E(a, b) + E(b, a))
            for a in range(3):
                modes.append(E(a, a))
            got = [np.einsum("j,ja,ja->", w, r @ M.T, r @ M.T) / (dx * dx) for M in modes]
            np.testing.assert_allclose(got, gold["diag_over_mp_over_dx2"][3:], atol=1e-13)
            for e in np.eye(3):
                assert np.einsum("j,a,a->", w, e, e) == pytest.approx(gold["translation"][0])


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("order", [2, 3])
def test_stencil_equals_brute_force_over_all_nodes(dim, order):
    res = 10 if dim == 3 else 14
    c = _cfg(dim, order, res=res, dx=0.1)
    rng = np.random.default_rng(3)
    for _ in range(6):
        xp = 0.35 + rng.random(dim) * 0.25
        rc, base, w, dw = oracle.stencil(c, xp)
        wa, dwa = oracle.weights_all(c, xp)
        dense_w = np.zeros_like(wa)
        dense_dw = np.zeros_like(dwa)
        K = order + 1
        for j in range(K ** dim):
            idx, r, mult = 0, j, 1
            for a in range(dim):
                idx += (base[a] + r % K) * mult
                r //= K
                mult *= res
            dense_w[idx] = w[j]
            dense_dw[idx] = dw[j]
        np.testing.assert_allclose(dense_w, wa, atol=1e-15)
        np.testing.assert_allclose(dense_dw, dwa, atol=1e-13)
        assert np.count_nonzero(wa) <= K ** dim


def test_stencil_out_of_grid_is_reported():
    c = _cfg(3, 2, res=8, dx=0.125)
    assert oracle.stencil(c, [0.01, 0.5, 0.5])[0] == -1
    assert oracle.stencil(c, [0.5, 0.5, 0.99])[0] == -1
    assert oracle.stencil(c, [0.5, 0.5, 0.5])[0] == 0
