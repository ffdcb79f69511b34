"""Pins of the oracle's SVD, polar rotation and fixed-corotated stress (Sec. 3.1: P = dPsi/dF)
against numpy's SVD, finite differences of the energy and invariances."""
import numpy as np
import pytest

import oracle

MU, LAM = oracle.lame(1e4, 0.3)


def _rot(rng, d):
    Q, _ = np.linalg.qr(rng.normal(size=(d, d)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


@pytest.mark.parametrize("d", [2, 3])
def test_svd_and_polar_against_numpy(d):
    rng = np.random.default_rng(0)
    mats = [rng.normal(size=(d, d)) for _ in range(200)]
    mats += [np.eye(d), np.diag([2.0] + [1.0] * (d - 1)), np.diag([1.0] * (d - 1) + [-1.0])]
    mats += [np.eye(d) + 1e-9 * rng.normal(size=(d, d)) for _ in range(10)]   # nearly equal sigmas
    mats += [np.outer(rng.normal(size=d), rng.normal(size=d))]                # rank one
    for F in mats:
        U, s, V = oracle.svd(F)
        np.testing.assert_allclose(U @ np.diag(s) @ V.T, F, atol=1e-12)
        np.testing.assert_allclose(U.T @ U, np.eye(d), atol=1e-12)
        np.testing.assert_allclose(V.T @ V, np.eye(d), atol=1e-12)
        assert np.linalg.det(U) == pytest.approx(1.0, abs=1e-12)
        assert np.linalg.det(V) == pytest.approx(1.0, abs=1e-12)
        ref = np.linalg.svd(F, compute_uv=False)
        np.testing.assert_allclose(np.sort(np.abs(s)), np.sort(ref), atol=1e-12)
        R = oracle.polar(F)
        np.testing.assert_allclose(R.T @ R, np.eye(d), atol=1e-12)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
        S = R.T @ F
        np.testing.assert_allclose(S, S.T, atol=1e-11)
        if np.linalg.det(F) > 1e-6:
            # numpy polar factor (unique for invertible F with det > 0)
            u, sv, vt = np.linalg.svd(F)
            np.testing.assert_allclose(R, u @ vt, atol=1e-10)


@pytest.mark.parametrize("d", [2, 3])
def test_stress_is_energy_derivative(d):
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(20):
        F = np.eye(d) + 0.3 * rng.uniform(-1, 1, size=(d, d))
        if np.linalg.det(F) < 0.2:
            continue
        P = oracle.stress_fcr(F, MU, LAM)
        fd = np.zeros_like(F)
        for a in range(d):
            for b in range(d):
                E = np.zeros_like(F); E[a, b] = h
                fd[a, b] = (oracle.psi_fcr(F + E, MU, LAM) - oracle.psi_fcr(F - E, MU, LAM)) / (2 * h)
        np.testing.assert_allclose(P, fd, rtol=1e-6, atol=1e-6 * np.abs(P).max())


@pytest.mark.parametrize("d", [2, 3])
def test_stress_invariances(d):
    rng = np.random.default_rng(2)
    for _ in range(20):
        Q = _rot(rng, d)
        # a pure rotation is stress free
        np.testing.assert_allclose(oracle.stress_fcr(Q, MU, LAM), 0.0, atol=1e-9)
        F = np.eye(d) + 0.3 * rng.uniform(-1, 1, size=(d, d))
        P = oracle.stress_fcr(F, MU, LAM)
        # frame indifference P(QF) = Q P(F), and P F^T symmetric (used in Sec. 5.3)
        np.testing.assert_allclose(oracle.stress_fcr(Q @ F, MU, LAM), Q @ P, atol=1e-8 * np.abs(P).max())
        tau = P @ F.T
        np.testing.assert_allclose(tau, tau.T, atol=1e-9 * np.abs(tau).max())
        # energy minimum at rotations
        assert oracle.psi_fcr(Q, MU, LAM) == pytest.approx(0.0, abs=1e-12)
        assert oracle.psi_fcr(F, MU, LAM) > 0.0


def test_stress_closed_form_uniaxial():
    # F = diag(s, 1, 1): R = I, P = diag(2 mu (s-1) + lam (s-1), lam (s-1) s, lam (s-1) s)
    s = 1.1
    F = np.diag([s, 1.0, 1.0])
    P = oracle.stress_fcr(F, MU, LAM)
    exp = np.diag([2 * MU * (s - 1) + LAM * (s - 1), LAM * (s - 1) * s, LAM * (s - 1) * s])
    np.testing.assert_allclose(P, exp, rtol=1e-12)
