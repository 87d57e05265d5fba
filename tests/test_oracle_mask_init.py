"""Pins of the mask-based initialisation oracle (Sec. 5 initialises by
mask-based covariance estimation; the steps are the readings stated in
oracle/mask_init.py), each against something independent of the oracle's
own formulas: numpy's weighted covariance, scipy's generalized Hermitian
eigensolver, constructed jointly diagonalisable covariances, a dense inverse.
"""
import numpy as np
import scipy.linalg as sl

from oracle import mask_init as mi

rng = np.random.default_rng(11)


def _cn(shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def _offdiag(R, P):
    M = np.einsum("fai,fjab,fbk->fjik", P.conj(), R, P)
    I = P.shape[1]
    d = np.einsum("fjii->fji", M)[..., None] * np.eye(I)
    return float(np.max(np.abs(M - d)) / np.max(np.abs(M)))


def test_masked_covariance_is_the_weighted_second_moment():
    """R_j = sum m y y^H / sum m is numpy's weighted covariance plus the outer
    product of the weighted mean (np.cov subtracts the mean)."""
    I, J, F, N = 3, 2, 2, 40
    y = _cn((I, F, N))
    m = rng.uniform(0.0, 1.0, (J, F, N))
    R = mi.masked_covariances(y, m)
    for f in range(F):
        for j in range(J):
            c = np.cov(y[:, f, :], aweights=m[j, f], bias=True)
            mu = (y[:, f, :] * m[j, f]).sum(axis=1) / m[j, f].sum()
            assert np.allclose(R[f, j], c + np.outer(mu, mu.conj()), rtol=1e-12, atol=1e-14)


def test_two_sources_are_diagonalised_exactly():
    """J = 2: the start is the GEVD; both covariances become diagonal and the
    ratios lambda_1 / (lambda_1 + lambda_2) are scipy's generalized
    eigenvalues of (R_1, R_1 + R_2), in ascending order."""
    I, F = 3, 3
    X = _cn((F, 2, I, 60))
    R = np.einsum("fjan,fjbn->fjab", X, X.conj()) / 60
    P, lam = mi.joint_diagonaliser(R, sweeps=0)
    assert _offdiag(R, P) < 1e-12
    for f in range(F):
        w = sl.eigh(R[f, 0], R[f, 0] + R[f, 1], eigvals_only=True)
        assert np.allclose(lam[f, 0] / (lam[f, 0] + lam[f, 1]), w, rtol=1e-10)


def test_jointly_diagonalisable_sources_are_recovered():
    """R_j = Q^{-H} D_j Q^{-1} for three sources: P diagonalises every R_j and
    the columns of P are those of Q up to scale and order (the ratios
    lambda_1i / lambda_2i are the D_1 / D_2 ratios)."""
    I, J, F = 4, 3, 3
    Q = np.eye(I) + 0.3 * _cn((F, I, I))
    D = np.exp(rng.standard_normal((F, J, I)))
    Qi = np.linalg.inv(Q)
    R = np.einsum("fba,fjb,fbc->fjac", Qi.conj(), D, Qi)
    P, lam = mi.joint_diagonaliser(R, sweeps=0)
    assert _offdiag(R, P) < 1e-10
    for f in range(F):
        assert np.allclose(np.sort(lam[f, 0] / lam[f, 1]), np.sort(D[f, 0] / D[f, 1]), rtol=1e-8)


def test_an_exact_joint_diagonaliser_is_a_fixed_point():
    """From an exact joint diagonaliser the alternations leave P where it is
    (p_i^H V_i p_i = 1, so Eq. FPI returns the same columns)."""
    I, J, F = 3, 3, 2
    Q = np.eye(I) + 0.3 * _cn((F, I, I))
    D = np.exp(rng.standard_normal((F, J, I)))
    Qi = np.linalg.inv(Q)
    R = np.einsum("fba,fjb,fbc->fjac", Qi.conj(), D, Qi)
    P0, _ = mi.joint_diagonaliser(R, sweeps=0)
    P1, _ = mi.joint_diagonaliser(R, sweeps=10)
    assert np.allclose(P1, P0, rtol=1e-10, atol=1e-12)


def test_sweeps_raise_the_criterion():
    """On covariances that no P diagonalises jointly (three sources) the
    alternations raise the criterion they maximise."""
    I, J, F = 3, 3, 4
    X = _cn((F, J, I, 40))
    R = np.einsum("fjan,fjbn->fjab", X, X.conj()) / 40
    crit = [mi.ajd_criterion(R, *mi.joint_diagonaliser(R, s)) for s in range(6)]
    assert np.all(np.diff(np.array(crit), axis=0) > 0)


def test_largest_entry_of_each_column_is_real_positive():
    X = _cn((2, 3, 3, 30))
    R = np.einsum("fjan,fjbn->fjab", X, X.conj()) / 30
    P = mi.gevd_start(R)
    for f in range(2):
        for i in range(3):
            z = P[f, np.argmax(np.abs(P[f, :, i])), i]
            assert abs(z.imag) < 1e-14 * abs(z) and z.real > 0


def test_initial_v_is_the_masked_quadratic_form():
    """v_j = max(m_j, delta) (1/I) y^H S_j^{-1} y with S_j = P^{-H} Lambda_j
    P^{-1} formed densely and solved."""
    I, J, F, N = 3, 2, 2, 15
    y = _cn((I, F, N))
    m = rng.uniform(0.0, 1.0, (J, F, N))
    m[0, 0, :4] = 0.0
    v, lam, P = mi.mask_init(y, m, sweeps=3, delta=1e-3)
    for f in range(F):
        Pi = np.linalg.inv(P[f])
        for j in range(J):
            S = Pi.conj().T @ np.diag(lam[f, j]) @ Pi
            q = np.einsum("an,an->n", y[:, f].conj(), np.linalg.solve(S, y[:, f])).real / I
            assert np.allclose(v[j, f], np.maximum(m[j, f], 1e-3) * q, rtol=1e-10)
    assert np.all(v > 0)
