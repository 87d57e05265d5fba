"""Pins of the FP64 oracle against routes other than itself.

Each test checks an oracle function against something the paper or the
mathematics fixes: dense covariance algebra (the full I x I matrices the
joint diagonalisation avoids), the Q-function the M-step maximises, the
Kronecker form of the fixed-point equation, finite differences of the
log-likelihood, exact identities of the Wiener filter, the generalised-EM
monotonicity guarantee, the FCA <-> FastFCA-AS correspondence, the scale
gauge of the model, and the operation counts the paper prints.
"""
import json
import os

import numpy as np
import pytest

from oracle import fastfca_as as ffa
from oracle import fca
from oracle.fastfca_as import OpCounter
from paper_1805_09498_gb300.synth import make_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SHAPES = [(3, 3, 2, 7), (2, 3, 3, 6), (1, 2, 2, 5), (4, 2, 2, 9), (3, 1, 2, 6), (2, 4, 1, 8)]


def _prob(I, J, F, N, seed=0):
    return make_problem(I, J, F, N, seed=seed)


# ------------------------------------------------------- dense helpers ----
def dense_R(v, lam, P):
    """R_j(n,f) = v_j P^{-H} Lambda_j P^{-1} built as full matrices.  [J,F,N,I,I]"""
    J, F, N = v.shape
    I = P.shape[1]
    R = np.empty((J, F, N, I, I), dtype=complex)
    for f in range(F):
        Pinv = np.linalg.inv(P[f])
        for j in range(J):
            S = Pinv.conj().T @ np.diag(lam[f, j]) @ Pinv
            for n in range(N):
                R[j, f, n] = v[j, f, n] * S
    return R


def dense_logpdf(y, R):
    """ln CN(y; 0, R) via a Cholesky factor, R = L L^H.  y [I,F,N], R [F,N,I,I]."""
    I, F, N = y.shape
    out = np.empty((F, N))
    for f in range(F):
        for n in range(N):
            L = np.linalg.cholesky(R[f, n])
            z = np.linalg.solve(L, y[:, f, n])
            out[f, n] = (-I * np.log(np.pi) - 2 * np.sum(np.log(np.abs(np.diag(L))))
                         - np.vdot(z, z).real)
    return out


# -------------------------------------------------------------- tests ----
@pytest.mark.parametrize("shape", SHAPES)
def test_loglik_equals_dense_density(shape):
    """Eq. L2 closed form == dense ln CN(y; 0, sum_j v_j P^-H Lambda_j P^-1)."""
    p = _prob(*shape)
    R = dense_R(p.v0, p.lam0, p.P0).sum(axis=0)
    ref = dense_logpdf(p.y, R)
    got = ffa.loglik_terms(p.y, p.v0, p.lam0, p.P0)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("shape", SHAPES)
def test_estep_equals_dense_posterior(shape):
    """Eqs. mutilde0/Phitilde0 == P^H mu_j and P^H Phi_j P of dense Eqs. MMSE/postquadexp;
    the transformed posterior covariance is diagonal."""
    p = _prob(*shape, seed=1)
    I, J, F, N = p.I, p.J, p.F, p.N
    Rj = dense_R(p.v0, p.lam0, p.P0)
    R = Rj.sum(axis=0)
    mu, phi = ffa.e_step(p.y, p.v0, p.lam0, p.P0)
    for j in range(J):
        for f in range(F):
            PH = p.P0[f].conj().T
            for n in range(N):
                Ri = np.linalg.inv(R[f, n])
                mu_d = Rj[j, f, n] @ Ri @ p.y[:, f, n]
                Phi_d = Rj[j, f, n] - Rj[j, f, n] @ Ri @ Rj[j, f, n]
                np.testing.assert_allclose(PH @ mu_d, mu[j, :, f, n], rtol=1e-10, atol=1e-12)
                Pt = PH @ Phi_d @ p.P0[f]
                # posterior covariance is bounded by the prior v_j Lambda_j
                scale = p.v0[j, f, n] * p.lam0[f, j].max()
                np.testing.assert_allclose(np.diag(Pt).real, phi[j, :, f, n], rtol=1e-9,
                                           atol=1e-12 * scale)
                off = Pt - np.diag(np.diag(Pt))
                assert np.abs(off).max() <= 1e-10 * scale


def _q_function(v, lam, P, mu_full, Phi_full):
    """Q(Psi) of Sec. 4.4.1 written with full matrices:
    -sum [ ln det(v_j P^-H Lambda_j P^-1) + tr((v_j Lambda_j)^{-1} (Phi~_j + mu~_j mu~_j^H)) ]."""
    J, F, N = v.shape
    total = 0.0
    for f in range(F):
        Pinv = np.linalg.inv(P[f])
        for j in range(J):
            S = Pinv.conj().T @ np.diag(lam[f, j]) @ Pinv
            for n in range(N):
                C = Phi_full[j, f, n] + np.outer(mu_full[j, f, n], mu_full[j, f, n].conj())
                _, ld = np.linalg.slogdet(v[j, f, n] * S)
                tr = np.trace(np.linalg.inv(v[j, f, n] * np.diag(lam[f, j])) @ C).real
                total -= ld + tr
    return total


@pytest.mark.parametrize("shape", [(3, 3, 2, 5), (2, 3, 2, 4), (1, 2, 1, 4)])
def test_mstep_maximises_q_function(shape):
    """Eq. updatev maximises Q over v at the current Lambda; Eq. Lambdaupdate
    maximises Q over Lambda at the new v (central differences of the dense Q)."""
    p = _prob(*shape, seed=2)
    J, F, N, I = p.J, p.F, p.N, p.I
    # posterior statistics from the dense route, transformed by P^H
    Rj = dense_R(p.v0, p.lam0, p.P0)
    R = Rj.sum(axis=0)
    mu_full = np.empty((J, F, N, I), complex)
    Phi_full = np.empty((J, F, N, I, I), complex)
    for j in range(J):
        for f in range(F):
            for n in range(N):
                Ri = np.linalg.inv(R[f, n])
                mu_full[j, f, n] = p.P0[f].conj().T @ (Rj[j, f, n] @ Ri @ p.y[:, f, n])
                Phi_full[j, f, n] = p.P0[f].conj().T @ (
                    Rj[j, f, n] - Rj[j, f, n] @ Ri @ Rj[j, f, n]) @ p.P0[f]
    mu, phi = ffa.e_step(p.y, p.v0, p.lam0, p.P0)
    v1 = ffa.m_step_v(mu, phi, p.lam0)
    lam1 = ffa.m_step_lambda(mu, phi, v1)
    h = 1e-5
    # d Q / d log v_j(n,f) == 0 at v1 (with Lambda = lam0)
    for idx in np.ndindex(v1.shape):
        vp = v1.copy(); vp[idx] *= np.exp(h)
        vm = v1.copy(); vm[idx] *= np.exp(-h)
        d = (_q_function(vp, p.lam0, p.P0, mu_full, Phi_full)
             - _q_function(vm, p.lam0, p.P0, mu_full, Phi_full)) / (2 * h)
        assert abs(d) < 1e-5 * (1 + I), (idx, d)
    # d Q / d log lambda_ji(f) == 0 at lam1 (with v = v1)
    for idx in np.ndindex(lam1.shape):
        lp = lam1.copy(); lp[idx] *= np.exp(h)
        lm = lam1.copy(); lm[idx] *= np.exp(-h)
        d = (_q_function(v1, lp, p.P0, mu_full, Phi_full)
             - _q_function(v1, lm, p.P0, mu_full, Phi_full)) / (2 * h)
        assert abs(d) < 1e-5 * N, (idx, d)
    # and it is a maximum: random perturbations lower Q
    q0 = _q_function(v1, lam1, p.P0, mu_full, Phi_full)
    rng = np.random.default_rng(5)
    for _ in range(3):
        vp = v1 * np.exp(0.05 * rng.standard_normal(v1.shape))
        lp = lam1 * np.exp(0.05 * rng.standard_normal(lam1.shape))
        assert _q_function(vp, lp, p.P0, mu_full, Phi_full) < q0


@pytest.mark.parametrize("shape", SHAPES)
def test_wiener_identities(shape):
    """Eq. MMSE0: the J estimates sum to the mixture, and equal the dense
    R_j (sum_k R_k)^{-1} y."""
    p = _prob(*shape, seed=3)
    xh = ffa.wiener(p.y, p.v0, p.lam0, p.P0)
    np.testing.assert_allclose(xh.sum(axis=0), p.y, rtol=1e-11, atol=1e-12)
    Rj = dense_R(p.v0, p.lam0, p.P0)
    R = Rj.sum(axis=0)
    for j in range(p.J):
        for f in range(p.F):
            for n in range(p.N):
                ref = Rj[j, f, n] @ np.linalg.solve(R[f, n], p.y[:, f, n])
                np.testing.assert_allclose(xh[j, :, f, n], ref, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("shape", SHAPES)
def test_fixed_point_equals_kronecker_form(shape):
    """Eq. FPI (column-wise) == Eq. vecP solved as one I^2 x I^2 system,
    [(1/N) sum_n D^{-1} kron y y^H]^{-1} vec(P^{-H}), vec stacking columns."""
    p = _prob(*shape, seed=4)
    I, F, N = p.I, p.F, p.N
    V = ffa.weighted_covariances(p.y, p.v0, p.lam0)
    got = ffa.fixed_point_P(p.P0, V, K=1, counter=OpCounter())
    D = np.einsum("jfn,fji->fni", p.v0, p.lam0)       # sigma, summed independently
    for f in range(F):
        M = np.zeros((I * I, I * I), complex)
        for n in range(N):
            yy = np.outer(p.y[:, f, n], p.y[:, f, n].conj())
            M += np.kron(np.diag(1.0 / D[f, n]), yy)
        M /= N
        rhs = np.linalg.inv(p.P0[f]).conj().T.reshape(-1, order="F")
        ref = np.linalg.solve(M, rhs).reshape(I, I, order="F")
        np.testing.assert_allclose(got[f], ref, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("shape", [(3, 3, 1, 6), (2, 2, 2, 5), (4, 3, 1, 9)])
def test_gradient_matches_finite_differences(shape):
    """Eq. partialP (Wirtinger derivative w.r.t. P^*) == 1/2 (d/dRe + i d/dIm)
    of the dense log-likelihood, by central differences."""
    p = _prob(*shape, seed=6)
    G = ffa.grad_P_conj(p.y, p.v0, p.lam0, p.P0)

    def L(P):
        R = dense_R(p.v0, p.lam0, P).sum(axis=0)
        return dense_logpdf(p.y, R).sum()

    h = 1e-6
    for f in range(p.F):
        for a in range(p.I):
            for i in range(p.I):
                E = np.zeros_like(p.P0); E[f, a, i] = h
                dre = (L(p.P0 + E) - L(p.P0 - E)) / (2 * h)
                dim = (L(p.P0 + 1j * E) - L(p.P0 - 1j * E)) / (2 * h)
                fd = 0.5 * (dre + 1j * dim)
                assert abs(fd - G[f, a, i]) <= 1e-5 * (1 + abs(G[f, a, i])), (f, a, i, fd, G[f, a, i])


def test_fixed_point_scalar_closed_form():
    """I = 1: Eq. FPI is p <- (1/V) / conj(p) = p / (V |p|^2) with
    V = (1/N) sum_n |y|^2 / sigma."""
    p = _prob(1, 3, 3, 11, seed=7)
    sigma = np.einsum("jfn,fj->fn", p.v0, p.lam0[:, :, 0])
    Vs = np.mean(np.abs(p.y[0]) ** 2 / sigma, axis=1)
    ref = p.P0[:, 0, 0] / (Vs * np.abs(p.P0[:, 0, 0]) ** 2)
    V = ffa.weighted_covariances(p.y, p.v0, p.lam0)
    got = ffa.fixed_point_P(p.P0, V, K=1, counter=OpCounter())[:, 0, 0]
    np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_fixed_point_scalar_is_involution():
    """I = 1: applying Eq. FPI twice returns the starting p (the column scale
    alternates c -> 1/c), which is why a plain fixed-point iteration at fixed
    v, Lambda is not expected to converge in scale."""
    p = _prob(1, 2, 4, 13, seed=14)
    V = ffa.weighted_covariances(p.y, p.v0, p.lam0)
    P2 = ffa.fixed_point_P(p.P0, V, K=2, counter=OpCounter())
    np.testing.assert_allclose(P2, p.P0, rtol=1e-12)


def test_stationary_point_is_fixed_point():
    """A stationary point of L2 in P (zero gradient, Eq. partialP) is a fixed
    point of Eq. FPI.  The stationary point is found by the fixed-point map
    followed by the rescaling p_i <- p_i / sqrt(p_i^H V_i p_i), which is the
    identity wherever the gradient vanishes (there p_i^H V_i p_i = 1)."""
    p = _prob(3, 3, 2, 400, seed=8)
    V = ffa.weighted_covariances(p.y, p.v_true, p.lam_true)
    P = p.P0.copy()
    for _ in range(1500):
        P = ffa.fixed_point_P(P, V, K=1, counter=OpCounter())
        d = np.einsum("fai,fiab,fbi->fi", P.conj(), V, P).real
        P = P / np.sqrt(d)[:, None, :]
    G = ffa.grad_P_conj(p.y, p.v_true, p.lam_true, P)
    assert np.abs(G).max() < 1e-9 * p.N
    np.testing.assert_allclose(ffa.fixed_point_P(P, V, K=1, counter=OpCounter()), P,
                               rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_em_half_does_not_decrease_loglik(seed):
    """The EM half is a generalised EM step (coordinate maxima of Q), so
    L2 (evaluated densely) does not decrease across it."""
    p = _prob(3, 3, 3, 40, seed=seed)
    v, lam, P = p.v0, p.lam0, p.P0
    for _ in range(5):
        before = dense_logpdf(p.y, dense_R(v, lam, P).sum(axis=0)).sum()
        v, lam = ffa.em_half(p.y, v, lam, P)
        after = dense_logpdf(p.y, dense_R(v, lam, P).sum(axis=0)).sum()
        assert after >= before - 1e-9 * abs(before)
        V = ffa.weighted_covariances(p.y, v, lam)
        P = ffa.fixed_point_P(P, V, 1, counter=OpCounter())


@pytest.mark.parametrize("seed", [0, 1])
def test_fca_loglik_monotone(seed):
    """Conventional FCA is an EM algorithm: L1 does not decrease."""
    p = _prob(3, 3, 2, 30, seed=seed)
    S = fca.spatial_from_joint(p.P0, p.lam0)
    _, _, tr = fca.iterate(p.y, p.v0, S, 8, counter=OpCounter())
    assert np.all(np.diff(tr) >= -1e-9 * np.abs(tr[:-1]))


@pytest.mark.parametrize("shape", [(3, 3, 2, 6), (2, 3, 2, 5), (4, 2, 1, 7)])
def test_fca_dense_loglik(shape):
    """Eq. L1 of the FCA oracle == Cholesky log density of sum_j v_j S_j."""
    p = _prob(*shape, seed=9)
    S = fca.spatial_from_joint(p.P0, p.lam0)
    R = (p.v0[:, :, :, None, None] * S.transpose(1, 0, 2, 3)[:, :, None]).sum(axis=0)
    np.testing.assert_allclose(fca.loglik_terms(p.y, p.v0, S), dense_logpdf(p.y, R), rtol=1e-11)


@pytest.mark.parametrize("shape", [(3, 3, 2, 9), (2, 3, 3, 6), (4, 4, 1, 10)])
def test_fca_and_fastfca_agree_from_joint_state(shape):
    """Started from S_j = P^-H Lambda_j P^-1 (Eq. diagconst): L1 == L2, the
    FCA v update (Eq. vupdate) == the FastFCA-AS one (Eq. updatev), and the
    diagonal of P^H S_j^new P (Eq. Supdate) == Lambda_j^new (Eq. Lambdaupdate)."""
    p = _prob(*shape, seed=10)
    S = fca.spatial_from_joint(p.P0, p.lam0)
    np.testing.assert_allclose(fca.loglik(p.y, p.v0, S), ffa.loglik(p.y, p.v0, p.lam0, p.P0),
                               rtol=1e-12)
    v_f, S_f = fca.iteration(p.y, p.v0, S, counter=OpCounter())
    v_a, lam_a = ffa.em_half(p.y, p.v0, p.lam0, p.P0)
    np.testing.assert_allclose(v_f, v_a, rtol=1e-10)
    D = np.einsum("fba,fjbc,fcd->fjad", p.P0.conj(), S_f, p.P0)
    np.testing.assert_allclose(np.diagonal(D, axis1=2, axis2=3).real, lam_a, rtol=1e-10)
    # the FCA Wiener filter equals the FastFCA-AS one on the same model
    np.testing.assert_allclose(fca.wiener(p.y, p.v0, S), ffa.wiener(p.y, p.v0, p.lam0, p.P0),
                               rtol=1e-9, atol=1e-12)


def test_scale_gauge_equivariance():
    """P -> P diag(c), lambda_ji -> |c_i|^2 lambda_ji and v_j -> a_j v_j,
    lambda_j -> lambda_j / a_j leave the model unchanged; the iteration is
    equivariant: the trajectories differ by the same gauge, and the
    gauge-invariant quantities (L2, Wiener output) are identical."""
    p = _prob(3, 3, 2, 25, seed=11)
    rng = np.random.default_rng(3)
    c = (0.5 + rng.random((p.F, p.I))) * np.exp(2j * np.pi * rng.random((p.F, p.I)))
    a = 0.5 + rng.random((p.J, p.F))
    P2 = p.P0 * c[:, None, :]
    lam2 = p.lam0 * np.abs(c[:, None, :]) ** 2 / a.T[:, :, None]
    v2 = p.v0 * a[:, :, None]
    A = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 6, counter=OpCounter())
    B = ffa.iterate(p.y, v2, lam2, P2, 6, counter=OpCounter())
    np.testing.assert_allclose(A[3], B[3], rtol=1e-9)
    # the parameters carry the gauge along unchanged
    np.testing.assert_allclose(A[0] * a[:, :, None], B[0], rtol=1e-8)
    np.testing.assert_allclose(A[1] * np.abs(c[:, None, :]) ** 2 / a.T[:, :, None], B[1],
                               rtol=1e-8)
    np.testing.assert_allclose(A[2] * c[:, None, :], B[2], rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(ffa.wiener(p.y, *A[:3]), ffa.wiener(p.y, *B[:3]),
                               rtol=1e-8, atol=1e-10)


def test_operation_counts_match_paper():
    """Sec. 3.4 / 4.5 print the matrix inversions and multiplications per
    iteration at I = J = 3, N = 249, F = 512, K = 1; the oracle's counters,
    incremented where it inverts or multiplies matrices, reproduce them."""
    g = json.load(open(os.path.join(GOLDEN, "op_counts.json")))
    c = g["fca"]
    p = _prob(c["I"], c["J"], c["F"], c["N"], seed=12)
    cnt = OpCounter()
    S = fca.spatial_from_joint(p.P0, p.lam0)
    fca.iteration(p.y, p.v0, S, counter=cnt)
    assert cnt.inversions == c["inversions"]
    assert cnt.multiplications == c["multiplications"]
    a = g["fastfca_as"]
    cnt = OpCounter()
    ffa.hybrid_iteration(p.y, p.v0, p.lam0, p.P0, K=a["K"], counter=cnt)
    assert cnt.inversions == a["inversions"]
    assert cnt.multiplications == a["multiplications"]


def test_iteration_increases_loglik_overall():
    """Statistical sanity (not a parity check): twenty hybrid iterations from
    the perturbed truth raise L2 well above its starting value."""
    p = _prob(3, 3, 4, 300, seed=13)
    _, _, _, tr = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 20, counter=OpCounter())
    assert tr[-1] > tr[0]
