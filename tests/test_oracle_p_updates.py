"""Pins of the oracle's alternative updates of P (Sec. 4.6: the gradient,
natural gradient and Newton methods in place of the fixed-point iteration).

The paper names these methods without stating them; the oracle's readings
(ascent on L2 with the V_i of Eq. FPI held fixed, K steps of size mu, Eq.
partialP scaled by 1/N) are pinned here by what the mathematics fixes:
the directional derivative of L2 along each step (central differences of
the log-likelihood, itself pinned against the dense density), the closed
forms at I = 1, the equivariance of the natural gradient under a change of
the microphone basis, stationarity at a stationary point of L2, and the
inversion counts; for Newton's method, the stationarity of its quadratic
model checked by central differences of the gradient, its quadratic
convergence and its closed form at I = 1.
"""
import numpy as np
import pytest

from oracle import fastfca_as as ffa
from oracle.fastfca_as import OpCounter
from paper_1805_09498_gb300.synth import cn, make_problem

SHAPES = [(3, 3, 2, 40), (2, 3, 3, 30), (1, 2, 2, 25), (4, 2, 2, 50), (8, 6, 1, 90)]


def _slope(y, v, lam, P, D, rel=1e-5):
    """d/dh L2(P + h D) at h = 0 by central differences."""
    h = rel / np.abs(D).max()
    return (ffa.loglik(y, v, lam, P + h * D) - ffa.loglik(y, v, lam, P - h * D)) / (2 * h)


@pytest.mark.parametrize("shape", SHAPES)
def test_gradient_step_is_the_scaled_wirtinger_gradient(shape):
    """For real L2 and G = dL2/dP^*, dL2 = 2 Re tr(G^H dP).  Along the step
    D = G / N the slope is therefore 2 N ||D||_F^2; any other D of the same
    slope would have a larger norm (Cauchy-Schwarz), so the equality fixes
    D = G / N."""
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=21 + I)
    V = ffa.weighted_covariances(p.y, p.v0, p.lam0)
    D = ffa.gradient_P(p.P0, V, 1.0, counter=OpCounter()) - p.P0
    s = _slope(p.y, p.v0, p.lam0, p.P0, D)
    ref = 2 * N * np.sum(np.abs(D) ** 2)
    assert s > 0
    assert abs(s - ref) <= 1e-6 * ref, (s, ref)


@pytest.mark.parametrize("shape", SHAPES)
def test_natural_gradient_step_slope(shape):
    """Along D = P P^H G / N the slope 2 Re tr(G^H D) equals
    2 N ||P^{-1} D||_F^2 (= 2 ||P^H G||^2 / N): an ascent direction whose
    slope is fixed by P and D alone."""
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=31 + I)
    V = ffa.weighted_covariances(p.y, p.v0, p.lam0)
    D = ffa.natural_gradient_P(p.P0, V, 1.0) - p.P0
    s = _slope(p.y, p.v0, p.lam0, p.P0, D)
    ref = 2 * N * np.sum(np.abs(np.linalg.solve(p.P0, D)) ** 2)
    assert s > 0
    assert abs(s - ref) <= 1e-6 * ref, (s, ref)


def test_scalar_closed_forms():
    """I = 1 with V = (1/N) sum_n |y|^2 / sigma:
    gradient  p <- p + mu (1 / conj(p) - V p);
    natural   p <- p (1 + mu (1 - V |p|^2))."""
    p = make_problem(1, 3, 4, 19, seed=41)
    sigma = np.einsum("jfn,fj->fn", p.v0, p.lam0[:, :, 0])
    Vs = np.mean(np.abs(p.y[0]) ** 2 / sigma, axis=1)
    q = p.P0[:, 0, 0]
    V = ffa.weighted_covariances(p.y, p.v0, p.lam0)
    mu = 0.3
    g = ffa.gradient_P(p.P0, V, mu, counter=OpCounter())[:, 0, 0]
    np.testing.assert_allclose(g, q + mu * (1 / q.conj() - Vs * q), rtol=1e-12)
    nat = ffa.natural_gradient_P(p.P0, V, mu)[:, 0, 0]
    np.testing.assert_allclose(nat, q * (1 + mu * (1 - Vs * np.abs(q) ** 2)), rtol=1e-12)


def test_natural_gradient_is_equivariant():
    """A change of the microphone basis y' = B y with P' = B^{-H} P leaves
    y~ = P^H y unchanged; the natural-gradient step commutes with it
    (step(P', V') = B^{-H} step(P, V)), the plain gradient step does not."""
    I, J, F, N = 3, 3, 3, 60
    p = make_problem(I, J, F, N, seed=51)
    B = np.eye(I)[None] + 0.5 * cn(np.random.default_rng(7), (F, I, I))
    BinvH = np.linalg.inv(B).conj().transpose(0, 2, 1)
    y2 = np.einsum("fab,bfn->afn", B, p.y)
    P2 = BinvH @ p.P0
    V = ffa.weighted_covariances(p.y, p.v0, p.lam0)
    V2 = ffa.weighted_covariances(y2, p.v0, p.lam0)
    mu = 0.2
    nat = ffa.natural_gradient_P(p.P0, V, mu, K=2)
    nat2 = ffa.natural_gradient_P(P2, V2, mu, K=2)
    np.testing.assert_allclose(nat2, BinvH @ nat, rtol=1e-11, atol=1e-12)
    g = ffa.gradient_P(p.P0, V, mu, counter=OpCounter())
    g2 = ffa.gradient_P(P2, V2, mu, counter=OpCounter())
    assert np.abs(g2 - BinvH @ g).max() > 1e-3


def test_steps_vanish_at_a_stationary_point():
    """Where Eq. partialP vanishes both steps leave P unchanged.  The
    stationary point is reached as in the fixed-point pins: Eq. FPI followed
    by the column rescaling p_i <- p_i / sqrt(p_i^H V_i p_i)."""
    p = make_problem(3, 3, 2, 400, seed=8)
    V = ffa.weighted_covariances(p.y, p.v_true, p.lam_true)
    P = p.P0.copy()
    for _ in range(1500):
        P = ffa.fixed_point_P(P, V, K=1, counter=OpCounter())
        d = np.einsum("fai,fiab,fbi->fi", P.conj(), V, P).real
        P = P / np.sqrt(d)[:, None, :]
    np.testing.assert_allclose(ffa.gradient_P(P, V, 0.5, K=3, counter=OpCounter()), P, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(ffa.natural_gradient_P(P, V, 0.5, K=3), P, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("p_update,mu", [("gradient", 0.02), ("natural_gradient", 0.02)])
def test_small_steps_do_not_decrease_loglik(p_update, mu):
    """With the EM half monotone (generalised EM) and a small ascent step in
    P, every iteration raises L2."""
    p = make_problem(3, 3, 4, 200, seed=61)
    _, _, _, tr = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 6, counter=OpCounter(), p_update=p_update, mu=mu)
    assert np.all(np.diff(tr) > 0), np.diff(tr)


def test_inversion_counts():
    """The gradient step inverts P once per frequency per step; the natural
    gradient step inverts nothing."""
    p = make_problem(3, 3, 5, 30, seed=71)
    c = OpCounter()
    ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, K=3, counter=c, p_update="gradient", mu=0.1)
    assert c.inversions == 2 * 3 * 5
    c = OpCounter()
    ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, K=3, counter=c, p_update="natural_gradient", mu=0.1)
    assert c.inversions == 0


# ------------------------------------------------------------ Newton's method
def _stationary(seed=8):
    """A stationary point of L2 in P at fixed V (as in the fixed-point pins)."""
    p = make_problem(3, 3, 2, 400, seed=seed)
    V = ffa.weighted_covariances(p.y, p.v_true, p.lam_true)
    P = p.P0.copy()
    for _ in range(1500):
        P = ffa.fixed_point_P(P, V, K=1, counter=OpCounter())
        d = np.einsum("fai,fiab,fbi->fi", P.conj(), V, P).real
        P = P / np.sqrt(d)[:, None, :]
    return P, V


def _G(P, V):
    """Eq. partialP / N with V fixed: P^{-H} - [V_1 p_1, ..., V_I p_I]."""
    return np.linalg.inv(P).conj().transpose(0, 2, 1) - np.einsum("fiab,fbi->fai", V, P)


def _real(D):
    """Real coordinates of complex I x I matrices (real parts, then imaginary)."""
    F = D.shape[0]
    return np.concatenate([D.real.reshape(F, -1), D.imag.reshape(F, -1)], axis=1)


@pytest.mark.parametrize("shape", [(3, 3, 2, 60), (2, 3, 3, 40), (4, 2, 2, 80), (8, 3, 1, 80)])
def test_newton_step_zeroes_the_linearised_gradient(shape):
    """The Newton step D makes the second-order model stationary in every
    direction that changes L2: the first-order change of the gradient along
    D, dG[D] by central differences of Eq. partialP (independent of the
    Hessian the oracle assembles), cancels G up to the column-phase
    directions i p_i, and D has no component along those."""
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=81 + I)
    V = ffa.weighted_covariances(p.y, p.v0, p.lam0)
    P = p.P0
    D = ffa.newton_P(P, V, 1.0, counter=OpCounter()) - P
    h = 1e-6 / np.abs(D).max()
    R = _G(P, V) + (_G(P + h * D, V) - _G(P - h * D, V)) / (2 * h)   # dl-residual, Wirtinger form
    def turn(i):  # the direction that turns column i in phase: i p_i in column i, zero elsewhere
        T = np.zeros_like(P)
        T[:, :, i] = 1j * P[:, :, i]
        return _real(T)
    turns = np.stack([turn(i) for i in range(I)], axis=2)         # [F, 2 I^2, I]
    Qn, _ = np.linalg.qr(turns)
    Qp = np.eye(2 * I * I)[None] - Qn @ Qn.transpose(0, 2, 1)
    r = np.einsum("fkl,fl->fk", Qp, _real(R))                   # residual off the phase directions
    assert np.abs(r).max() <= 1e-6 * np.abs(_G(P, V)).max()
    assert np.abs(np.einsum("fki,fk->fi", Qn, _real(D))).max() <= 1e-10 * np.abs(D).max()


def test_newton_converges_quadratically_near_a_stationary_point():
    Ps, V = _stationary()
    rng = np.random.default_rng(0)
    P = Ps * (1 + 0.05 * (rng.standard_normal(Ps.shape) + 1j * rng.standard_normal(Ps.shape)))
    err = []
    for _ in range(4):
        P = ffa.newton_P(P, V, 1.0, counter=OpCounter())
        err.append(np.abs(_G(P, V)).max())
    assert err[1] < 1e-2 and err[2] < 1e-5 and err[3] < 1e-10, err
    assert err[3] < 1e3 * err[2] ** 2 + 1e-13  # quadratic (a linear rate would leave ~1e-8)
    np.testing.assert_allclose(ffa.newton_P(Ps, V, 1.0, counter=OpCounter()), Ps, rtol=1e-10, atol=1e-12)


def test_newton_scalar_closed_form():
    """I = 1: l = ln|p|^2 - V |p|^2 depends on r = |p| only; Newton in r is
    r <- r - l'(r) / l''(r) = 2 r / (1 + V r^2), the phase unchanged."""
    p = make_problem(1, 2, 4, 23, seed=91)
    sigma = np.einsum("jfn,fj->fn", p.v0, p.lam0[:, :, 0])
    Vs = np.mean(np.abs(p.y[0]) ** 2 / sigma, axis=1)
    q = p.P0[:, 0, 0]
    V = ffa.weighted_covariances(p.y, p.v0, p.lam0)
    got = ffa.newton_P(p.P0, V, 1.0, counter=OpCounter())[:, 0, 0]
    np.testing.assert_allclose(got, q * 2.0 / (1.0 + Vs * np.abs(q) ** 2), rtol=1e-10)


def test_newton_inversion_count():
    p = make_problem(3, 3, 5, 30, seed=72)
    c = OpCounter()
    ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, K=3, counter=c, p_update="newton", mu=1.0)
    assert c.inversions == 2 * 3 * 5 * 2


# ------------------------------------------------------- the normal EM for P
@pytest.mark.parametrize("shape", [(3, 3, 2, 7), (2, 3, 2, 6), (4, 2, 1, 9), (1, 2, 2, 5), (8, 2, 1, 12)])
def test_em_matrices_are_the_dense_posterior_moments(shape):
    """W_i / (J N) of the normal EM from the transformed posterior equals the
    sum over n, j of the dense posterior second moments E[x_j x_j^H | y] =
    mu_j mu_j^H + Phi_j (the FCA oracle's Eqs. MMSE / postquadexp with
    S_j = P^{-H} Lambda_j P^{-1}) over v_j^new lambda_ji^new."""
    from oracle import fca
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=101 + I)
    vn, ln = ffa.em_half(p.y, p.v0, p.lam0, p.P0)
    W = ffa.em_covariances(p.y, p.v0, p.lam0, p.P0, vn, ln)
    mu, Phi = fca.e_step(p.y, p.v0, fca.spatial_from_joint(p.P0, p.lam0), counter=OpCounter())
    C = mu[..., :, None] * mu[..., None, :].conj() + Phi
    ref = np.einsum("jfnab,jfn,fji->fiab", C, 1.0 / vn, 1.0 / ln) / (J * N)
    np.testing.assert_allclose(W, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


def test_em_m_step_for_p_ascends_and_the_em_step_does_not_decrease_loglik():
    """With the M-step for P run to its stationary point (Eq. FPI on the
    M-step's matrices, with the column rescaling of the fixed-point pins),
    the expected complete-data log-likelihood rises over P and the whole EM
    step does not decrease L2 (the EM guarantee)."""
    p = make_problem(3, 3, 3, 120, seed=111)
    vn, ln = ffa.em_half(p.y, p.v0, p.lam0, p.P0)
    W = ffa.em_covariances(p.y, p.v0, p.lam0, p.P0, vn, ln)

    def q(P):  # the P-dependent part of the expected complete-data log-likelihood / (J N)
        _, la = np.linalg.slogdet(P)
        return 2 * la - np.einsum("fai,fiab,fbi->f", P.conj(), W, P).real

    P = p.P0.copy()
    for _ in range(800):
        P = ffa.fixed_point_P(P, W, K=1, counter=OpCounter())
        d = np.einsum("fai,fiab,fbi->fi", P.conj(), W, P).real
        P = P / np.sqrt(d)[:, None, :]
    G = np.linalg.inv(P).conj().transpose(0, 2, 1) - np.einsum("fiab,fbi->fai", W, P)
    assert np.abs(G).max() < 1e-9
    assert np.all(q(P) >= q(p.P0) - 1e-12)
    assert ffa.loglik(p.y, vn, ln, P) >= ffa.loglik(p.y, p.v0, p.lam0, p.P0)


def test_em_iterations_rise():
    """K = 1 sweep per M-step (the hybrid's budget): monitored, L2 rises."""
    p = make_problem(3, 3, 4, 200, seed=121)
    _, _, _, tr = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 6, counter=OpCounter(), p_update="em")
    assert np.all(np.diff(tr) > 0), np.diff(tr)
