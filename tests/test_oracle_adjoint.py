"""Pins of the gradient oracle (oracle/adjoint.py) to things other than
itself: central finite differences of the two losses (themselves pinned to
the dense model density and to the Wiener identities in test_oracle_pins),
and points where a gradient vanishes in closed form.

A real loss L of complex P changes by dL = 2 Re sum conj(dL/dP^*) dP, so a
directional finite difference checks all three gradients at once.
"""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import fastfca_as as ffa
from paper_1805_09498_gb300.synth import make_problem


def _directional(loss, grads, args, rng, h=1e-6):
    """Central difference of loss along a random direction in (v, lam, P)
    against the gradients' prediction; relative steps keep v, lam > 0."""
    y, v, lam, P = args
    dv = v * rng.standard_normal(v.shape)
    dl = lam * rng.standard_normal(lam.shape)
    dP = rng.standard_normal(P.shape) + 1j * rng.standard_normal(P.shape)
    Lp = loss(y, v + h * dv, lam + h * dl, P + h * dP)
    Lm = loss(y, v - h * dv, lam - h * dl, P - h * dP)
    fd = (Lp - Lm) / (2 * h)
    gv, gl, gP = grads
    pred = np.sum(gv * dv) + np.sum(gl * dl) + 2.0 * np.real(np.sum(gP.conj() * dP))
    return fd, pred


SHAPES = [(1, 1, 2, 6), (2, 1, 3, 7), (2, 3, 2, 9), (3, 2, 2, 8), (3, 3, 3, 5), (4, 3, 2, 6), (4, 4, 2, 5), (8, 3, 2, 6)]


@pytest.mark.parametrize("shape", SHAPES)
def test_nll_gradient_matches_central_differences(shape):
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=70 + I + 5 * J)
    rng = np.random.default_rng(I * 10 + J)
    args = (p.y, p.v0, p.lam0, p.P0)
    g = adj.nll_grad(*args)
    for _ in range(3):
        fd, pred = _directional(adj.nll, g, args, rng)
        assert abs(fd - pred) <= 1e-7 * max(1.0, abs(pred)), (fd, pred)


@pytest.mark.parametrize("shape", SHAPES)
def test_wiener_se_gradient_matches_central_differences(shape):
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=90 + I + 5 * J, keep_images=True)
    rng = np.random.default_rng(I * 7 + J)
    se = lambda y, v, lam, P: adj.wiener_se(y, p.x, v, lam, P)  # noqa: E731
    args = (p.y, p.v0, p.lam0, p.P0)
    g = adj.wiener_se_grad(p.y, p.x, *args[1:])
    for _ in range(3):
        fd, pred = _directional(se, g, args, rng)
        assert abs(fd - pred) <= 1e-7 * max(1.0, abs(pred)), (fd, pred)


def test_each_gradient_block_separately():
    """Perturb v, lam and P one at a time (a dropped block or a wrong factor
    in one of them cannot be hidden by the others)."""
    p = make_problem(3, 2, 2, 7, seed=5, keep_images=True)
    rng = np.random.default_rng(0)
    for loss, grad in ((adj.nll, adj.nll_grad(p.y, p.v0, p.lam0, p.P0)),
                       (lambda y, v, l, P: adj.wiener_se(y, p.x, v, l, P),
                        adj.wiener_se_grad(p.y, p.x, p.v0, p.lam0, p.P0))):
        gv, gl, gP = grad
        h = 1e-6
        dv = p.v0 * rng.standard_normal(p.v0.shape)
        fd = (loss(p.y, p.v0 + h * dv, p.lam0, p.P0) - loss(p.y, p.v0 - h * dv, p.lam0, p.P0)) / (2 * h)
        assert abs(fd - np.sum(gv * dv)) <= 1e-7 * max(1, abs(fd))
        dl = p.lam0 * rng.standard_normal(p.lam0.shape)
        fd = (loss(p.y, p.v0, p.lam0 + h * dl, p.P0) - loss(p.y, p.v0, p.lam0 - h * dl, p.P0)) / (2 * h)
        assert abs(fd - np.sum(gl * dl)) <= 1e-7 * max(1, abs(fd))
        dP = 1j * rng.standard_normal(p.P0.shape)   # imaginary direction: pins the conjugation
        fd = (loss(p.y, p.v0, p.lam0, p.P0 + h * dP) - loss(p.y, p.v0, p.lam0, p.P0 - h * dP)) / (2 * h)
        assert abs(fd - 2 * np.real(np.sum(gP.conj() * dP))) <= 1e-7 * max(1, abs(fd))


def test_nll_gradient_is_minus_eq_partialP():
    """dNLL/dP^* is minus the L2 gradient of Eq. partialP (pinned separately)."""
    p = make_problem(3, 3, 4, 11, seed=8)
    _, _, gP = adj.nll_grad(p.y, p.v0, p.lam0, p.P0)
    np.testing.assert_allclose(gP, -ffa.grad_P_conj(p.y, p.v0, p.lam0, p.P0), rtol=1e-12, atol=1e-12)


def test_nll_stationary_points_in_closed_form():
    """I = J = 1: NLL = sum ln(v lam / |p|^2) + |p|^2 |y|^2 / (v lam) is
    stationary in v at v = |p y|^2 / lam and in p at |p|^2 = N / sum |y|^2 / (v lam)."""
    rng = np.random.default_rng(3)
    N = 6
    y = (rng.standard_normal((1, 1, N)) + 1j * rng.standard_normal((1, 1, N)))
    lam = np.array([[[1.7]]])
    P = np.array([[[0.8 * np.exp(0.4j)]]])
    v = (np.abs(P[0, 0, 0] * y) ** 2 / lam[0, 0, 0]).real.reshape(1, 1, N)
    gv, _, _ = adj.nll_grad(y, v, lam, P)
    np.testing.assert_allclose(gv, 0.0, atol=1e-12)
    v = rng.uniform(0.5, 2.0, (1, 1, N))
    r = N / np.sum(np.abs(y[0, 0]) ** 2 / (v[0, 0] * lam[0, 0, 0]))
    P = np.array([[[np.sqrt(r) * np.exp(1.1j)]]])
    _, _, gP = adj.nll_grad(y, v, lam, P)
    np.testing.assert_allclose(gP, 0.0, atol=1e-10)


def test_wiener_se_gradient_vanishes_at_zero_error():
    """With s equal to the Wiener estimate itself the loss is 0, its minimum,
    so every gradient is 0."""
    p = make_problem(3, 2, 3, 9, seed=12)
    s = ffa.wiener(p.y, p.v0, p.lam0, p.P0)
    assert adj.wiener_se(p.y, s, p.v0, p.lam0, p.P0) < 1e-25
    for g in adj.wiener_se_grad(p.y, s, p.v0, p.lam0, p.P0):
        assert np.max(np.abs(g)) < 1e-10
