"""Planted mistakes in the FP64 oracle, one at a time and on the CPU only,
each of which some pin must catch.

The pins (dense covariance algebra, the Q-function, the Kronecker form of
Eq. FPI, finite differences, the Wiener identities, the closed forms, the
scale gauge and the FCA correspondence) do not share the oracle's code, so a
plausible slip in any step of it (a transposed or unconjugated operand, a
dropped term, a wrong normalisation, the wrong (v, Lambda) in an update)
has to fail at least one of them.  This guards the pins themselves: a pin
that a mistake slips past is no pin.
"""
import numpy as np
import pytest

from oracle import fastfca_as as ffa
from oracle import fca

import test_oracle_p_updates as pu
import test_oracle_pins as pins

LN_PI = np.log(np.pi)


def _bt_no_conj(y, P):  # P^T y instead of P^H y
    return np.einsum("fai,afn->ifn", P, y)


def _sigma_wrong_source(v, lam):  # lambda of the wrong source
    return np.einsum("jfn,fji->ifn", v, lam[:, ::-1, :])


def _estep_no_correction(y, v, lam, P):  # Phi~ without its second term
    yt = ffa.basis_transform(y, P)
    sigma = ffa.model_variances(v, lam)
    vl = v[:, None] * lam.transpose(1, 2, 0)[:, :, :, None]
    return vl / sigma[None] * yt[None], vl


def _estep_conj_mean(y, v, lam, P):  # conj(y~) in the posterior mean
    yt = ffa.basis_transform(y, P)
    sigma = ffa.model_variances(v, lam)
    vl = v[:, None] * lam.transpose(1, 2, 0)[:, :, :, None]
    return vl / sigma[None] * yt.conj()[None], vl - vl * vl / sigma[None]


def _v_over_J(mu, phi, lam):  # 1/J instead of 1/I
    q = np.abs(mu) ** 2 + phi
    return np.einsum("jifn,fji->jfn", q, 1.0 / lam) / mu.shape[0]


def _v_times_lambda(mu, phi, lam):  # Lambda instead of Lambda^{-1}
    q = np.abs(mu) ** 2 + phi
    return np.einsum("jifn,fji->jfn", q, lam) / mu.shape[1]


def _lambda_over_n_minus_1(mu, phi, v):
    q = np.abs(mu) ** 2 + phi
    return np.einsum("jifn->fji", q / v[:, None]) / (mu.shape[3] - 1)


def _cov_transposed(y, v, lam):  # conj(y) y^T instead of y y^H
    sigma = ffa.model_variances(v, lam)
    return np.einsum("afn,bfn,ifn->fiab", y.conj(), y, 1.0 / sigma) / y.shape[2]


def _fpi_no_conj(P, V, K=1, counter=ffa.COUNTER):  # P^{-T} instead of P^{-H}
    for _ in range(K):
        Q = np.linalg.inv(P).transpose(0, 2, 1)
        P = np.stack([np.linalg.solve(V[:, i], Q[:, :, i][..., None])[..., 0] for i in range(P.shape[1])], axis=2)
    return P


def _fpi_v_transposed(P, V, K=1, counter=ffa.COUNTER):  # V_i^T instead of V_i
    for _ in range(K):
        Q = np.linalg.inv(P).conj().transpose(0, 2, 1)
        P = np.stack([np.linalg.solve(V[:, i].transpose(0, 2, 1), Q[:, :, i][..., None])[..., 0]
                      for i in range(P.shape[1])], axis=2)
    return P


def _ll_no_pi(y, v, lam, P):  # the -I ln(pi) constant dropped
    yt = ffa.basis_transform(y, P)
    sigma = ffa.model_variances(v, lam)
    _, la = np.linalg.slogdet(P)
    return 2.0 * la[:, None] - np.sum(np.log(sigma) + np.abs(yt) ** 2 / sigma, axis=0)


def _ll_det_once(y, v, lam, P):  # ln|det P| instead of ln|det P|^2
    yt = ffa.basis_transform(y, P)
    sigma = ffa.model_variances(v, lam)
    _, la = np.linalg.slogdet(P)
    return -y.shape[0] * LN_PI + la[:, None] - np.sum(np.log(sigma) + np.abs(yt) ** 2 / sigma, axis=0)


def _wiener_p_inverse(y, v, lam, P):  # P^{-1} instead of P^{-H}
    mu, _ = ffa.e_step(y, v, lam, P)
    return np.einsum("fab,jbfn->jafn", np.linalg.inv(P), mu)


def _em_lambda_with_old_v(y, v, lam, P):  # Eq. Lambdaupdate with the old v
    mu, phi = ffa.e_step(y, v, lam, P)
    return ffa.m_step_v(mu, phi, lam), ffa.m_step_lambda(mu, phi, v)


def _grad_no_conj(P, V, mu, K=1, counter=ffa.COUNTER):  # P^{-T} in the gradient step
    for _ in range(K):
        P = P + mu * (np.linalg.inv(P).transpose(0, 2, 1) - np.einsum("fiab,fbi->fai", V, P))
    return P


def _natgrad_no_h(P, V, mu, K=1):  # (I - C) instead of (I - C)^H
    eye = np.eye(P.shape[1])[None]
    for _ in range(K):
        C = np.einsum("fai,fiab,fbk->fik", P.conj(), V, P)
        P = P + mu * (P @ (eye - C))
    return P


def _fca_phi_plus(y, v, S, counter=ffa.COUNTER):  # Phi_j = R_j + R_j R^{-1} R_j
    Rj = v[:, :, :, None, None] * S.transpose(1, 0, 2, 3)[:, :, None, :, :]
    RjRinv = Rj @ np.linalg.inv(Rj.sum(axis=0))[None]
    mu = np.einsum("jfnab,fnb->jfna", RjRinv, y.transpose(1, 2, 0))
    return mu, Rj + RjRinv @ Rj


def _fca_v_without_inverse(mu, Phi, S, counter=ffa.COUNTER):  # tr(S_j C) instead of tr(S_j^{-1} C)
    J, F, N, I = mu.shape
    C = mu[..., :, None] * mu[..., None, :].conj() + Phi
    v = np.einsum("fjab,jfnba->jfn", S, C).real / I
    return v, np.einsum("jfnab->fjab", C / v[..., None, None]) / N


def _fca_outer_transposed(mu, Phi, S, counter=ffa.COUNTER):  # mu^* mu^T instead of mu mu^H
    J, F, N, I = mu.shape
    C = mu[..., :, None].conj() * mu[..., None, :] + Phi
    v = np.einsum("fjab,jfnba->jfn", np.linalg.inv(S), C).real / I
    return v, np.einsum("jfnab->fjab", C / v[..., None, None]) / N


def _newton_no_logdet_curvature(P, V, mu=1.0, K=1, counter=ffa.COUNTER):  # Hessian without ln|det P|^2
    F, I, _ = P.shape
    E = ffa._real_basis(I)
    for _ in range(K):
        G = np.linalg.inv(P).conj().transpose(0, 2, 1) - np.einsum("fiab,fbi->fai", V, P)
        g = 2.0 * np.real(np.einsum("fai,kai->fk", G.conj(), E))
        H = -2.0 * np.real(np.einsum("kai,fiab,lbi->fkl", E.conj(), V, E))
        P = P + mu * np.einsum("fk,kai->fai", np.linalg.solve(H, -g[..., None])[..., 0], E)
    return P


FCA_MUTANTS = [("e_step", _fca_phi_plus), ("m_step", _fca_v_without_inverse), ("m_step", _fca_outer_transposed)]

def _em_no_phi(y, v, lam, P, v_new, lam_new):  # the posterior covariance term dropped
    J, I, N = v.shape[0], y.shape[0], y.shape[2]
    mu, _ = ffa.e_step(y, v, lam, P)
    T = np.einsum("jafn,jbfn,jfn->fjab", mu, mu.conj(), 1.0 / v_new)
    Om = np.einsum("fjab,fji->fiab", T, 1.0 / lam_new)
    PinvH = np.linalg.inv(P).conj().transpose(0, 2, 1)
    return np.einsum("fac,ficd,fbd->fiab", PinvH, Om, PinvH.conj()) / (J * N)


MUTANTS = [
    ("basis_transform", _bt_no_conj), ("model_variances", _sigma_wrong_source),
    ("e_step", _estep_no_correction), ("e_step", _estep_conj_mean),
    ("m_step_v", _v_over_J), ("m_step_v", _v_times_lambda), ("m_step_lambda", _lambda_over_n_minus_1),
    ("weighted_covariances", _cov_transposed), ("fixed_point_P", _fpi_no_conj),
    ("fixed_point_P", _fpi_v_transposed), ("loglik_terms", _ll_no_pi), ("loglik_terms", _ll_det_once),
    ("wiener", _wiener_p_inverse), ("em_half", _em_lambda_with_old_v),
    ("gradient_P", _grad_no_conj), ("natural_gradient_P", _natgrad_no_h),
    ("newton_P", _newton_no_logdet_curvature), ("em_covariances", _em_no_phi),
]

# every pin on one of its cases (two where I = J would hide a mix-up of I and J)
PINS = [
    (pins.test_loglik_equals_dense_density, dict(shape=pins.SHAPES[0])),
    (pins.test_estep_equals_dense_posterior, dict(shape=pins.SHAPES[0])),
    (pins.test_mstep_maximises_q_function, dict(shape=(3, 3, 2, 5))),
    (pins.test_mstep_maximises_q_function, dict(shape=(2, 3, 2, 4))),  # I != J
    (pins.test_wiener_identities, dict(shape=pins.SHAPES[0])),
    (pins.test_fixed_point_equals_kronecker_form, dict(shape=pins.SHAPES[0])),
    (pins.test_gradient_matches_finite_differences, dict(shape=(3, 3, 1, 6))),
    (pins.test_fixed_point_scalar_closed_form, {}),
    (pins.test_em_half_does_not_decrease_loglik, dict(seed=0)),
    (pins.test_fca_and_fastfca_agree_from_joint_state, dict(shape=(3, 3, 2, 9))),
    (pins.test_scale_gauge_equivariance, {}),
    (pu.test_gradient_step_is_the_scaled_wirtinger_gradient, dict(shape=pu.SHAPES[0])),
    (pu.test_natural_gradient_step_slope, dict(shape=pu.SHAPES[0])),
    (pu.test_natural_gradient_is_equivariant, {}),
    (pu.test_newton_step_zeroes_the_linearised_gradient, dict(shape=(3, 3, 2, 60))),
    (pu.test_em_matrices_are_the_dense_posterior_moments, dict(shape=(3, 3, 2, 7))),
]


@pytest.mark.parametrize("name,mutant", MUTANTS, ids=[m.__name__.strip("_") for _, m in MUTANTS])
def test_a_pin_catches_the_planted_mistake(monkeypatch, name, mutant):
    monkeypatch.setattr(ffa, name, mutant)
    for pin, kw in PINS:
        try:
            pin(**kw)
        except AssertionError:
            return  # caught
    pytest.fail(f"no pin caught {mutant.__name__} in {name}")


FCA_PINS = [
    (pins.test_fca_loglik_monotone, dict(seed=0)),
    (pins.test_fca_dense_loglik, dict(shape=(3, 3, 2, 6))),
    (pins.test_fca_and_fastfca_agree_from_joint_state, dict(shape=(3, 3, 2, 9))),
]


@pytest.mark.parametrize("name,mutant", FCA_MUTANTS, ids=[m.__name__.strip("_") for _, m in FCA_MUTANTS])
def test_a_pin_catches_the_planted_fca_mistake(monkeypatch, name, mutant):
    monkeypatch.setattr(fca, name, mutant)
    for pin, kw in FCA_PINS:
        try:
            pin(**kw)
        except AssertionError:
            return
    pytest.fail(f"no pin caught {mutant.__name__} in fca.{name}")


def test_the_pins_pass_on_the_oracle():
    for pin, kw in PINS + FCA_PINS:
        pin(**kw)


# ---------------------------------------------------- the mask-based initialisation
from oracle import mask_init as mi  # noqa: E402

import test_oracle_mask_init as mpins  # noqa: E402


def _mcov_over_n(y, m):  # divided by the frame count instead of the mask's sum
    return np.einsum("jfn,afn,bfn->fjab", m, y, y.conj()) / y.shape[2]


def _mcov_transposed(y, m):  # conj(y) y^T instead of y y^H
    num = np.einsum("jfn,afn,bfn->fjab", m, y.conj(), y)
    return num / np.sum(m, axis=2).T[:, :, None, None]


def _gevd_wrong_side(R):  # L^{-H} R_1 L^{-1} instead of L^{-1} R_1 L^{-H}, no phase rule
    L = np.linalg.cholesky(R.sum(axis=1))
    Li = np.linalg.inv(L)
    W = Li.conj().transpose(0, 2, 1) @ R[:, 0] @ Li
    _, U = np.linalg.eigh(W)
    return Li.conj().transpose(0, 2, 1) @ U


def _powers_no_conj(R, P):  # p_i^T R_j p_i
    return np.einsum("fai,fjab,fbi->fji", P, R, P).real


def _v_mask_squared(y, m, P, lam, delta=mi.DELTA):  # m^2 and no floor
    I = y.shape[0]
    e2 = np.abs(ffa.basis_transform(y, P)) ** 2
    return m ** 2 * np.einsum("ifn,fji->jfn", e2, 1.0 / lam) / I


def _ajd_times_lambda(R, sweeps=mi.SWEEPS):  # V_i = sum_j R_j lambda_ji / J
    J = R.shape[1]
    P = mi.gevd_start(R)
    for _ in range(sweeps):
        lam = mi.diag_powers(R, P)
        P = ffa.fixed_point_P(P, np.einsum("fjab,fji->fiab", R, lam) / J, 1, ffa.OpCounter())
    return P, mi.diag_powers(R, P)


MASK_MUTANTS = [("masked_covariances", _mcov_over_n), ("masked_covariances", _mcov_transposed),
                ("gevd_start", _gevd_wrong_side), ("diag_powers", _powers_no_conj),
                ("initial_v", _v_mask_squared), ("joint_diagonaliser", _ajd_times_lambda)]
MASK_PINS = [(mpins.test_masked_covariance_is_the_weighted_second_moment, {}),
             (mpins.test_two_sources_are_diagonalised_exactly, {}),
             (mpins.test_jointly_diagonalisable_sources_are_recovered, {}),
             (mpins.test_an_exact_joint_diagonaliser_is_a_fixed_point, {}),
             (mpins.test_sweeps_raise_the_criterion, {}),
             (mpins.test_initial_v_is_the_masked_quadratic_form, {})]


@pytest.mark.parametrize("name,mutant", MASK_MUTANTS, ids=[m.__name__.strip("_") for _, m in MASK_MUTANTS])
def test_a_pin_catches_the_planted_mask_init_mistake(monkeypatch, name, mutant):
    monkeypatch.setattr(mi, name, mutant)
    for pin, kw in MASK_PINS:
        try:
            pin(**kw)
        except (AssertionError, np.linalg.LinAlgError):
            return
    pytest.fail(f"no pin caught {mutant.__name__} in mask_init.{name}")


def test_the_mask_init_pins_pass_on_the_oracle():
    for pin, kw in MASK_PINS:
        pin(**kw)
