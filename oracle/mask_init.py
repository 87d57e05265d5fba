"""FP64 CPU oracle of the mask-based initialisation of FastFCA-AS (Sec. 5).

TEST INFRASTRUCTURE ONLY. Only tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module; the library never does.
It shares no code with the CUDA path.

Sec. 5 initialises the parameters by mask-based covariance matrix
estimation, with time-frequency masks from a cited method, and states no
further step.  The masks are the caller's here (the masking method is not
part of this build); the readings of the rest, listed with their reasons in
the design notes:

1. Masked spatial covariance of source j:
       R_j(f) = sum_n m_j(n,f) y(n,f) y(n,f)^H / sum_n m_j(n,f).
2. (P, Lambda) jointly diagonalise the R_j: P starts as the generalized
   eigenvectors of the pencil (R_1, R_y), R_y = sum_j R_j (the GEVD that
   yields P and Lambda for two sources, Sec. 4.1; exact whenever the R_j are
   jointly diagonalisable, any J):  R_y = L L^H,  W = L^{-1} R_1 L^{-H} =
   U diag(w) U^H (ascending w),  P = L^{-H} U, each column turned in phase so
   that its entry of largest magnitude is real and positive.  Then `sweeps`
   alternations that raise
       sum_j [ ln|det P|^2 - sum_i ( ln lambda_ji + p_i^H R_j p_i / lambda_ji ) ],
   the log-likelihood of Eq. L2 with R_j standing in for the covariance of
   the data of source j alone:
       lambda_ji <- p_i^H R_j p_i                         (its exact maximiser)
       V_i = (1/J) sum_j R_j / lambda_ji,  p_i <- V_i^{-1} [P^{-H}]_i   (Eq. FPI)
   (an exact joint diagonaliser is a fixed point of this map); finally
   lambda_ji = p_i^H R_j p_i of the final P.
3. Source powers: the maximum-likelihood v_j of the masked image
   m_j(n,f) y(n,f) under S_j = P^{-H} Lambda_j P^{-1} is
   (1/I) m_j^2 y^H S_j^{-1} y; with the mask itself in place of its square
   (the same for binary masks) and a floor delta that keeps every v_j > 0 (a
   v_j of 0 stays 0 under Eq. updatev):
       v_j(n,f) = max(m_j(n,f), delta) (1/I) sum_i |y~_i|^2 / lambda_ji,  y~ = P^H y.

Layouts as oracle.fastfca_as; masks m [J, F, N] real.
"""
from __future__ import annotations

import numpy as np

from .fastfca_as import OpCounter, basis_transform, fixed_point_P

DELTA = 1e-3    # floor of the mask in the source powers
SWEEPS = 10     # alternations of the joint diagonalisation after the GEVD start


def masked_covariances(y, m):
    """R_j(f) = sum_n m_j y y^H / sum_n m_j (step 1).  Returns [F, J, I, I]."""
    num = np.einsum("jfn,afn,bfn->fjab", m, y, y.conj())
    return num / np.sum(m, axis=2).T[:, :, None, None]


def diag_powers(R, P):
    """lambda_ji = p_i^H R_j p_i (real).  Returns [F, J, I]."""
    return np.einsum("fai,fjab,fbi->fji", P.conj(), R, P).real


def gevd_start(R):
    """The generalized eigenvectors of (R_1, R_y) (step 2's start): [F, I, I]."""
    L = np.linalg.cholesky(R.sum(axis=1))                     # R_y = L L^H
    Li = np.linalg.inv(L)
    W = Li @ R[:, 0] @ Li.conj().transpose(0, 2, 1)
    _, U = np.linalg.eigh(W)                                  # ascending eigenvalues
    P = Li.conj().transpose(0, 2, 1) @ U                      # L^{-H} U
    k = np.argmax(np.abs(P), axis=1)                          # [F, I]: row of the largest entry per column
    big = np.take_along_axis(P, k[:, None, :], axis=1)[:, 0]  # [F, I]
    return P * (np.abs(big) / big)[:, None, :]


def joint_diagonaliser(R, sweeps=SWEEPS):
    """Step 2: (P [F, I, I], lambda [F, J, I]) from the covariances R [F, J, I, I]."""
    J = R.shape[1]
    P = gevd_start(R)
    cnt = OpCounter()
    for _ in range(sweeps):
        lam = diag_powers(R, P)
        V = np.einsum("fjab,fji->fiab", R, 1.0 / lam) / J
        P = fixed_point_P(P, V, 1, cnt)
    return P, diag_powers(R, P)


def initial_v(y, m, P, lam, delta=DELTA):
    """Step 3: v_j = max(m_j, delta) (1/I) sum_i |y~_i|^2 / lambda_ji.  [J, F, N]."""
    I = y.shape[0]
    e2 = np.abs(basis_transform(y, P)) ** 2                   # [I, F, N]
    q = np.einsum("ifn,fji->jfn", e2, 1.0 / lam) / I
    return np.maximum(m, delta) * q


def mask_init(y, m, sweeps=SWEEPS, delta=DELTA):
    """The three steps: returns (v [J, F, N], lam [F, J, I], P [F, I, I])."""
    R = masked_covariances(y, m)
    P, lam = joint_diagonaliser(R, sweeps)
    return initial_v(y, m, P, lam, delta), lam, P


def ajd_criterion(R, P, lam):
    """The maximised criterion of step 2, per frequency [F]."""
    _, logabsdet = np.linalg.slogdet(P)
    quad = np.einsum("fai,fjab,fbi->fji", P.conj(), R, P).real / lam
    return R.shape[1] * 2.0 * logabsdet - np.sum(np.log(lam) + quad, axis=(1, 2))
