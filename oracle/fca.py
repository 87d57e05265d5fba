"""FP64 CPU oracle of conventional FCA (full-rank spatial covariance analysis,
Sec. 3 of Ito & Nakatani, arXiv 1805.09498; the EM of Duong et al.).

TEST INFRASTRUCTURE ONLY. Only tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module; the library never does.
It shares no code with the CUDA path.

Dense I x I algebra at every time-frequency point, exactly as Eqs. MMSE,
postquadexp, vupdate and Supdate state it.  Layouts:
    y [I, F, N] complex, v [J, F, N] real,
    S [F, J, I, I] complex Hermitian positive definite, S[f, j] = S_j(f).
Reading taken where the paper is silent: the M-step updates v (with the
current S_j^{-1}) before S_j (with the new v), the order Eqs. vupdate and
Supdate are listed in.
"""
from __future__ import annotations

import numpy as np

from .fastfca_as import COUNTER, LN_PI


def _covariances(v, S):
    """R_j(n,f) = v_j(n,f) S_j(f) (Eq. fullrank).  Returns [J, F, N, I, I]."""
    return v[:, :, :, None, None] * S.transpose(1, 0, 2, 3)[:, :, None, :, :]


def e_step(y, v, S, counter=COUNTER):
    """Eqs. MMSE and postquadexp:
        mu_j  = R_j (sum_k R_k)^{-1} y
        Phi_j = R_j - R_j (sum_k R_k)^{-1} R_j
    Returns mu [J, F, N, I] and Phi [J, F, N, I, I]."""
    J, F, N = v.shape
    Rj = _covariances(v, S)
    Rinv = np.linalg.inv(Rj.sum(axis=0))                      # N F inversions
    counter.inversions += F * N
    RjRinv = Rj @ Rinv[None]                                  # J N F products
    counter.multiplications += J * F * N
    yv = y.transpose(1, 2, 0)                                 # [F, N, I]
    mu = np.einsum("jfnab,fnb->jfna", RjRinv, yv)
    Phi = Rj - RjRinv @ Rj                                    # J N F products
    counter.multiplications += J * F * N
    return mu, Phi


def m_step(mu, Phi, S, counter=COUNTER):
    """Eq. vupdate then Eq. Supdate:
        v_j <- (1/I) tr(S_j^{-1} (mu_j mu_j^H + Phi_j))      (current S_j)
        S_j <- (1/N) sum_n (mu_j mu_j^H + Phi_j) / v_j        (new v_j)
    Returns (v [J, F, N], S [F, J, I, I])."""
    J, F, N, I = mu.shape
    C = mu[..., :, None] * mu[..., None, :].conj() + Phi      # mu mu^H + Phi
    Sinv = np.linalg.inv(S)                                   # J F inversions
    counter.inversions += J * F
    v = np.einsum("fjab,jfnba->jfn", Sinv, C).real / I
    S_new = np.einsum("jfnab->fjab", C / v[..., None, None]) / N
    return v, S_new


def loglik_terms(y, v, S):
    """Per-(n,f) ln N(y; 0, sum_j v_j S_j) of Eq. L1, the circular complex
    Gaussian density: -I ln(pi) - ln det R - y^H R^{-1} y.  Returns [F, N]."""
    I = y.shape[0]
    R = _covariances(v, S).sum(axis=0)
    yv = y.transpose(1, 2, 0)
    _, logdet = np.linalg.slogdet(R)
    quad = np.einsum("fna,fnab,fnb->fn", yv.conj(), np.linalg.inv(R), yv).real
    return -I * LN_PI - logdet - quad


def loglik(y, v, S):
    """Eq. L1: sum over (n, f) of the per-point log densities."""
    return float(np.sum(loglik_terms(y, v, S)))


def iteration(y, v, S, counter=COUNTER):
    """One EM iteration of FCA (Sec. 3.3): E-step then M-step."""
    mu, Phi = e_step(y, v, S, counter)
    return m_step(mu, Phi, S, counter)


def iterate(y, v, S, iters, counter=COUNTER):
    """Run `iters` EM iterations; trace[t] = L1 entering iteration t, plus the final L1."""
    trace = []
    for _ in range(iters):
        trace.append(loglik(y, v, S))
        v, S = iteration(y, v, S, counter)
    trace.append(loglik(y, v, S))
    return v, S, np.array(trace)


def wiener(y, v, S):
    """Eq. MMSE0: x^_j = R_j (sum_k R_k)^{-1} y.  Returns [J, I, F, N]."""
    mu, _ = e_step(y, v, S, counter=_NullCounter())
    return mu.transpose(0, 3, 1, 2)


def spatial_from_joint(P, lam):
    """Eq. diagconst: S_j(f) = P(f)^{-H} Lambda_j(f) P(f)^{-1}.  Returns [F, J, I, I]."""
    Pinv = np.linalg.inv(P)
    PinvH = Pinv.conj().transpose(0, 2, 1)
    return np.einsum("fab,fjb,fbc->fjac", PinvH, lam, Pinv)


class _NullCounter:
    inversions = 0
    multiplications = 0
