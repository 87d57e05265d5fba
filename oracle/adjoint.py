"""FP64 CPU oracle of the FastFCA-AS gradients (the adjoint of Eq. L2 and of
the Wiener estimate of Eq. MMSE0).

TEST INFRASTRUCTURE ONLY. Only tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module; the library never does.
It shares no code with the CUDA path.

Two losses of the model parameters Psi = (v, Lambda, P) at fixed data:

  NLL(Psi) = -L2(Psi)                                  (Eq. L2)
  SE(Psi)  = sum_{j,n,f} |x^_j(n,f) - s_j(n,f)|^2      (x^_j of Eq. MMSE0 with
                                                         Eq. covmodelprop)

Gradients are returned as (dv [J,F,N], dlam [F,J,I], dPc [F,I,I]) with dPc
the conjugate Wirtinger derivative dLoss/dP^* (the convention of Eq.
partialP); for a real loss, dLoss = 2 Re sum conj(dPc) dP.

Derivations (per (n,f); y~ = P^H y, sigma_i = sum_j v_j lambda_ji, Q = P^{-H}):

NLL per point: I ln(pi) - ln|det P|^2 + sum_i (ln sigma_i + |y~_i|^2 / sigma_i).
  dNLL/dsigma_i = 1/sigma_i - |y~_i|^2 / sigma_i^2 =: t_i
  dNLL/dv_j = sum_i lambda_ji t_i;  dNLL/dlambda_ji = sum_n v_j t_i
  dNLL/dP^* = -N P^{-H} + sum_n y y^H P D^{-1}  (D = diag(sigma)), i.e. minus
  Eq. partialP; column i of the sum is sum_n y conj(y~_i) / sigma_i.

SE per point, with g_ji = v_j lambda_ji / sigma_i, x^_j = Q (g_j * y~),
e_j = x^_j - s_j and b_j = Q^H e_j = P^{-1} e_j:
  dSE/dg_ji = 2 Re(conj(b_ji) y~_i) =: G_ji
  dg_ji/dv_k = [j = k] lambda_ji / sigma_i - g_ji lambda_ki / sigma_i, so
  dSE/dv_k = sum_i lambda_ki / sigma_i (G_ki - h_i),  h_i = sum_j G_ji g_ji
  dSE/dlambda_ki = sum_n v_k / sigma_i (G_ki - h_i)
  x^_j = P^{-H} D_j P^H y (D_j = diag(g_j)) gives dx^_j = -P^{-H} dP^H x^_j
  + P^{-H} D_j dP^H y, hence dSE = 2 Re tr(A dP) with
  A = sum_j (D_j b_j y^H - b_j x^_j^H) and dSE/dP^* = A^H
    = sum_j (y (g_j * b_j)^H - x^_j b_j^H), summed over n.
"""
from __future__ import annotations

import numpy as np

from .fastfca_as import basis_transform, loglik, model_variances, wiener


def nll(y, v, lam, P):
    """NLL = -L2 (Eq. L2)."""
    return -loglik(y, v, lam, P)


def nll_grad(y, v, lam, P):
    """(dv, dlam, dPc) of NLL; see the module docstring."""
    N = y.shape[2]
    yt = basis_transform(y, P)                   # [I, F, N]
    sigma = model_variances(v, lam)              # [I, F, N]
    t = 1.0 / sigma - np.abs(yt) ** 2 / sigma ** 2
    dv = np.einsum("fji,ifn->jfn", lam, t)
    dlam = np.einsum("jfn,ifn->fji", v, t)
    PinvH = np.linalg.inv(P).conj().transpose(0, 2, 1)
    S = np.einsum("afn,ifn->fai", y, yt.conj() / sigma)
    return dv, dlam, -N * PinvH + S


def wiener_se(y, s, v, lam, P):
    """SE = sum |x^_j - s_j|^2 over j, mics, n, f; s [J, I, F, N] complex."""
    return float(np.sum(np.abs(wiener(y, v, lam, P) - s) ** 2))


def wiener_se_grad(y, s, v, lam, P):
    """(dv, dlam, dPc) of SE; see the module docstring."""
    yt = basis_transform(y, P)                              # [I, F, N]
    sigma = model_variances(v, lam)                         # [I, F, N]
    g = v[:, None] * lam.transpose(1, 2, 0)[:, :, :, None] / sigma[None]   # [J, I, F, N]
    Q = np.linalg.inv(P).conj().transpose(0, 2, 1)          # P^{-H}, [F, I, I]
    xh = np.einsum("fab,jbfn->jafn", Q, g * yt[None])       # x^_j
    e = xh - s
    b = np.einsum("fba,jbfn->jafn", Q.conj(), e)            # Q^H e_j
    G = 2.0 * np.real(b.conj() * yt[None])                  # [J, I, F, N]
    h = np.sum(G * g, axis=0)                               # [I, F, N]
    w = (G - h[None]) / sigma[None]                         # [J, I, F, N]
    dv = np.einsum("fji,jifn->jfn", lam, w)
    dlam = np.einsum("jfn,jifn->fji", v, w)
    dPc = (np.einsum("afn,jcfn->fac", y, (g * b).conj())
           - np.einsum("jafn,jcfn->fac", xh, b.conj()))
    return dv, dlam, dPc
