"""FP64 CPU oracle of FastFCA-AS (Ito & Nakatani, arXiv 1805.09498, Sec. 4).

TEST INFRASTRUCTURE ONLY. Only tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module; the library never does.
It shares no code with the CUDA path.

Plain NumPy, float64 / complex128, vectorised over (n, f) with no blocking,
fusion or reordering beyond what each equation states. Every function names
the equation it follows.

Layouts (mic-planar, as in the synthetic generator):
    y   [I, F, N] complex   mixture y(n,f)                 (Sec. 2)
    v   [J, F, N] real      source power spectra v_j(n,f)  (Eq. fullrank)
    lam [F, J, I] real      lam[f, j, i] = [Lambda_j(f)]_ii (Eq. diagconst)
    P   [F, I, I] complex   P[f, a, i] = [P(f)]_{a i}; column i is p_i

Readings taken where the paper is silent (listed with reasons in the design
notes): the M-step updates v first (with the current Lambda) and then
Lambda (with the new v); the K fixed-point sweeps update all columns of P
simultaneously from P^{-H} of the previous sweep; the log-likelihood keeps
the -I ln(pi) constant of the circular complex Gaussian density.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

LN_PI = np.log(np.pi)


@dataclass
class OpCounter:
    """Counts the matrix inversions / multiplications performed (Sec. 3.4, 4.5)."""
    inversions: int = 0
    multiplications: int = 0

    def reset(self):
        self.inversions = 0
        self.multiplications = 0


COUNTER = OpCounter()


# ---------------------------------------------------------------- E-step ----
def basis_transform(y, P):
    """y~(n,f) = P(f)^H y(n,f): the transformed observation in Eq. mutilde0."""
    return np.einsum("fai,afn->ifn", P.conj(), y)


def model_variances(v, lam):
    """sigma_i(n,f) = sum_j v_j(n,f) [Lambda_j(f)]_ii: the diagonal matrix
    sum_k v_k Lambda_k inverted in Eqs. mutilde0 / Phitilde0 and in Eq. FPI."""
    return np.einsum("jfn,fji->ifn", v, lam)


def e_step(y, v, lam, P):
    """Posterior mean and covariance in the transformed basis.

    Eq. mutilde0: mu~_j = v_j Lambda_j (sum_k v_k Lambda_k)^{-1} y~
    Eq. Phitilde0: Phi~_j = v_j Lambda_j - v_j Lambda_j (sum_k v_k Lambda_k)^{-1} v_j Lambda_j
    All matrices are diagonal, so both are entrywise.  Returns
    mu [J, I, F, N] complex and phi [J, I, F, N] real (the diagonal of Phi~_j).
    """
    yt = basis_transform(y, P)
    sigma = model_variances(v, lam)
    vl = v[:, None, :, :] * lam.transpose(1, 2, 0)[:, :, :, None]   # v_j [Lambda_j]_ii
    mu = vl / sigma[None] * yt[None]
    phi = vl - vl * vl / sigma[None]
    return mu, phi


# ---------------------------------------------------------------- M-step ----
def m_step_v(mu, phi, lam):
    """Eq. updatev: v_j <- (1/I) tr(Lambda_j^{-1} (diag(|mu~_j|^2) + Phi~_j))."""
    I = mu.shape[1]
    q = np.abs(mu) ** 2 + phi
    return np.einsum("jifn,fji->jfn", q, 1.0 / lam) / I


def m_step_lambda(mu, phi, v):
    """Eq. Lambdaupdate: Lambda_j <- (1/N) sum_n (diag(|mu~_j|^2) + Phi~_j) / v_j."""
    N = mu.shape[3]
    q = np.abs(mu) ** 2 + phi
    return np.einsum("jifn->fji", q / v[:, None, :, :]) / N


# ------------------------------------------------------ fixed point for P ----
def weighted_covariances(y, v, lam):
    """V_i(f) = (1/N) sum_n y(n,f) y(n,f)^H / sigma_i(n,f), the matrix inverted
    in Eq. FPI.  Returns V [F, I(i), I, I]."""
    N = y.shape[2]
    sigma = model_variances(v, lam)
    return np.einsum("afn,bfn,ifn->fiab", y, y.conj(), 1.0 / sigma) / N


def fixed_point_P(P, V, K=1, counter=COUNTER):
    """Eq. FPI, iterated K times: p_i <- V_i^{-1} [P^{-H}]_i for every column i.

    Each sweep computes P^{-H} once from the previous sweep's P and updates
    all columns from it (one fixed-point map, Eq. vecP), which is I+1 matrix
    inversions per frequency per sweep (Sec. 4.5).
    """
    F, I, _ = P.shape
    P = P.copy()
    for _ in range(K):
        PinvH = np.linalg.inv(P).conj().transpose(0, 2, 1)
        counter.inversions += F
        Pn = np.empty_like(P)
        for i in range(I):
            Pn[:, :, i] = np.linalg.solve(V[:, i], PinvH[:, :, i][..., None])[..., 0]
            counter.inversions += F
        P = Pn
    return P


def grad_P_conj(y, v, lam, P):
    """Eq. partialP: dL2/dP(f)^* = N P^{-H} - sum_n y y^H P D^{-1},
    D = sum_j v_j Lambda_j.  Column i of the sum is N V_i p_i."""
    N = y.shape[2]
    V = weighted_covariances(y, v, lam)
    PinvH = np.linalg.inv(P).conj().transpose(0, 2, 1)
    VP = np.einsum("fiab,fbi->fai", V, P)
    return N * (PinvH - VP)


# ------------------------------------ alternative updates of P (Sec. 4.6) ----
# Sec. 4.6 names the gradient and natural gradient methods as replacements of
# the fixed-point iteration without stating them.  Readings: both ascend L2
# (Eq. L2) with the V_i of Eq. FPI held fixed (sigma from the new v and
# Lambda, as for the fixed point), take K steps of a caller-chosen size mu
# per iteration, and scale Eq. partialP by 1/N so that mu does not depend on
# the number of frames.
def gradient_P(P, V, mu, K=1, counter=COUNTER):
    """K steps of gradient ascent on L2 along Eq. partialP:
    P <- P + mu (P^{-H} - [V_1 p_1, ..., V_I p_I]) = P + (mu / N) dL2/dP^*.
    One matrix inversion (P^{-H}) per frequency per step."""
    F = P.shape[0]
    P = P.copy()
    for _ in range(K):
        PinvH = np.linalg.inv(P).conj().transpose(0, 2, 1)
        counter.inversions += F
        VP = np.einsum("fiab,fbi->fai", V, P)     # column i: V_i p_i
        P = P + mu * (PinvH - VP)
    return P


def natural_gradient_P(P, V, mu, K=1):
    """K steps of the natural (relative) gradient method.  With the
    demixing matrix W = P^H (y~ = W y, Eq. mutilde0) and
    C = (1/N) sum_n D^{-1} y~ y~^H, i.e. C_ik = p_i^H V_i p_k, the step is
    W <- W + mu (I - C) W, so P <- P + mu P (I - C)^H.  It equals
    P + (mu / N) P P^H dL2/dP^* and needs no matrix inversion."""
    F, I, _ = P.shape
    P = P.copy()
    eye = np.eye(I)[None]
    for _ in range(K):
        C = np.einsum("fai,fiab,fbk->fik", P.conj(), V, P)
        P = P + mu * (P @ (eye - C).conj().transpose(0, 2, 1))
    return P


def em_covariances(y, v, lam, P, v_new, lam_new):
    """The matrices of the M-step for P in the normal EM algorithm (the other
    alternative named in Sec. 4.6).  Reading: the complete data are the
    source images x_j of Eq. fullrank, x_j ~ CN(0, v_j P^{-H} Lambda_j P^{-1})
    (Eq. diagconst); the expected complete-data log-likelihood is, over P,
        J N ln|det P|^2 - sum_i p_i^H W_i p_i,
        W_i = sum_{n,j} E[x_j x_j^H | y] / (v_j lambda_ji)
    with the posterior of the current (v, Lambda, P) and the new v, Lambda of
    Eqs. updatev and Lambdaupdate (whose updates are the same in the normal
    EM).  E[x_j x_j^H | y] = P^{-H} (mu~_j mu~_j^H + diag(phi~_j)) P^{-1}
    with mu~, phi~ of Eqs. mutilde0 / Phitilde0.  Setting the derivative in
    P^* to zero gives Eq. FPI's form with V_i replaced by W_i / (J N), which
    is returned, [F, I(i), I, I]."""
    J, I, F, N = v.shape[0], y.shape[0], y.shape[1], y.shape[2]
    mu, phi = e_step(y, v, lam, P)                                     # [J, I, F, N]
    T = np.einsum("jafn,jbfn,jfn->fjab", mu, mu.conj(), 1.0 / v_new)  # sum_n mu~ mu~^H / v_j
    T[:, :, np.arange(I), np.arange(I)] += np.einsum("jafn,jfn->fja", phi, 1.0 / v_new)
    Om = np.einsum("fjab,fji->fiab", T, 1.0 / lam_new)                 # sum_j T_j / lambda_ji
    PinvH = np.linalg.inv(P).conj().transpose(0, 2, 1)
    W = np.einsum("fac,ficd,fbd->fiab", PinvH, Om, PinvH.conj())       # P^{-H} Om_i P^{-1}
    return W / (J * N)


def _real_basis(I):
    """The 2 I^2 real directions of C^{I x I}: E_k = e_a e_i^T (k < I^2) and
    i e_a e_i^T (k >= I^2), k = a I + i within each half."""
    E = np.zeros((2 * I * I, I, I), dtype=np.complex128)
    for k in range(I * I):
        E[k, k // I, k % I] = 1.0
        E[I * I + k, k // I, k % I] = 1j
    return E


def newton_P(P, V, mu=1.0, K=1, counter=COUNTER):
    """K steps of Newton's method on L2 / N as a function of P with the V_i
    of Eq. FPI fixed (another of the alternatives named in Sec. 4.6; reading:
    the Newton step in the 2 I^2 real coordinates of P, restricted to the
    directions that change L2, scaled by mu).

    With l(P) = ln|det P|^2 - sum_i p_i^H V_i p_i (L2 / N up to terms free
    of P), the first and second differentials along complex directions D,
    D' are
        dl[D]      = 2 Re tr(G^H D),  G = P^{-H} - [V_1 p_1, ..., V_I p_I]
        d2l[D, D'] = -2 Re tr(P^{-1} D P^{-1} D') - 2 Re sum_i d_i^H V_i d'_i
    (from ln det(P + D) = ln det P + tr(P^{-1} D) - tr(P^{-1} D P^{-1} D) / 2
    + ...).  In the real basis E_k the gradient is g_k = dl[E_k] and the
    Hessian H_kl = d2l[E_k, E_l].  l does not change when a column turns in
    phase (p_i -> e^{i theta} p_i), so the I directions i p_i carry no
    information (g is orthogonal to them, and at a stationary point H is
    singular along them): with Pi the orthogonal projector onto them and
    Q = 1 - Pi, the step solves (Q H Q - Pi) s = -Q g, i.e. the Newton step
    within the directions orthogonal to the phase turns, and moves P by
    mu sum_k s_k E_k.  Two inversions per frequency per step: P and the
    2 I^2 x 2 I^2 system.  Newton's method converges quadratically near a
    nondegenerate stationary point and is not globally convergent (H is
    indefinite away from it); mu damps the step."""
    F, I, _ = P.shape
    E = _real_basis(I)
    eye = np.eye(2 * I * I)[None]
    P = P.copy()
    for _ in range(K):
        Pinv = np.linalg.inv(P)
        counter.inversions += F
        G = Pinv.conj().transpose(0, 2, 1) - np.einsum("fiab,fbi->fai", V, P)
        g = 2.0 * np.real(np.einsum("fai,kai->fk", G.conj(), E))
        A = np.einsum("fab,kbc->fkac", Pinv, E)                   # P^{-1} E_k
        H = -2.0 * np.real(np.einsum("fkab,flba->fkl", A, A))     # -2 Re tr(P^{-1}E_k P^{-1}E_l)
        H -= 2.0 * np.real(np.einsum("kai,fiab,lbi->fkl", E.conj(), V, E))
        # the phase-turn directions i p_i in real coordinates, orthonormalised
        turn = np.zeros((F, I, I, I), dtype=np.complex128)      # [f, column i, a, c]
        for i in range(I):
            turn[:, i, :, i] = 1j * P[:, :, i]
        Nt = np.concatenate([turn.real.reshape(F, I, -1), turn.imag.reshape(F, I, -1)], axis=2)
        Qn, _ = np.linalg.qr(Nt.transpose(0, 2, 1))               # [F, 2 I^2, I]
        Pi = Qn @ Qn.transpose(0, 2, 1)
        Qp = eye - Pi
        s = np.linalg.solve(Qp @ H @ Qp - Pi, -np.einsum("fkl,fl->fk", Qp, g)[..., None])[..., 0]
        counter.inversions += F  # the 2 I^2 x 2 I^2 system
        P = P + mu * np.einsum("fk,kai->fai", s, E)
    return P


# --------------------------------------------------------- log-likelihood ----
def loglik_terms(y, v, lam, P):
    """Per-(n,f) value of ln N(y; 0, P^{-H} D P^{-1}) in Eq. L2, D = sum_j v_j Lambda_j.

    For R = P^{-H} D P^{-1}: ln det R = sum_i ln sigma_i - ln |det P|^2 and
    y^H R^{-1} y = y^H P D^{-1} P^H y = sum_i |y~_i|^2 / sigma_i, so
    ln N = -I ln(pi) + ln|det P|^2 - sum_i (ln sigma_i + |y~_i|^2 / sigma_i).
    Returns [F, N].
    """
    I = y.shape[0]
    yt = basis_transform(y, P)
    sigma = model_variances(v, lam)
    _, logabsdet = np.linalg.slogdet(P)
    return (-I * LN_PI + 2.0 * logabsdet[:, None]
            - np.sum(np.log(sigma) + np.abs(yt) ** 2 / sigma, axis=0))


def loglik(y, v, lam, P):
    """Eq. L2: L2(Psi) = sum_{n,f} ln N(y(n,f); 0, sum_j v_j P^{-H} Lambda_j P^{-1})."""
    return float(np.sum(loglik_terms(y, v, lam, P)))


# ----------------------------------------------------------- the hybrid ----
def em_half(y, v, lam, P):
    """Step 1 of the hybrid algorithm (Sec. 4.4): one EM iteration for
    (v, Lambda): E-step (Eqs. mutilde0, Phitilde0), then Eq. updatev with the
    current Lambda, then Eq. Lambdaupdate with the new v."""
    mu, phi = e_step(y, v, lam, P)
    v_new = m_step_v(mu, phi, lam)
    lam_new = m_step_lambda(mu, phi, v_new)
    return v_new, lam_new


def hybrid_iteration(y, v, lam, P, K=1, counter=COUNTER, p_update="fpi", mu=0.0):
    """One iteration of the hybrid algorithm (Sec. 4.4): the EM half, then an
    update of P.  p_update selects it (the four alternatives are those Sec.
    4.6 names in place of the fixed-point iteration):

      "fpi"               Eq. FPI, K sweeps with the V_i of the new v, Lambda;
                          mu is not used.
      "gradient"          K gradient-ascent steps of size mu (gradient_P).
      "natural_gradient"  K natural-gradient steps of size mu
                          (natural_gradient_P).
      "newton"            K Newton steps scaled by mu (newton_P); mu = 0 is
                          taken as the undamped step mu = 1.
      "em"                the normal EM: K sweeps of Eq. FPI's form on the
                          M-step matrices W_i / (J N) of em_covariances, which
                          use the posterior of the entering state; mu is not
                          used.
    """
    if p_update == "em":  # the normal EM: Eq. FPI's form on the M-step's matrices
        v_new, lam_new = em_half(y, v, lam, P)
        P = fixed_point_P(P, em_covariances(y, v, lam, P, v_new, lam_new), K, counter)
        return v_new, lam_new, P
    v, lam = em_half(y, v, lam, P)
    V = weighted_covariances(y, v, lam)
    if p_update == "fpi":
        P = fixed_point_P(P, V, K, counter)
    elif p_update == "gradient":
        P = gradient_P(P, V, mu, K, counter)
    elif p_update == "natural_gradient":
        P = natural_gradient_P(P, V, mu, K)
    elif p_update == "newton":
        P = newton_P(P, V, mu if mu else 1.0, K, counter)
    else:
        raise ValueError(p_update)
    return v, lam, P


def iterate(y, v, lam, P, iters, K=1, counter=COUNTER, p_update="fpi", mu=0.0):
    """Run `iters` hybrid iterations.  Returns (v, lam, P, trace) where
    trace[t] is L2 of the state entering iteration t and trace[iters] is L2
    of the final state (length iters + 1)."""
    trace = []
    for _ in range(iters):
        trace.append(loglik(y, v, lam, P))
        v, lam, P = hybrid_iteration(y, v, lam, P, K, counter, p_update, mu)
    trace.append(loglik(y, v, lam, P))
    return v, lam, P, np.array(trace)


# ----------------------------------------------------------------- Wiener ----
def wiener(y, v, lam, P):
    """Multichannel Wiener filter, Eq. MMSE0, with R_j of Eq. covmodelprop.

    x^_j = R_j (sum_k R_k)^{-1} y = P^{-H} mu~_j with mu~_j from Eq. mutilde0
    (mu~_j = P^H mu_j).  Returns [J, I, F, N] complex.
    """
    mu, _ = e_step(y, v, lam, P)
    PinvH = np.linalg.inv(P).conj().transpose(0, 2, 1)
    return np.einsum("fab,jbfn->jafn", PinvH, mu)
