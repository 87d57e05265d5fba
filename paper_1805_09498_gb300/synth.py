"""Seeded synthetic mixtures drawn from the FastFCA-AS generative model.

This module only draws random numbers and assembles the mixture the model
describes; it holds none of the estimation method's arithmetic, so both the
FP64 oracle (tests) and the CUDA path (library, benchmark) can take their
inputs from it.

Model (Sec. 3.1, Eqs. srcmodel and fullrank; Sec. 4.1, Eq. diagconst):
    x_j(n,f) ~ CN(0, v_j(n,f) S_j(f)),   S_j(f) = P(f)^{-H} Lambda_j(f) P(f)^{-1}
    y(n,f)   = sum_j x_j(n,f)
Sampling x_j = P^{-H} s_j with s_j ~ CN(0, v_j Lambda_j) (independent entries)
gives exactly Cov x_j = v_j P^{-H} Lambda_j P^{-1}.

Recipe (the paper's speech/RIR data are not available; these stand in):
    P(f)        = I + alpha * G,  G_kl ~ CN(0, 1), redrawn until cond_2(P) < kappa
    lambda_ji(f) = exp(N(0, 1))              (log-normal, sigma = 1)
    v_j(n,f)    ~ Gamma(shape 0.5, scale 1)
    CN(0, 1): real and imaginary parts each N(0, 1/2).
Initial estimate ("perturbed truth", separate stream seed + 1000):
    P0 = P (I + 0.1 G'),  lambda0 = lambda * exp(0.3 xi),  v0 = v * exp(0.3 xi')

Array layouts (mic-planar, the layout the CUDA kernels stream):
    y      [I][F][N]    complex128   the observed mixture (called x in some APIs)
    x      [J][I][F][N] complex128   source images (only when keep_images)
    v      [J][F][N]    float64      source power spectra
    lam    [F][J][I]    float64      diagonal entries of Lambda_j(f)
    P      [F][I][I]    complex128   row-major: P[f, a, i] = [P(f)]_{a i}
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["Problem", "make_problem", "batch_lengths", "make_batch", "make_batch_device", "CONFIGS",
           "cn", "draw_P"]


def cn(rng: np.random.Generator, shape) -> np.ndarray:
    """Standard circular complex Gaussian CN(0, 1) samples."""
    s = np.sqrt(0.5)
    return s * rng.standard_normal(shape) + 1j * (s * rng.standard_normal(shape))


def draw_P(rng: np.random.Generator, F: int, I: int, alpha: float, kappa: float) -> np.ndarray:
    """P(f) = I + alpha*G, redrawn until its 2-norm condition number is below kappa."""
    P = np.empty((F, I, I), dtype=np.complex128)
    eye = np.eye(I)
    for f in range(F):
        while True:
            M = eye + alpha * cn(rng, (I, I))
            if np.linalg.cond(M) < kappa:
                break
        P[f] = M
    return P


@dataclass
class Problem:
    I: int
    J: int
    F: int
    N: int
    y: np.ndarray
    v_true: np.ndarray
    lam_true: np.ndarray
    P_true: np.ndarray
    v0: np.ndarray
    lam0: np.ndarray
    P0: np.ndarray
    x: np.ndarray | None = None


def make_problem(I: int, J: int, F: int, N: int, seed: int, alpha: float = 0.3,
                 kappa: float = 10.0, keep_images: bool = False) -> Problem:
    """Draw one mixture and its perturbed-truth initial estimate.

    The draw order is fixed (P, lambda, v, then sources j = 0..J-1), so a seed
    always gives the same problem.
    """
    rng = np.random.default_rng(seed)
    P = draw_P(rng, F, I, alpha, kappa)
    lam = np.exp(rng.standard_normal((F, J, I)))
    v = rng.gamma(0.5, 1.0, size=(J, F, N))
    # P^{-H} for every f: the mixing of the (independent) transformed sources.
    PinvH = np.linalg.inv(P).conj().transpose(0, 2, 1)
    y = np.zeros((I, F, N), dtype=np.complex128)
    x = np.empty((J, I, F, N), dtype=np.complex128) if keep_images else None
    for j in range(J):
        std = np.sqrt(v[j][None, :, :] * lam[:, j, :].T[:, :, None])   # [I, F, N]
        s = std * cn(rng, (I, F, N))
        xj = np.einsum("fab,bfn->afn", PinvH, s)
        y += xj
        if keep_images:
            x[j] = xj
    r2 = np.random.default_rng(seed + 1000)
    P0 = np.einsum("fab,fbc->fac", P, np.eye(I)[None] + 0.1 * cn(r2, (F, I, I)))
    lam0 = lam * np.exp(0.3 * r2.standard_normal(lam.shape))
    v0 = v * np.exp(0.3 * r2.standard_normal(v.shape))
    return Problem(I, J, F, N, y, v, lam, P, v0, lam0, P0, x)


def batch_lengths(M: int, N_min: int, N_max: int, seed: int) -> np.ndarray:
    """M mixture lengths drawn uniformly from the integers [N_min, N_max]."""
    return np.random.default_rng(seed).integers(N_min, N_max + 1, size=M)


def make_batch(I: int, J: int, F: int, Ns, seed: int, alpha: float = 0.3,
               kappa: float = 10.0) -> list[Problem]:
    """Independent mixtures of lengths Ns; mixture m is make_problem(seed + 7919 m)."""
    return [make_problem(I, J, F, int(n), seed + 7919 * m, alpha, kappa) for m, n in enumerate(Ns)]


def make_batch_device(I: int, J: int, F: int, Ns, seed: int, device, alpha: float = 0.3,
                      kappa: float = 10.0, complex_dtype=None):
    """The same model as make_problem for M mixtures, drawn on the device
    (torch's generator) straight into the mixture-major batch layout: flat y
    and v holding mixture m's blocks [I,F,ld_m] and [J,F,ld_m] one after
    another, ld_m = off[m+1] - off[m] = Ns[m] rounded up to a multiple of 4.

    Used where numpy would take minutes (hundreds of mixtures); the numbers
    differ from make_problem's (another generator), the distributions are
    the same.  Gamma(shape 1/2, scale 1) is drawn as z^2 / 2, z ~ N(0, 1).
    Returns (y, v0, lam0 [M,F,J,I] f64, P0 [M,F,I,I] c128, Ns, off); padding
    frames hold y = 0, v = 1.
    """
    import torch
    cdt = torch.complex64 if complex_dtype is None else complex_dtype
    rdt = torch.float32 if cdt == torch.complex64 else torch.float64
    Ns = [int(n) for n in Ns]
    M = len(Ns)
    off = np.zeros(M + 1, dtype=np.int64)
    off[1:] = np.cumsum([(n + 3) // 4 * 4 for n in Ns])
    ld = int(off[-1])
    rng = np.random.default_rng(seed)
    P = draw_P(rng, M * F, I, alpha, kappa).reshape(M, F, I, I)
    lam = np.exp(rng.standard_normal((M, F, J, I)))
    r2 = np.random.default_rng(seed + 1000)
    P0 = np.einsum("mfab,mfbc->mfac", P, np.eye(I) + 0.1 * cn(r2, (M, F, I, I)))
    lam0 = lam * np.exp(0.3 * r2.standard_normal(lam.shape))
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    PinvH = torch.from_numpy(np.linalg.inv(P).conj().swapaxes(-1, -2)).to(device)  # [M,F,I,I]
    lam_d = torch.from_numpy(lam).to(device)
    y = torch.zeros(I * F * ld, dtype=cdt, device=device)
    v0 = torch.ones(J * F * ld, dtype=rdt, device=device)
    s2 = float(np.sqrt(0.5))
    for m in range(M):
        o, n, ldm = int(off[m]), Ns[m], int(off[m + 1] - off[m])
        yb = y[I * F * o: I * F * (o + ldm)].view(I, F, ldm)
        vb = v0[J * F * o: J * F * (o + ldm)].view(J, F, ldm)
        z = torch.randn((J, F, n), generator=g, device=device, dtype=torch.float64)
        v = 0.5 * z * z                                                   # Gamma(0.5, 1)
        ym = torch.zeros((F, I, n), dtype=torch.complex128, device=device)
        for j in range(J):
            std = torch.sqrt(v[j][:, None, :] * lam_d[m, :, j, :][:, :, None])   # [F, I, n]
            re = torch.randn((F, I, n), generator=g, device=device, dtype=torch.float64)
            im = torch.randn((F, I, n), generator=g, device=device, dtype=torch.float64)
            ym += torch.matmul(PinvH[m], torch.complex(s2 * std * re, s2 * std * im))
        yb[:, :, :n] = ym.permute(1, 0, 2).to(cdt)
        xi = torch.randn((J, F, n), generator=g, device=device, dtype=torch.float64)
        vb[:, :, :n] = (v * torch.exp(0.3 * xi)).to(rdt)
    return (y, v0, torch.from_numpy(lam0).to(device), torch.from_numpy(P0).to(device), Ns, off)


# Workloads: sizes, value distributions and precision of each measured case.
CONFIGS = {
    "plain_fp64": dict(I=3, J=3, F=257, N=600, iters=20, prec="fp64", alpha=0.3, kappa=10.0),
    "long_mixed": dict(I=3, J=3, F=513, N=20000, iters=50, prec="mixed", alpha=0.3, kappa=10.0),
    "large_array": dict(I=8, J=6, F=513, N=4000, iters=30, prec="mixed", alpha=0.2, kappa=50.0),
    "batched": dict(I=4, J=3, F=257, M=256, N_min=200, N_max=4000, iters=20, prec="mixed",
                    alpha=0.3, kappa=10.0),
    "adjoint": dict(I=4, J=4, F=257, N=2000, prec="fp32", alpha=0.3, kappa=10.0),
}
