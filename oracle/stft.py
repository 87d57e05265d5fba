"""FP64 CPU oracle of the STFT front end and its inverse (Table 1 of Ito &
Nakatani, arXiv 1805.09498: frame length 1024, frame shift 512, square root
of the Hann window; bins up to the Nyquist frequency, Sec. 2).

TEST INFRASTRUCTURE ONLY. Only tests and the benchmark may import this
module; the library never does.  It shares no code with the CUDA path.

Readings (the paper states only the table's parameters):
  * the Hann window is the periodic one, w_H(t) = (1 - cos(2 pi t / L)) / 2,
    so that w_H(t) + w_H(t + L/2) = 1 and the square-root window used for
    analysis and again for synthesis reconstructs exactly with shift L/2;
    its square root is sin(pi t / L);
  * frame n holds samples n H .. n H + L - 1 (no padding: N = 1 + (S - L) // H
    frames of a signal of S >= L samples);
  * X(n, f) = sum_t w(t) x(n H + t) exp(-2 pi i f t / L), f = 0 .. L/2,
    unnormalised; the inverse is the weighted overlap-add of the windowed
    inverse DFTs, x(s) = sum_n w(s - n H) IDFT_L(X(n, .))(s - n H) with the
    1 / L of the inverse DFT and X(n, L - f) = conj(X(n, f)).
Layouts: signals [C, S] real, spectra [C, F, N] complex (the mic-planar
layout of the mixture y in the estimation API).
"""
from __future__ import annotations

import numpy as np

L = 1024   # frame length (Table 1)
H = 512    # frame shift (Table 1)
F = L // 2 + 1


def window(n: int = L) -> np.ndarray:
    """Square root of the periodic Hann window of length n."""
    t = np.arange(n)
    return np.sqrt(0.5 - 0.5 * np.cos(2.0 * np.pi * t / n))


def frames_of(S: int) -> int:
    """Frames of a signal of S samples (no padding)."""
    return 1 + (S - L) // H if S >= L else 0


def stft(x: np.ndarray) -> np.ndarray:
    """x [C, S] real -> X [C, F, N] complex128; np.fft.rfft is the DFT step."""
    x = np.asarray(x, dtype=np.float64)
    C, S = x.shape
    N = frames_of(S)
    w = window()
    idx = np.arange(N)[:, None] * H + np.arange(L)[None, :]     # [N, L]
    seg = x[:, idx] * w[None, None, :]                          # [C, N, L]
    return np.fft.rfft(seg, axis=-1).transpose(0, 2, 1)         # [C, F, N]


def istft(X: np.ndarray) -> np.ndarray:
    """X [C, F, N] complex -> x [C, (N - 1) H + L] real: weighted overlap-add
    of the windowed inverse DFTs (np.fft.irfft is the inverse DFT step)."""
    X = np.asarray(X, dtype=np.complex128)
    C, Fb, N = X.shape
    assert Fb == F
    w = window()
    seg = np.fft.irfft(X.transpose(0, 2, 1), n=L, axis=-1) * w[None, None, :]   # [C, N, L]
    out = np.zeros((C, (N - 1) * H + L)) if N else np.zeros((C, 0))
    for n in range(N):
        out[:, n * H: n * H + L] += seg[:, n]
    return out
