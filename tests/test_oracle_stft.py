"""Pins of the STFT oracle (Table 1 analysis conditions) against routes
other than itself: the window identity that makes the square-root Hann pair
reconstruct, the closed-form transform of an impulse and of a single
windowed exponential (direct sums, no FFT), Parseval per frame, and exact
reconstruction by the overlap-add inverse."""
import numpy as np
import pytest

from oracle import stft as so


def test_window_is_sqrt_periodic_hann_and_sums_to_one():
    w = so.window()
    t = np.arange(so.L)
    assert np.allclose(w, np.sin(np.pi * t / so.L), atol=1e-15)
    # analysis x synthesis = Hann; Hann(t) + Hann(t + L/2) = 1 (shift H = L/2)
    assert np.allclose(w[:so.H] ** 2 + w[so.H:] ** 2, 1.0, atol=1e-15)


def test_impulse_closed_form():
    """x = delta(s - s0): X(n, f) = w(s0 - n H) exp(-2 pi i f (s0 - n H) / L)
    for the frames that hold s0, zero elsewhere."""
    S, s0 = 4096, 1500
    x = np.zeros((1, S))
    x[0, s0] = 1.0
    X = so.stft(x)[0]
    N = so.frames_of(S)
    f = np.arange(so.F)
    for n in range(N):
        t = s0 - n * so.H
        want = np.zeros(so.F, complex) if not 0 <= t < so.L else \
            so.window()[t] * np.exp(-2j * np.pi * f * t / so.L)
        assert np.allclose(X[:, n], want, atol=1e-12), n


def test_direct_dft_of_random_frames():
    """Every bin against the defining sum, written out (no FFT)."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, so.L + 3 * so.H + 17))
    X = so.stft(x)
    N = X.shape[2]
    t = np.arange(so.L)
    E = np.exp(-2j * np.pi * np.outer(np.arange(so.F), t) / so.L)   # [F, L]
    for c in range(2):
        for n in range(N):
            seg = so.window() * x[c, n * so.H: n * so.H + so.L]
            assert np.allclose(X[c, :, n], E @ seg, atol=1e-9)


def test_parseval_per_frame():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((1, 3 * so.L))
    X = so.stft(x)[0]
    for n in range(X.shape[1]):
        seg = so.window() * x[0, n * so.H: n * so.H + so.L]
        e = (abs(X[0, n]) ** 2 + 2 * np.sum(abs(X[1:-1, n]) ** 2) + abs(X[-1, n]) ** 2) / so.L
        assert np.isclose(e, np.sum(seg ** 2), rtol=1e-12)


@pytest.mark.parametrize("S", [so.L, so.L + so.H, 5000, 20 * so.H + so.L])
def test_overlap_add_reconstructs(S):
    rng = np.random.default_rng(S)
    x = rng.standard_normal((3, S))
    X = so.stft(x)
    N = X.shape[2]
    y = so.istft(X)
    assert y.shape == (3, (N - 1) * so.H + so.L)
    # samples covered by two frames come back exactly
    assert np.allclose(y[:, so.H: N * so.H], x[:, so.H: N * so.H], atol=1e-12)
    # the outer half frames carry the squared window
    w2 = so.window() ** 2
    assert np.allclose(y[:, :so.H], x[:, :so.H] * w2[:so.H], atol=1e-12)


def test_frames_of():
    assert so.frames_of(so.L - 1) == 0
    assert so.frames_of(so.L) == 1
    assert so.frames_of(so.L + so.H - 1) == 1
    assert so.frames_of(so.L + so.H) == 2
