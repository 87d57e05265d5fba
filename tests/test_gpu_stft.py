"""GPU parity of the STFT front end and overlap-add back end (ffca_stft,
ffca_istft through the C ABI) against the FP64 oracle: random signals of
several channel counts and lengths (one frame, a ragged last CTA of frames,
padded frame strides), zeroed padding frames, the round trip, and the
length of the benchmark mixture.  FP32 arithmetic: normwise relative error
per bin (per channel for signals) below 1e-5."""
import numpy as np
import pytest

from oracle import stft as so

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1805_09498_gb300 import build
    build.build()


def _relerr_bins(got, ref):
    num = np.linalg.norm(got - ref, axis=-1)
    den = np.maximum(np.linalg.norm(ref, axis=-1), 1e-30)
    return float(np.max(num / den))


@pytest.mark.parametrize("C,S,extra_ld", [(1, so.L, 0), (3, so.L + 7 * so.H + 100, 0), (2, so.L + 8 * so.H, 4),
                                          (4, so.L + 36 * so.H + 511, 8), (1, so.L + 63 * so.H, 0)])
def test_stft_matches_oracle(C, S, extra_ld):
    import torch
    from paper_1805_09498_gb300 import ffca
    rng = np.random.default_rng(C * 1000 + S)
    x = rng.standard_normal((C, S)).astype(np.float32)
    N = so.frames_of(S)
    ld = ffca.padded_ld(N) + extra_ld
    X, Ng = ffca.stft(torch.from_numpy(x).cuda(), ld=ld)
    torch.cuda.synchronize()
    assert Ng == N
    Xg = X.cpu().numpy()
    ref = so.stft(x.astype(np.float64))
    assert _relerr_bins(Xg[:, :, :N], ref) <= TOL
    assert np.all(Xg[:, :, N:] == 0)


@pytest.mark.parametrize("C,N,extra_ld", [(1, 1, 0), (2, 7, 0), (3, 8, 4), (1, 9, 0), (2, 37, 8)])
def test_istft_matches_oracle(C, N, extra_ld):
    import torch
    from paper_1805_09498_gb300 import ffca
    rng = np.random.default_rng(7 * N + C)
    # arbitrary spectra (the inverse ignores the imaginary parts of bins 0 and L/2, as irfft does)
    X = (rng.standard_normal((C, so.F, N)) + 1j * rng.standard_normal((C, so.F, N)))
    ld = ffca.padded_ld(N) + extra_ld
    Xd = np.zeros((C, so.F, ld), np.complex64)
    Xd[:, :, :N] = X
    Xd[:, :, N:] = 1e30           # padding frames must not be read
    y = ffca.istft(torch.from_numpy(Xd).cuda(), N)
    torch.cuda.synchronize()
    ref = so.istft(X.astype(np.complex64).astype(np.complex128))
    yg = y.cpu().numpy()
    assert yg.shape == ref.shape
    assert float(np.max(np.linalg.norm(yg - ref, axis=1) / np.linalg.norm(ref, axis=1))) <= TOL


def test_round_trip_and_benchmark_length():
    """Three channels of the long mixture's length (N = 20000 frames): the
    GPU round trip returns the interior samples; sampled frames match the
    oracle."""
    import torch
    from paper_1805_09498_gb300 import ffca
    N = 20000
    S = (N - 1) * so.H + so.L
    rng = np.random.default_rng(11)
    x = rng.standard_normal((3, S)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    X, Ng = ffca.stft(xd)
    y = ffca.istft(X, Ng)
    torch.cuda.synchronize()
    assert Ng == N
    yi = y[:, so.H: N * so.H].cpu().numpy()
    xi = x[:, so.H: N * so.H]
    assert float(np.max(np.linalg.norm(yi - xi, axis=1) / np.linalg.norm(xi, axis=1))) <= TOL
    for n in (0, 1, 7, 8, 9999, N - 1):
        seg = x[:, n * so.H: n * so.H + so.L].astype(np.float64) * so.window()[None]
        ref = np.fft.rfft(seg, axis=-1)                           # [C, F]
        got = X[:, :, n].cpu().numpy()
        assert _relerr_bins(got, ref) <= TOL


def test_persistent_loop_and_unaligned_buffers():
    """More groups of frames than resident CTAs (several per CTA, each
    CTA's next group copied while it transforms one), with a signal that
    starts 4 bytes past a 16-byte boundary and an odd length (4-byte
    copies), and an inverse written 4 bytes past a 16-byte boundary
    (scalar stores), against the oracle."""
    import ctypes
    import torch
    from paper_1805_09498_gb300 import ffca
    C, N = 2, 3001
    S = (N - 1) * so.H + so.L + 3
    rng = np.random.default_rng(5)
    x = rng.standard_normal((C, S)).astype(np.float32)
    flat = torch.zeros(C * S + 1, dtype=torch.float32, device="cuda")
    flat[1:] = torch.from_numpy(x.ravel()).cuda()
    xd = flat[1:].view(C, S)
    X, Ng = ffca.stft(xd)
    torch.cuda.synchronize()
    assert Ng == N
    Xg = X.cpu().numpy()
    for n in (0, 1, 8, 1500, N - 2, N - 1):
        seg = x[:, n * so.H: n * so.H + so.L].astype(np.float64) * so.window()[None]
        assert _relerr_bins(Xg[:, :, n], np.fft.rfft(seg, axis=-1)) <= TOL
    assert np.all(Xg[:, :, N:] == 0)
    out = torch.full((C * (N + 1) * so.H + 1,), float("nan"), dtype=torch.float32, device="cuda")
    L = ffca.lib()
    s = torch.cuda.current_stream().cuda_stream
    assert L.ffca_istft(X.data_ptr(), C, N, X.shape[2], ctypes.c_void_p(out.data_ptr() + 4), s) == 0
    torch.cuda.synchronize()
    y = out[1:].view(C, -1).cpu().numpy()
    ref = so.istft(Xg[:, :, :N].astype(np.complex128))
    assert float(np.max(np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1))) <= TOL


def test_bad_arguments_are_rejected():
    import torch
    from paper_1805_09498_gb300 import ffca
    x = torch.zeros((1, so.L), dtype=torch.float32, device="cuda")
    out = torch.zeros((1, so.F, 4), dtype=torch.complex64, device="cuda")
    L = ffca.lib()
    s = torch.cuda.current_stream().cuda_stream
    assert L.ffca_stft(x.data_ptr(), 1, so.L, out.data_ptr(), 3, s) == 1       # ld % 4 != 0
    assert L.ffca_stft(x.data_ptr(), 1, so.L, out.data_ptr() + 8, 4, s) == 1   # misaligned output
    assert L.ffca_stft(x.data_ptr(), 1, so.L - 1, out.data_ptr(), 4, s) == 0   # no frame: no-op
    assert L.ffca_istft(out.data_ptr(), 1, 5, 4, x.data_ptr(), s) == 1         # ld < N


def test_time_domain_pipeline():
    """Time-domain mixture -> STFT -> FastFCA-AS iterations -> Wiener filter ->
    overlap-add: the separated images of the J sources sum back to the
    mixture on the samples two frames cover (the Wiener gains sum to one per
    point, Eq. MMSE0)."""
    import torch
    from paper_1805_09498_gb300 import ffca
    from paper_1805_09498_gb300.synth import make_problem
    I, J, F, N = 3, 3, so.F, 64
    p = make_problem(I, J, F, N, seed=21)
    # a consistent mixture: the time signal of the model's mixture spectra
    xt = so.istft(p.y)                                     # [I, (N+1) H]
    xd = torch.from_numpy(xt.astype(np.float32)).cuda()
    Y, Ng = ffca.stft(xd)                                  # [I, F, ld] c64, Ng = N
    assert Ng == N
    v = torch.ones((J, F, Y.shape[2]), dtype=torch.float32, device="cuda")
    v[:, :, :N] = torch.from_numpy(p.v0.astype(np.float32)).cuda()
    lam = torch.from_numpy(p.lam0).cuda()
    P = torch.from_numpy(p.P0).cuda()
    est = ffca.FastFCA(Y, v, lam, P, N=N)
    tr = est.iterate(5)
    X = est.wiener()                                       # [J, I, F, ld]
    imgs = ffca.istft(X.view(J * I, F, -1).contiguous(), N)  # [J I, (N+1) H]
    torch.cuda.synchronize()
    est.close()
    assert np.all(np.isfinite(tr))
    s = imgs.view(J, I, -1).sum(dim=0).cpu().numpy()
    mix = ffca.istft(Y, N).cpu().numpy()
    lo, hi = so.H, N * so.H
    err = np.linalg.norm(s[:, lo:hi] - mix[:, lo:hi], axis=1) / np.linalg.norm(mix[:, lo:hi], axis=1)
    assert float(err.max()) <= TOL
