"""Accuracy of the mixed-precision path as the mixture gets longer.

The mixed path sums over the frames n in FP32 (compensated: Kahan sums per
thread where the registers hold them, flushes into FP64 slots where they do
not) and finishes in FP64.  The error of a plain FP32 sum grows with the
number of terms each thread adds; these tests run one hybrid iteration (the
well-conditioned one-step map, Sec. 4.4) on mixtures long enough that every
thread adds hundreds of units per segment, and check the result against the
FP64 oracle on sampled frequencies: within the stated tolerances (1e-4 on
parameters, 1e-5 per time-frequency point on L2) and, for the long-mixture
shape, no larger at N = 200000 than at N = 2000.

Inputs are drawn on the device (synth.make_batch_device with one mixture:
the single-mixture layout); the oracle reads the same values, widened to
FP64.
"""
import numpy as np
import pytest

from helpers import per_f_relerr

pytestmark = pytest.mark.gpu


def _draw(I, J, F, N, seed):
    import torch
    from paper_1805_09498_gb300.synth import make_batch_device
    alpha, kappa = (0.2, 50.0) if I == 8 else (0.3, 10.0)
    y, v, lam, P, _, off = make_batch_device(I, J, F, [N], seed=seed, device="cuda", alpha=alpha,
                                             kappa=kappa)
    ld = int(off[1])
    torch.cuda.synchronize()
    return y.view(I, F, ld), v.view(J, F, ld), lam[0].contiguous(), P[0].contiguous()


def _host(y, v, lam, P, fs, N):
    """FP64 host copies of the sampled frequencies (the values the GPU reads)."""
    return (y[:, fs, :N].cpu().numpy().astype(np.complex128), v[:, fs, :N].cpu().numpy().astype(np.float64),
            lam[fs].cpu().numpy(), P[fs].cpu().numpy())


def _oracle_loglik_all(y, v, lam, P, N, chunk=32):
    """L2 of the whole mixture by the oracle, frequency block by block."""
    from oracle import fastfca_as as ffa
    F = y.shape[1]
    tot = 0.0
    for f0 in range(0, F, chunk):
        fs = list(range(f0, min(F, f0 + chunk)))
        tot += ffa.loglik(*_host(y, v, lam, P, fs, N))
    return tot


def _one_iteration_errors(I, J, F, N, fs, seed=3, with_l2=False):
    import torch
    from oracle import fastfca_as as ffa
    from oracle.fastfca_as import OpCounter
    from paper_1805_09498_gb300 import ffca
    y, v, lam, P = _draw(I, J, F, N, seed)
    yh, vh, lh, Ph = _host(y, v, lam, P, fs, N)
    l2_ref = _oracle_loglik_all(y, v, lam, P, N) if with_l2 else None
    est = ffca.FastFCA(y, v, lam, P, N=N)
    tr = est.iterate(1)
    torch.cuda.synchronize()
    vg, lg, Pg = v[:, fs, :N].double().cpu().numpy(), lam[fs].cpu().numpy(), P[fs].cpu().numpy()
    est.close()
    vr, lr, Pr = ffa.hybrid_iteration(yh, vh, lh, Ph, 1, OpCounter())
    e = {"v": per_f_relerr(vg, vr, 1), "lambda": per_f_relerr(lg, lr, 0), "P": per_f_relerr(Pg, Pr, 0)}
    if with_l2:
        e["l2_per_point"] = abs(tr[0] - l2_ref) / (F * N)
    del y, v, lam, P
    torch.cuda.empty_cache()
    return e


def test_long_mixture_error_does_not_grow_with_n():
    """I = J = 3, F = 513 (the long-mixture shape): N = 2000, 20000, 200000;
    per thread and segment that is about 7, 75 and 750 units of two frames."""
    fs = [0, 171, 342, 512]
    errs = {N: _one_iteration_errors(3, 3, 513, N, fs, with_l2=True) for N in (2000, 20000, 200000)}
    print("errors by N:", errs)
    for N, e in errs.items():
        assert max(e["v"], e["lambda"], e["P"]) < 1e-4, (N, e)
        assert e["l2_per_point"] < 1e-5, (N, e)
    for k in ("lambda", "P", "l2_per_point"):
        assert errs[200000][k] <= 2.0 * max(errs[2000][k], errs[20000][k]) + 1e-9, (k, errs)


@pytest.mark.parametrize("I,J,F,N", [(4, 3, 64, 300000), (8, 6, 64, 160000)])
def test_flushed_sums_long_mixture(I, J, F, N):
    """The shapes whose per-thread sums are flushed into FP64 slots instead of
    compensated in registers (pass B at I = 4; both passes at I = 8), long
    enough that every group flushes within a segment."""
    e = _one_iteration_errors(I, J, F, N, [0, F - 1])
    print(f"I={I} J={J} F={F} N={N}:", e)
    assert max(e["v"], e["lambda"], e["P"]) < 1e-4, e
