"""GPU parity of the batched FastFCA-AS path (many mixtures of uneven length
in one set of launches, ffca_batch_*) against the FP64 CPU oracle run on
each mixture separately, and against the single-mixture entry points.

Tolerances as for one mixture, per mixture m:
    FP64 path:  1e-9 normwise per frequency on v, Lambda, P; 1e-9 relative on L2
    mixed path: 1e-4 on v, Lambda, P; |dL2_m| / (N_m F) <= 1e-5 nats per point
"""
import numpy as np
import pytest

from oracle import fastfca_as as ffa
from oracle.fastfca_as import OpCounter
from paper_1805_09498_gb300.synth import batch_lengths, make_batch

from helpers import per_f_relerr

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(par=1e-9, ll_rel=1e-9), "mixed": dict(par=1e-4, ll_tf=1e-5)}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1805_09498_gb300 import build
    build.build()


def _run_batch(probs, iters, prec, K=1, graph=False, pad_value=None, trace=True):
    import torch
    from paper_1805_09498_gb300 import ffca
    y, v, lam, P, Ns, off = ffca.batch_to_device([p.y for p in probs], [p.v0 for p in probs],
                                                 [p.lam0 for p in probs], [p.P0 for p in probs],
                                                 prec=prec, pad_value=pad_value)
    est = ffca.FastFCABatch(y, v, lam, P, Ns, K=K, graph=graph)
    tr = est.iterate(iters, trace=trace)
    ll = est.loglik()
    torch.cuda.synchronize()
    vh = v.double().cpu()
    J, F = probs[0].J, probs[0].F
    vs = [b[:, :, :Ns[m]].numpy() for m, b in enumerate(ffca.batch_views(vh, J, F, off))]
    vh = vh.numpy()
    out = dict(v=vs, lam=lam.cpu().numpy(), P=P.cpu().numpy(), trace=tr, ll=ll, vall=vh)
    est.close()
    return out


def _check(prec, probs, refs, got):
    tol = TOL[prec]
    for m, (p, r) in enumerate(zip(probs, refs)):
        e = dict(v=per_f_relerr(got["v"][m], r[0], 1), lam=per_f_relerr(got["lam"][m], r[1], 0),
                 P=per_f_relerr(got["P"][m], r[2], 0))
        for k, x in e.items():
            assert x <= tol["par"], (m, k, x, e)
        ll_ref = ffa.loglik(p.y, r[0], r[1], r[2])
        if prec == "fp64":
            assert abs(got["ll"][m] - ll_ref) <= tol["ll_rel"] * abs(ll_ref), (m, got["ll"][m], ll_ref)
        else:
            assert abs(got["ll"][m] - ll_ref) <= tol["ll_tf"] * p.N * p.F, (m, got["ll"][m], ll_ref)
    # the trace is the sum over mixtures of each mixture's trace
    t_ref = np.sum([r[3] for r in refs], axis=0)
    NF = sum(p.N * p.F for p in probs)
    if prec == "fp64":
        assert np.all(np.abs(got["trace"] - t_ref) <= tol["ll_rel"] * np.abs(t_ref))
    else:
        assert np.all(np.abs(got["trace"] - t_ref) <= tol["ll_tf"] * NF)


RAGGED = [37, 200, 5, 129, 64, 8, 301]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("IJ", [(3, 2), (4, 3), (2, 3), (1, 2)])
def test_ragged_batch_matches_oracle(prec, IJ):
    """Seven mixtures of 5 to 301 frames (several below one tile, one of them
    shorter than a vector unit pair) run together for three iterations."""
    I, J = IJ
    Ns = [max(n, I) for n in RAGGED]
    probs = make_batch(I, J, 6, Ns, seed=40 + I)
    refs = [ffa.iterate(p.y, p.v0, p.lam0, p.P0, 3, counter=OpCounter()) for p in probs]
    got = _run_batch(probs, 3, prec)
    _check(prec, probs, refs, got)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_workload_shape(prec):
    """The batched workload's shape (I = 4, J = 3, lengths uniform in
    [200, 4000]) at 12 mixtures and 9 frequencies, five iterations, K = 2."""
    Ns = batch_lengths(12, 200, 4000, seed=3)
    probs = make_batch(4, 3, 9, Ns, seed=11)
    refs = [ffa.iterate(p.y, p.v0, p.lam0, p.P0, 5, K=2, counter=OpCounter()) for p in probs]
    got = _run_batch(probs, 5, prec, K=2)
    _check(prec, probs, refs, got)


def test_batch_agrees_with_single_mixture_api():
    """FP64: each mixture of a batch equals the same mixture run alone
    (different work partitions, so equal up to summation order)."""
    import torch
    from paper_1805_09498_gb300 import ffca
    probs = make_batch(3, 3, 5, [77, 1030, 12], seed=2)
    got = _run_batch(probs, 4, "fp64")
    for m, p in enumerate(probs):
        yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="fp64")
        est = ffca.FastFCA(yd, vd, ld_, Pd, N=N)
        est.iterate(4, trace=False)
        ll = est.loglik()
        torch.cuda.synchronize()
        assert per_f_relerr(got["v"][m], vd[:, :, :N].cpu().numpy(), 1) < 1e-12
        assert per_f_relerr(got["P"][m], Pd.cpu().numpy(), 0) < 1e-12
        assert abs(got["ll"][m] - ll) <= 1e-12 * abs(ll)
        est.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_replay_is_bit_identical(prec):
    """Iterations replayed from the captured CUDA graph give the same bits as
    the plain launch sequence (same kernels, same partition), also when the
    graph is replayed more than once."""
    probs = make_batch(4, 3, 5, [300, 41, 1200, 96], seed=8)
    a = _run_batch(probs, 3, prec, trace=False)
    import torch
    from paper_1805_09498_gb300 import ffca
    y, v, lam, P, Ns, off = ffca.batch_to_device([p.y for p in probs], [p.v0 for p in probs],
                                                 [p.lam0 for p in probs], [p.P0 for p in probs],
                                                 prec=prec)
    est = ffca.FastFCABatch(y, v, lam, P, Ns, graph=True)
    est.iterate(1, trace=False)   # captures a one-iteration graph
    est.iterate(1, trace=False)   # replays it
    est.iterate(1, trace=False)
    torch.cuda.synchronize()
    assert np.array_equal(v.double().cpu().numpy(), a["vall"])
    assert np.array_equal(lam.cpu().numpy(), a["lam"])
    assert np.array_equal(P.cpu().numpy(), a["P"])
    est.close()


def test_padding_between_mixtures_is_ignored():
    """NaN in every padding frame of every mixture's rows changes nothing in
    the estimates (the padding is never read as data)."""
    probs = make_batch(3, 2, 4, [13, 50, 7], seed=4)
    a = _run_batch(probs, 2, "mixed")
    b = _run_batch(probs, 2, "mixed", pad_value=float("nan"))
    for m in range(3):
        assert np.array_equal(a["v"][m], b["v"][m])
    assert np.array_equal(a["lam"], b["lam"]) and np.array_equal(a["P"], b["P"])


def test_singular_problem_reports_its_index():
    """A mixture whose frequency 2 is all zero makes P(f)'s system singular
    there; the error names problem m F + f."""
    from paper_1805_09498_gb300 import ffca
    probs = make_batch(3, 2, 4, [40, 60, 30], seed=6)
    probs[1].y[:, 2, :] = 0.0
    with pytest.raises(ffca.FFCAError) as ei:
        _run_batch(probs, 2, "fp64")
    assert ei.value.status == 4 and ei.value.frequency == 1 * 4 + 2


def test_invalid_batches_are_rejected():
    import torch
    from paper_1805_09498_gb300 import ffca
    probs = make_batch(2, 2, 3, [10, 20], seed=1)
    y, v, lam, P, Ns, off = ffca.batch_to_device([p.y for p in probs], [p.v0 for p in probs],
                                                 [p.lam0 for p in probs], [p.P0 for p in probs])
    with pytest.raises(ffca.FFCAError):
        ffca.FastFCABatch(y, v, lam, P, Ns, offsets=[0, 10, int(off[-1])])  # not a multiple of 4
    with pytest.raises(ffca.FFCAError):
        ffca.FastFCABatch(y, v, lam, P, [13, 20], offsets=off)  # mixture 0 overruns its rows
    est = ffca.FastFCABatch(y, v, lam, P, Ns)
    dv = torch.zeros_like(v)
    dl = torch.empty_like(lam)
    dP = torch.empty_like(P)
    with pytest.raises(ffca.FFCAError) as ei:  # gradient outputs must be 16-byte aligned
        ffca.ffca_nll_grad(est.ctx, dv.data_ptr() + 4, dl.data_ptr(), dP.data_ptr())
    assert ei.value.status == 1
    est.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_autotune_iterations_are_iterations(prec):
    """ffca_batch_autotune runs real hybrid iterations (one per candidate
    partition); with two more ordinary iterations the state equals the
    oracle's after the same total number of iterations."""
    import torch
    from paper_1805_09498_gb300 import ffca
    probs = make_batch(4, 3, 5, [300, 41, 1200, 96, 700], seed=13)
    n_auto = ffca.ffca_batch_config_count()
    refs = [ffa.iterate(p.y, p.v0, p.lam0, p.P0, n_auto + 2, counter=OpCounter()) for p in probs]
    y, v, lam, P, Ns, off = ffca.batch_to_device([p.y for p in probs], [p.v0 for p in probs],
                                                 [p.lam0 for p in probs], [p.P0 for p in probs], prec=prec)
    est = ffca.FastFCABatch(y, v, lam, P, Ns)
    ca, cb, ma, mb = est.autotune(rounds=1)
    assert 0 <= ca < n_auto and 0 <= cb < n_auto and all(t > 0 for t in ma + mb)
    est.iterate(2, trace=False)
    ll = est.loglik()
    torch.cuda.synchronize()
    vh = v.double().cpu()
    got = dict(v=[b[:, :, :Ns[m]].numpy() for m, b in enumerate(ffca.batch_views(vh, 3, 5, off))],
               lam=lam.cpu().numpy(), P=P.cpu().numpy(), ll=ll,
               trace=np.sum([r[3] for r in refs], axis=0))  # no trace from the tuning run
    _check(prec, probs, refs, got)
    est.close()


def test_fixed_config_is_reproducible():
    """Every candidate partition gives the oracle's result; a fixed candidate
    gives the same bits on every run."""
    import torch
    from paper_1805_09498_gb300 import ffca
    probs = make_batch(3, 3, 4, [150, 900, 33], seed=14)
    refs = [ffa.iterate(p.y, p.v0, p.lam0, p.P0, 3, counter=OpCounter()) for p in probs]
    outs = {}
    for cand in range(ffca.ffca_batch_config_count()):
        for rep in range(2 if cand == 3 else 1):
            y, v, lam, P, Ns, off = ffca.batch_to_device([p.y for p in probs], [p.v0 for p in probs],
                                                         [p.lam0 for p in probs], [p.P0 for p in probs])
            est = ffca.FastFCABatch(y, v, lam, P, Ns)
            est.set_config(cand, cand)
            tr = est.iterate(3)
            ll = est.loglik()
            torch.cuda.synchronize()
            vh = v.double().cpu()
            got = dict(v=[b[:, :, :Ns[m]].numpy() for m, b in enumerate(ffca.batch_views(vh, 3, 4, off))],
                       lam=lam.cpu().numpy(), P=P.cpu().numpy(), ll=ll, trace=tr)
            _check("mixed", probs, refs, got)
            outs.setdefault(cand, []).append((vh.numpy(), got["lam"], got["P"]))
            est.close()
    a, b = outs[3]
    assert all(np.array_equal(x, z) for x, z in zip(a, b))


@pytest.mark.parametrize("prec,I", [("mixed", 3), ("fp64", 3), ("mixed", 4), ("mixed", 8)])
def test_batch_wiener_matches_oracle(prec, I):
    """The Wiener filter of a batch context (Eq. MMSE0 per mixture): each
    mixture's block equals the oracle's filter of that mixture after the same
    iterations, the images sum to the mixture, and padding frames are zero."""
    import torch
    from paper_1805_09498_gb300 import ffca
    J = 6 if I == 8 else 3
    kw = dict(alpha=0.2, kappa=50.0) if I == 8 else {}
    probs = make_batch(I, J, 4, [37, 203, 8, 130], seed=12, **kw)
    y, v, lam, P, Ns, off = ffca.batch_to_device([p.y for p in probs], [p.v0 for p in probs],
                                                 [p.lam0 for p in probs], [p.P0 for p in probs],
                                                 prec=prec)
    est = ffca.FastFCABatch(y, v, lam, P, Ns)
    est.iterate(2, trace=False)
    out = est.wiener()
    torch.cuda.synchronize()
    tol = TOL[prec]["par"]
    vh = ffca.batch_views(v.double().cpu(), J, 4, off)
    for m, (p, blk) in enumerate(zip(probs, ffca.batch_views(out.cpu(), J * I, 4, off))):
        n = int(Ns[m])
        xh = blk.view(J, I, 4, -1).numpy()
        ref = ffa.wiener(p.y, vh[m][:, :, :n].numpy(), lam[m].cpu().numpy(), P[m].cpu().numpy())
        assert per_f_relerr(xh[..., :n], ref, 2) <= tol, m
        assert per_f_relerr(xh[..., :n].sum(axis=0), p.y, 1) <= tol, m
        assert np.all(xh[..., n:] == 0), m
    est.close()
