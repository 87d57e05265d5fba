"""GPU parity of the resident form of the hybrid iterations (ffca_set_resident:
one CTA per problem keeps y and v in shared memory for up to 32 iterations
of one launch) against the FP64 CPU oracle, for single mixtures and ragged
batches, and against the streaming kernels on the same inputs.

Tolerances as for the streaming path (normwise relative error per frequency):
    FP64 path:  1e-9 on v, Lambda, P and on L2
    mixed path: 1e-4 on v, Lambda, P; |dL2| / (N F) <= 1e-5 nats per point
"""
import numpy as np
import pytest

from oracle import fastfca_as as ffa
from oracle.fastfca_as import OpCounter
from paper_1805_09498_gb300.synth import make_batch, make_problem

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


def _run(p, iters, prec, K=1, ld=None, pad_value=None, resident=True, graph=False, trace=True):
    import torch
    from paper_1805_09498_gb300 import ffca
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=prec, ld=ld)
    if pad_value is not None and yd.shape[2] > N:
        yd[:, :, N:] = pad_value
        vd[:, :, N:] = pad_value
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N, K=K)
    if resident:
        est.set_resident(True)
    if graph:
        est.set_graph(True)
    ffca.ffca_timing_read(est.ctx)
    tr = est.iterate(iters, trace=trace)
    counts = ffca.ffca_timing_read(est.ctx)
    inv = est.inversion_count()
    torch.cuda.synchronize()
    out = dict(v=vd[:, :, :N].double().cpu().numpy(), lam=ld_.cpu().numpy(), P=Pd.cpu().numpy(), trace=tr,
               counts=counts, inv=inv, vpad=vd[:, :, N:].double().cpu().numpy())
    est.close()
    return out


def _compare(prec, ref, got, N, F, trace=True):
    v_r, l_r, P_r, t_r = ref
    e = dict(v=per_f_relerr(got["v"], v_r, 1), lam=per_f_relerr(got["lam"], l_r, 0),
             P=per_f_relerr(got["P"], P_r, 0))
    tol = TOL[prec]
    for k, x in e.items():
        assert x <= tol["par"], (k, x, e)
    if trace:
        t_g = got["trace"]
        if prec == "fp64":
            assert np.all(np.abs(t_g - t_r) <= tol["ll_rel"] * np.abs(t_r)), (t_g, t_r)
        else:
            assert np.all(np.abs(t_g - t_r) <= tol["ll_tf"] * N * F), (t_g - t_r) / (N * F)
    return e


SHAPES = [(3, 3, 5, 37), (2, 3, 4, 50), (1, 2, 3, 17), (4, 2, 3, 41), (3, 1, 2, 33), (2, 4, 3, 29),
          (4, 3, 7, 301), (3, 3, 3, 1030), (3, 6, 2, 123), (4, 6, 2, 257), (2, 5, 3, 64), (8, 6, 2, 300),
          (8, 3, 3, 150)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", SHAPES)
def test_matches_oracle(prec, shape):
    """Three iterations in one launch, every compiled I <= 4 and J, frames
    below one CTA's threads, ragged against 256 and several times it."""
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=300 + I * 10 + J)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 3, counter=OpCounter())
    got = _run(p, 3, prec)
    _compare(prec, ref, got, N, F)
    assert got["counts"]["resident"][1] == 1 and got["counts"]["estep"][1] == 0
    assert got["inv"] == (I + 1) * F * 3


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_plain_workload_across_launches(prec):
    """The plain FP64 workload's shape (I = J = 3, F = 257, N = 600) for 40
    iterations: two launches (32 + 8) with the trace of every iteration."""
    p = make_problem(3, 3, 257, 600, seed=0)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 40, counter=OpCounter())
    got = _run(p, 40, prec)
    _compare(prec, ref, got, 600, 257)
    assert got["counts"]["resident"][1] == 2
    assert got["trace"][-1] > got["trace"][0]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_k_sweeps_and_padding(prec):
    """K = 3 fixed-point sweeps; NaN in the padding frames is not read and
    not written."""
    p = make_problem(3, 3, 6, 257, seed=5)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, K=3, counter=OpCounter())
    got = _run(p, 2, prec, K=3, ld=268, pad_value=float("nan"))
    _compare(prec, ref, got, 257, 6)
    assert np.all(np.isnan(got["vpad"]))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_close_to_streaming(prec):
    """The resident and streaming forms agree to the order of their sums."""
    p = make_problem(4, 3, 9, 2000, seed=12)
    a = _run(p, 10, prec)
    b = _run(p, 10, prec, resident=False)
    tol = 1e-11 if prec == "fp64" else 1e-4
    for k, ax in (("v", 1), ("lam", 0), ("P", 0)):
        assert per_f_relerr(a[k], b[k], ax) <= tol, k
    assert np.max(np.abs(a["trace"] - b["trace"]) / np.abs(b["trace"])) <= tol


def test_graph_replay_is_bit_exact():
    """Trace-less calls replayed from a captured graph give the launches'
    results bit for bit."""
    p = make_problem(3, 3, 8, 400, seed=13)
    a = _run(p, 35, "mixed", trace=False)
    b = _run(p, 35, "mixed", trace=False, graph=True)
    for k in ("v", "lam", "P"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_oracle(prec):
    """A ragged batch (5 to 1500 frames) with each problem resident, against
    the oracle per mixture; the trace is the sum of the mixtures' traces.

    The 5-frame mixture at I = 4 ends with cond(P) up to 160, where a
    relative change of 1e-6 in P moves its L2 by about 1e-2: in the mixed
    path its L2 is checked as the oracle's L2 of the GPU's own final state
    (the evaluation's accuracy) rather than against the oracle's trajectory."""
    import torch
    from paper_1805_09498_gb300 import ffca
    I, J, F = 4, 3, 5
    Ns = [37, 200, 5, 1500, 129, 64, 8, 301]
    probs = make_batch(I, J, F, Ns, seed=77)
    y, v, lam, P, Ns_, off = ffca.batch_to_device([q.y for q in probs], [q.v0 for q in probs],
                                                  [q.lam0 for q in probs], [q.P0 for q in probs], prec=prec)
    est = ffca.FastFCABatch(y, v, lam, P, Ns_)
    est.set_resident(True)
    tr = est.iterate(4)
    ll = est.loglik()
    torch.cuda.synchronize()
    vv = ffca.batch_views(v.double().cpu(), J, F, off)
    yv = ffca.batch_views(y.cpu(), I, F, off)
    refs = [ffa.iterate(q.y, q.v0, q.lam0, q.P0, 4, counter=OpCounter()) for q in probs]
    tol = TOL[prec]
    for m, (q, r) in enumerate(zip(probs, refs)):
        e = dict(v=per_f_relerr(vv[m][:, :, :q.N].numpy(), r[0], 1), lam=per_f_relerr(lam[m].cpu().numpy(), r[1], 0),
                 P=per_f_relerr(P[m].cpu().numpy(), r[2], 0))
        assert max(e.values()) <= tol["par"], (m, e)
        if prec == "fp64":
            ll_ref = ffa.loglik(q.y, r[0], r[1], r[2])
            bound = tol["ll_rel"] * abs(ll_ref)
        else:
            ll_ref = ffa.loglik(yv[m][:, :, :q.N].numpy().astype(np.complex128), vv[m][:, :, :q.N].numpy(),
                                lam[m].cpu().numpy(), P[m].cpu().numpy())
            bound = tol["ll_tf"] * q.N * F
        assert abs(ll[m] - ll_ref) <= bound, (m, ll[m], ll_ref)
    t_ref = np.sum([r[3] for r in refs], axis=0)
    NF = sum(q.N * F for q in probs)
    bound = tol["ll_rel"] * np.abs(t_ref) if prec == "fp64" else tol["ll_tf"] * NF
    assert np.all(np.abs(tr - t_ref) <= bound)
    est.close()


def test_unsupported_forms():
    """A problem longer than the shared memory holds is refused and the
    context keeps streaming; another update of P streams."""
    from paper_1805_09498_gb300 import ffca
    p = make_problem(8, 6, 2, 2400, seed=8, alpha=0.2, kappa=50.0)
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="mixed")
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N)
    with pytest.raises(ffca.FFCAError) as e:
        est.set_resident(True)
    assert e.value.status == 7
    est.close()
    p = make_problem(3, 3, 2, 6000, seed=9)
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="mixed")
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N)
    with pytest.raises(ffca.FFCAError) as e:
        est.set_resident(True)
    assert e.value.status == 7
    tr = est.iterate(2)
    assert np.all(np.isfinite(tr))
    est.close()
    p = make_problem(3, 3, 4, 300, seed=10)
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="mixed")
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N)
    est.set_resident(True)
    est.set_p_update("em")
    ffca.ffca_timing_read(est.ctx)
    est.iterate(2, trace=False)
    c = ffca.ffca_timing_read(est.ctx)
    assert c["resident"][1] == 0 and c["estep"][1] == 2
    est.close()


@pytest.mark.parametrize("I", [3, 8])
def test_singular_bin_is_reported(I):
    """A frequency whose mixture is all zeros has singular V_i: the resident
    form reports FFCA_ERR_SINGULAR at that frequency, as the streaming one
    does."""
    from paper_1805_09498_gb300 import ffca
    kw = dict(alpha=0.2, kappa=50.0) if I == 8 else {}
    p = make_problem(I, 3, 4, 60, seed=16, **kw)
    p.y[:, 2, :] = 0.0
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="fp64")
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N)
    est.set_resident(True)
    with pytest.raises(ffca.FFCAError) as ei:
        est.iterate(1)
    assert ei.value.status == 4 and ei.value.frequency == 2
    est.close()


@pytest.mark.parametrize("prec,N", [("mixed", 5688), ("fp64", 2844)])
def test_largest_problem_that_fits(prec, N):
    """The longest problem the shared memory holds at I = J = 3 (200 KB at
    36 bytes per frame in the mixed precision, 72 in FP64), two iterations,
    against the oracle; one frame more is refused."""
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 3, 2, N, seed=17)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, counter=OpCounter())
    got = _run(p, 2, prec)
    _compare(prec, ref, got, N, 2)
    assert got["counts"]["resident"][1] == 1
    q = make_problem(3, 3, 2, N + 1, seed=17)
    yd, vd, ld_, Pd, n1 = ffca.to_device(q.y, q.v0, q.lam0, q.P0, prec=prec)
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=n1)
    with pytest.raises(ffca.FFCAError) as e:
        est.set_resident(True)
    assert e.value.status == 7
    est.close()
