"""GPU parity of the FastFCA-AS path (called through the C ABI) against the
FP64 CPU oracle on the same seeded inputs.

Tolerances (normwise relative error per frequency, max over f):
    FP64 path:  1e-9 on v, Lambda, P and on L2
    mixed path: 1e-4 on v, Lambda, P; |dL2| / (N F) <= 1e-5 nats per point
"""
import numpy as np
import pytest

from oracle import fastfca_as as ffa
from oracle.fastfca_as import OpCounter
from paper_1805_09498_gb300.synth import make_problem

from helpers import per_f_relerr, run_gpu

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(par=1e-9, ll_rel=1e-9), "mixed": dict(par=1e-4, ll_tf=1e-5)}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1805_09498_gb300 import build
    build.build()


def _compare(prec, ref, got, N, F):
    v_r, l_r, P_r, t_r = ref
    v_g, l_g, P_g, t_g = got
    e = dict(v=per_f_relerr(v_g, v_r, 1), lam=per_f_relerr(l_g, l_r, 0),
             P=per_f_relerr(P_g, P_r, 0))
    tol = TOL[prec]
    for k, x in e.items():
        assert x <= tol["par"], (k, x, e)
    if prec == "fp64":
        assert np.all(np.abs(t_g - t_r) <= tol["ll_rel"] * np.abs(t_r)), (t_g, t_r)
    else:
        assert np.all(np.abs(t_g - t_r) <= tol["ll_tf"] * N * F), (t_g - t_r) / (N * F)
    return e


SMALL = [(3, 3, 5, 37), (2, 3, 4, 50), (1, 2, 3, 17), (4, 2, 3, 41), (3, 1, 2, 33),
         (2, 4, 3, 29), (4, 3, 7, 301), (3, 3, 3, 1030), (3, 6, 2, 123), (2, 5, 3, 64)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", SMALL)
def test_one_iteration_matches_oracle(prec, shape):
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=100 + I * 10 + J)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 1, counter=OpCounter())
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 1, prec)
    _compare(prec, ref, got, N, F)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_trajectory_plain_config(prec):
    """20 iterations at I = J = 3, F = 257, N = 600 (the plain FP64 workload)."""
    p = make_problem(3, 3, 257, 600, seed=0)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 20, counter=OpCounter())
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 20, prec)
    _compare(prec, ref, got, 600, 257)
    # the trace is a log-likelihood trajectory that rises overall
    assert got[3][-1] > got[3][0]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_k_sweeps(prec):
    """K = 3 fixed-point sweeps per iteration (Sec. 4.5's K)."""
    p = make_problem(3, 3, 6, 257, seed=5)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, K=3, counter=OpCounter())
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 2, prec, K=3)
    _compare(prec, ref, got, 257, 6)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_padding_is_ignored(prec):
    """Frames beyond N (ld > N) may hold anything, NaN included."""
    p = make_problem(3, 3, 4, 45, seed=6)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, counter=OpCounter())
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 2, prec, ld=52, pad_value=float("nan"))
    _compare(prec, ref, got, 45, 4)


def test_long_mixed_trajectory():
    """50 mixed-precision iterations at a longer N stay within tolerance."""
    p = make_problem(3, 3, 9, 5000, seed=7)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 50, counter=OpCounter())
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 50, "mixed")
    _compare("mixed", ref, got, 5000, 9)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_loglik_and_wiener(prec):
    import torch
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 3, 5, 203, seed=8)
    yd, vd, lam_d, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=prec)
    est = ffca.FastFCA(yd, vd, lam_d, Pd, N=N)
    L = est.loglik()
    L_ref = ffa.loglik(p.y, p.v0, p.lam0, p.P0)
    xh = est.wiener()
    torch.cuda.synchronize()
    xh = xh.cpu().numpy()
    ref = ffa.wiener(p.y, p.v0, p.lam0, p.P0)
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert abs(L - L_ref) <= (1e-9 * abs(L_ref) if prec == "fp64" else 1e-5 * N * 5)
    assert per_f_relerr(xh[:, :, :, :N], ref, 2) <= tol
    # the J estimates sum to the mixture; padding frames are zero
    assert per_f_relerr(xh[:, :, :, :N].sum(axis=0), p.y, 1) <= tol
    assert np.all(xh[:, :, :, N:] == 0)
    est.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_inversion_count(prec):
    """(I+1) F K small inversions per iteration (Sec. 4.5)."""
    from paper_1805_09498_gb300 import ffca
    I, J, F, N, K, it = 3, 3, 7, 64, 2, 3
    p = make_problem(I, J, F, N, seed=9)
    yd, vd, lam_d, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=prec)
    est = ffca.FastFCA(yd, vd, lam_d, Pd, N=N, K=K)
    est.iterate(it, trace=False)
    assert est.inversion_count() == (I + 1) * F * K * it
    est.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_deterministic_and_resumable(prec):
    """Fixed-order reductions: 3 + 3 iterations in two calls equal 6 in one,
    bit for bit, and a rerun reproduces them."""
    p = make_problem(3, 3, 6, 777, seed=10)
    a = run_gpu(p.y, p.v0, p.lam0, p.P0, 6, prec)
    b1 = run_gpu(p.y, p.v0, p.lam0, p.P0, 3, prec)
    b = run_gpu(p.y, b1[0], b1[1], b1[2], 3, prec)
    c = run_gpu(p.y, p.v0, p.lam0, p.P0, 6, prec)
    for x, z in zip(a[:3], c[:3]):
        assert np.array_equal(x, z)
    assert np.array_equal(a[3], c[3])
    for x, z in zip(a[:3], b[:3]):
        assert np.array_equal(x, z)
    assert np.array_equal(a[3][3:], b[3])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("F", [768, 769])
@pytest.mark.parametrize("p_update", [None, "em"])
def test_p_step_forms_either_side_of_the_switch(prec, F, p_update):
    """The fixed-point and EM steps run one warp per problem up to 768
    problems at I = 3 and pack ten problems in a warp above: both forms
    against the oracle over two iterations, and 2 + 1 iterations equal 3 bit
    for bit."""
    p = make_problem(3, 3, F, 24, seed=15)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, counter=OpCounter(), p_update=p_update or "fpi")
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 2, prec, p_update=p_update)
    _compare(prec, ref, got, 24, F)
    a = run_gpu(p.y, p.v0, p.lam0, p.P0, 3, prec, p_update=p_update)
    b = run_gpu(p.y, got[0], got[1], got[2], 1, prec, p_update=p_update)
    for x, z in zip(a[:3], b[:3]):
        assert np.array_equal(x, z)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("p_update,mu", [(None, 0.0), ("gradient", 0.05), ("em", 0.0)])
def test_resumable_bit_exact_i4(prec, p_update, mu):
    """I = 4: 2 + 2 iterations in two calls equal 4 in one, bit for bit.  The
    P^{-H} that a step carries (one warp per problem for the fixed point and
    the EM, four problems per warp for the gradient) has the bits of the one
    that the next call's prep (one warp per problem) forms from P."""
    p = make_problem(4, 3, 7, 150, seed=17)
    a = run_gpu(p.y, p.v0, p.lam0, p.P0, 4, prec, p_update=p_update, mu=mu)
    b1 = run_gpu(p.y, p.v0, p.lam0, p.P0, 2, prec, p_update=p_update, mu=mu)
    b = run_gpu(p.y, b1[0], b1[1], b1[2], 2, prec, p_update=p_update, mu=mu)
    for x, z in zip(a[:3], b[:3]):
        assert np.array_equal(x, z)
    assert np.array_equal(a[3][2:], b[3])


@pytest.mark.parametrize("F", [1024, 1025])
@pytest.mark.parametrize("p_update", [None, "em"])
def test_p_step_forms_either_side_of_the_switch_i4(F, p_update):
    """At I = 4 the fixed-point step, the EM step and prep run one warp per
    problem up to 1024 problems and pack eight in a warp above: both
    against the oracle."""
    p = make_problem(4, 3, F, 12, seed=18)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 1, counter=OpCounter(), p_update=p_update or "fpi")
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 1, "fp64", p_update=p_update)
    _compare("fp64", ref, got, 12, F)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("p_update", [None, "em"])
def test_traced_graph_replay_is_bit_exact(prec, p_update):
    """iterate() with a trace replayed from a CUDA graph gives the state and
    the trace of the plain launches bit for bit, on the first replay (the
    capture) and on a later one; the cached graph without a trace is kept
    apart from the traced one."""
    import torch
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 3, 6, 300, seed=14)
    outs = []
    for graph in (False, True):
        yd, vd, lam_d, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=prec)
        est = ffca.FastFCA(yd, vd, lam_d, Pd, N=N)
        if p_update is not None:
            est.set_p_update(p_update)
        est.set_graph(graph)
        t1 = est.iterate(3)
        est.iterate(2, trace=False)
        t2 = est.iterate(3)
        torch.cuda.synchronize()
        outs.append((vd.cpu().numpy(), lam_d.cpu().numpy(), Pd.cpu().numpy(), t1, t2))
        est.close()
    for x, z in zip(outs[0], outs[1]):
        assert np.array_equal(x, z)


def test_resume_mixed_in_place():
    """Mixed path: resuming from the device state is bitwise equal too."""
    import torch
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 3, 6, 777, seed=10)
    outs = []
    for split in (None, 3):
        yd, vd, lam_d, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="mixed")
        est = ffca.FastFCA(yd, vd, lam_d, Pd, N=N)
        if split is None:
            tr = est.iterate(6)
        else:
            t1 = est.iterate(split)
            est.close()
            est = ffca.FastFCA(yd, vd, lam_d, Pd, N=N)   # a fresh context on the saved state
            t2 = est.iterate(6 - split)
            tr = np.concatenate([t1[:-1], t2])
        torch.cuda.synchronize()
        outs.append((vd.cpu().numpy(), lam_d.cpu().numpy(), Pd.cpu().numpy(), tr))
        est.close()
    for x, z in zip(outs[0], outs[1]):
        assert np.array_equal(x, z)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_zero_frequency_is_singular(prec):
    """y(., f) = 0 makes every V_i(f) zero: the P update reports
    FFCA_ERR_SINGULAR at that frequency instead of producing garbage."""
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 3, 4, 40, seed=11)
    y = p.y.copy()
    y[:, 2, :] = 0
    yd, vd, lam_d, Pd, N = ffca.to_device(y, p.v0, p.lam0, p.P0, prec=prec)
    est = ffca.FastFCA(yd, vd, lam_d, Pd, N=N)
    with pytest.raises(ffca.FFCAError) as ei:
        est.iterate(1)
    assert ei.value.status == 4 and ei.value.frequency == 2
    est.close()


def test_fewer_frames_than_mics_is_singular():
    """N < I: V_i has rank N < I (FP64 path detects it)."""
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 2, 3, 2, seed=12)
    yd, vd, lam_d, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="fp64")
    est = ffca.FastFCA(yd, vd, lam_d, Pd, N=N)
    with pytest.raises(ffca.FFCAError) as ei:
        est.iterate(1)
    assert ei.value.status == 4
    est.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nonfinite_input_is_reported(prec):
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 3, 5, 60, seed=13)
    v = p.v0.copy()
    v[1, 3, 17] = np.nan
    yd, vd, lam_d, Pd, N = ffca.to_device(p.y, v, p.lam0, p.P0, prec=prec)
    est = ffca.FastFCA(yd, vd, lam_d, Pd, N=N)
    with pytest.raises(ffca.FFCAError) as ei:
        est.iterate(1)
    assert ei.value.status == 3 and ei.value.frequency == 3
    est.close()


def test_empty_frequency_axis():
    import torch
    from paper_1805_09498_gb300 import ffca
    y = torch.zeros((3, 0, 8), dtype=torch.complex64, device="cuda")
    v = torch.zeros((3, 0, 8), dtype=torch.float32, device="cuda")
    lam = torch.zeros((0, 3, 3), dtype=torch.float64, device="cuda")
    P = torch.zeros((0, 3, 3), dtype=torch.complex128, device="cuda")
    est = ffca.FastFCA(y, v, lam, P, N=5)
    assert np.array_equal(est.iterate(3), np.zeros(4))
    assert est.loglik() == 0.0
    est.close()


def test_full_size_long_mixture_sampled():
    """I = J = 3, F = 513, N = 20000 in the benchmark's launch configuration:
    one iteration; frequencies are independent, so the oracle checks a sample
    of them exactly, and L2 of the entering state over all of them."""
    p = make_problem(3, 3, 513, 20000, seed=0)
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 1, "mixed")
    fs = np.array([0, 1, 77, 256, 300, 411, 511, 512])
    ref = ffa.iterate(p.y[:, fs], p.v0[:, fs], p.lam0[fs], p.P0[fs], 1, counter=OpCounter())
    e = dict(v=per_f_relerr(got[0][:, fs], ref[0], 1), lam=per_f_relerr(got[1][fs], ref[1], 0),
             P=per_f_relerr(got[2][fs], ref[2], 0))
    assert max(e.values()) <= 1e-4, e
    L0 = sum(ffa.loglik(p.y[:, s], p.v0[:, s], p.lam0[s], p.P0[s])
             for s in np.array_split(np.arange(513), 16))
    assert abs(got[3][0] - L0) <= 1e-5 * 513 * 20000
