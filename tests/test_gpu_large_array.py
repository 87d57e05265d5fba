"""GPU parity of the FastFCA-AS path at I = 8 microphones (the large-array
workload: J = 6, P(f) = I + 0.2 G with cond < 50), where pass A reads P and
Lambda from the stage, pass B splits the I^3 sums per point over threads,
and the per-problem FP64 step uses elimination and Cholesky solves.

Tolerances as for the small arrays: FP64 1e-9, mixed 1e-4 on parameters
(normwise per frequency) and 1e-5 per point on L2.
"""
import numpy as np
import pytest

from oracle import fastfca_as as ffa
from oracle.fastfca_as import OpCounter
from paper_1805_09498_gb300.synth import make_problem

from helpers import per_f_relerr, run_gpu

pytestmark = pytest.mark.gpu


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
    e = dict(v=per_f_relerr(v_g, v_r, 1), lam=per_f_relerr(l_g, l_r, 0), P=per_f_relerr(P_g, P_r, 0))
    par = 1e-9 if prec == "fp64" else 1e-4
    for k, x in e.items():
        assert x <= par, (k, x, e)
    if prec == "fp64":
        assert np.all(np.abs(t_g - t_r) <= 1e-9 * np.abs(t_r)), (t_g, t_r)
    else:
        assert np.all(np.abs(t_g - t_r) <= 1e-5 * N * F), (t_g - t_r) / (N * F)
    return e


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(8, 6, 3, 50), (8, 2, 2, 37), (8, 6, 4, 1030), (8, 1, 2, 64)])
def test_one_iteration_matches_oracle(prec, shape):
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=500 + J, alpha=0.2, kappa=50.0)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 1, counter=OpCounter())
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 1, prec)
    _compare(prec, ref, got, N, F)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_trajectory_large_array(prec):
    """10 iterations at the large-array shape (I = 8, J = 6, N = 4000) on 6
    frequencies, K = 2 sweeps in the last check."""
    p = make_problem(8, 6, 6, 4000, seed=3, alpha=0.2, kappa=50.0)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 10, counter=OpCounter())
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 10, prec)
    _compare(prec, ref, got, 4000, 6)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, K=2, counter=OpCounter())
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 2, prec, K=2)
    _compare(prec, ref, got, 4000, 6)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_resumable_bit_exact_large_array(prec):
    """2 + 2 iterations in two calls equal 4 in one, bit for bit: the P^{-H}
    that the fixed-point step carries to the next step (one warp per problem
    at I = 8) has the bits of the one a call recomputes from P at its start."""
    p = make_problem(8, 6, 5, 300, seed=21, alpha=0.2, kappa=50.0)
    a = run_gpu(p.y, p.v0, p.lam0, p.P0, 4, prec)
    b1 = run_gpu(p.y, p.v0, p.lam0, p.P0, 2, prec)
    b = run_gpu(p.y, b1[0], b1[1], b1[2], 2, prec)
    for x, z in zip(a[:3], b[:3]):
        assert np.array_equal(x, z)
    assert np.array_equal(a[3][2:], b[3])


@pytest.mark.parametrize("F", [1536, 1537])
@pytest.mark.parametrize("p_update", [None, "em"])
def test_p_step_forms_either_side_of_the_switch_large_array(F, p_update):
    """At I = 8 the fixed-point and EM steps run one warp per problem up to
    1536 problems and pack four in a warp above: both against the oracle."""
    p = make_problem(8, 6, F, 12, seed=16, alpha=0.2, kappa=50.0)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 1, counter=OpCounter(), p_update=p_update or "fpi")
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 1, "fp64", p_update=p_update)
    _compare("fp64", ref, got, 12, F)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_loglik_and_wiener_large_array(prec):
    import torch
    from paper_1805_09498_gb300 import ffca
    p = make_problem(8, 6, 3, 203, seed=8, alpha=0.2, kappa=50.0)
    yd, vd, lam_d, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=prec)
    est = ffca.FastFCA(yd, vd, lam_d, Pd, N=N)
    L = est.loglik()
    L_ref = ffa.loglik(p.y, p.v0, p.lam0, p.P0)
    xh = est.wiener()
    torch.cuda.synchronize()
    xh = xh.cpu().numpy()
    ref = ffa.wiener(p.y, p.v0, p.lam0, p.P0)
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert abs(L - L_ref) <= (1e-9 * abs(L_ref) if prec == "fp64" else 1e-5 * N * 3)
    assert per_f_relerr(xh[:, :, :, :N], ref, 2) <= tol
    assert per_f_relerr(xh[:, :, :, :N].sum(axis=0), p.y, 1) <= tol
    est.close()


def test_singular_bin_is_reported_large_array():
    from paper_1805_09498_gb300 import ffca
    p = make_problem(8, 3, 4, 40, seed=6, alpha=0.2, kappa=50.0)
    p.y[:, 2, :] = 0.0
    with pytest.raises(ffca.FFCAError) as ei:
        run_gpu(p.y, p.v0, p.lam0, p.P0, 1, "fp64")
    assert ei.value.status == 4 and ei.value.frequency == 2


def test_batch_of_large_arrays():
    """The batch path at I = 8: three mixtures of uneven length."""
    from paper_1805_09498_gb300.synth import make_batch
    from test_gpu_batch import _check, _run_batch
    probs = make_batch(8, 6, 3, [57, 400, 130], seed=9, alpha=0.2, kappa=50.0)
    refs = [ffa.iterate(q.y, q.v0, q.lam0, q.P0, 2, counter=OpCounter()) for q in probs]
    _check("mixed", probs, refs, _run_batch(probs, 2, "mixed"))


def test_full_size_large_array_sampled():
    """I = 8, J = 6, F = 513, N = 4000 (the large-array workload), mixed, 30
    iterations; 6 sampled frequencies checked against the oracle run on them."""
    from paper_1805_09498_gb300 import ffca
    import torch
    I, J, F, N, it = 8, 6, 513, 4000, 30
    p = make_problem(I, J, F, N, seed=1, alpha=0.2, kappa=50.0)
    yd, vd, lam_d, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="mixed")
    est = ffca.FastFCA(yd, vd, lam_d, Pd, N=N)
    tr = est.iterate(it)
    torch.cuda.synchronize()
    fs = np.array([0, 100, 255, 256, 400, 512])
    ref = ffa.iterate(p.y[:, fs], p.v0[:, fs], p.lam0[fs], p.P0[fs], it, counter=OpCounter())
    got = (vd[:, fs, :N].double().cpu().numpy(), lam_d[fs].cpu().numpy(), Pd[fs].cpu().numpy(), None)
    e = dict(v=per_f_relerr(got[0], ref[0], 1), lam=per_f_relerr(got[1], ref[1], 0),
             P=per_f_relerr(got[2], ref[2], 0))
    assert max(e.values()) <= 1e-4, e
    assert np.all(np.isfinite(tr)) and tr[-1] > tr[0]
    est.close()
