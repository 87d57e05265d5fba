"""GPU parity of the alternative updates of P (Sec. 4.6: the gradient and
natural gradient methods, the normal EM and Newton's method,
ffca_set_p_update) against the
FP64 oracle, for single mixtures at every compiled I, with K > 1 steps, on
batches and under graph replay; the inversion counts and the argument checks.

Tolerances as for the fixed point (normwise relative error per frequency,
max over f): FP64 1e-9 on v, Lambda, P and L2; mixed 1e-4 on the
parameters and 1e-5 nats per point on L2.
"""
import numpy as np
import pytest

from oracle import fastfca_as as ffa
from oracle.fastfca_as import OpCounter
from paper_1805_09498_gb300.synth import make_batch, make_problem

from helpers import per_f_relerr, run_gpu

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(par=1e-9, ll_rel=1e-9), "mixed": dict(par=1e-4, ll_tf=1e-5)}
STEP = {"gradient": 0.05, "natural_gradient": 0.2}


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
    for k, x in e.items():
        assert x <= TOL[prec]["par"], (k, x, e)
    if prec == "fp64":
        assert np.all(np.abs(t_g - t_r) <= TOL[prec]["ll_rel"] * np.abs(t_r)), (t_g, t_r)
    else:
        assert np.all(np.abs(t_g - t_r) <= TOL[prec]["ll_tf"] * N * F), (t_g - t_r) / (N * F)


SHAPES = [(1, 2, 3, 41), (2, 3, 4, 50), (3, 3, 5, 137), (4, 3, 3, 301), (3, 6, 2, 123), (8, 6, 3, 260)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("method", ["gradient", "natural_gradient"])
@pytest.mark.parametrize("shape", SHAPES)
def test_iterations_match_oracle(prec, method, shape):
    """Three hybrid iterations with K = 1, from the perturbed truth."""
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=200 + 10 * I + J)
    mu = STEP[method]
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 3, counter=OpCounter(), p_update=method, mu=mu)
    assert np.all(np.diff(ref[3]) > 0)  # an ascent at these step sizes
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 3, prec, p_update=method, mu=mu)
    _compare(prec, ref, got, N, F)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("method", ["gradient", "natural_gradient"])
@pytest.mark.parametrize("I", [2, 3, 8])
def test_several_steps_per_iteration(prec, method, I):
    """K = 3 steps per iteration with V_i fixed (the gradient method forms
    P^{-H} of each intermediate P).  Smaller steps than above: at I = 8 three
    gradient steps of 0.05 overshoot and L2 falls (-7.7e3 to -5.0e4 in two
    iterations), a trajectory that amplifies the rounding of the mixed path."""
    J = 3
    p = make_problem(I, J, 4, 90, seed=300 + I)
    mu = {"gradient": 0.02, "natural_gradient": 0.1}[method]
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, K=3, counter=OpCounter(), p_update=method, mu=mu)
    assert np.all(np.diff(ref[3]) > 0)
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 2, prec, K=3, p_update=method, mu=mu)
    _compare(prec, ref, got, 90, 4)


@pytest.mark.parametrize("method,per_iter", [("gradient", lambda I, K: K), ("natural_gradient", lambda I, K: 0),
                                             ("fixed_point", lambda I, K: (I + 1) * K)])
@pytest.mark.parametrize("I", [2, 4])
def test_inversion_counts(method, per_iter, I):
    import torch
    from paper_1805_09498_gb300 import ffca
    p = make_problem(I, 2, 7, 40, seed=5)
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="mixed")
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N, K=2)
    est.set_p_update(method, 0.1)
    est.iterate(3, trace=False)
    assert est.inversion_count() == 3 * 7 * per_iter(I, 2)
    est.close()


def test_argument_checks_keep_the_previous_update():
    """An unknown method or a step size that is not finite and positive is
    an argument error; the context keeps its update (here the natural
    gradient chosen before)."""
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 3, 4, 60, seed=9)
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="fp64")
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N)
    est.set_p_update("natural_gradient", 0.2)
    L = ffca.lib()
    for method, mu in [(9, 0.1), (-1, 0.1), (1, 0.0), (2, -0.5), (1, float("nan")), (2, float("inf"))]:
        assert L.ffca_set_p_update(est.ctx, method, mu) == 1
    with pytest.raises(ValueError):
        est.set_p_update("bogus", 0.1)
    tr = est.iterate(2)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, counter=OpCounter(), p_update="natural_gradient", mu=0.2)
    got = (vd[:, :, :N].cpu().numpy(), ld_.cpu().numpy(), Pd.cpu().numpy(), tr)
    _compare("fp64", ref, got, N, 4)
    est.close()


def test_switching_drops_the_captured_graph():
    """Graph replays hold their launch arguments: after a change of the
    update the next replay runs the new one.  Two iterations with the fixed
    point (captured, replayed), then two with the gradient method."""
    import torch
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 3, 5, 80, seed=12)
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="fp64")
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N)
    est.set_graph(True)
    est.iterate(2, trace=False)
    est.set_p_update("gradient", 0.05)
    est.iterate(2, trace=False)
    torch.cuda.synchronize()
    v, lam, P, _ = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, counter=OpCounter())
    ref = ffa.iterate(p.y, v, lam, P, 2, counter=OpCounter(), p_update="gradient", mu=0.05)
    got = (vd[:, :, :N].cpu().numpy(), ld_.cpu().numpy(), Pd.cpu().numpy(), ref[3])
    _compare("fp64", ref, got, N, 5)
    est.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("I,J", [(4, 3), (2, 2), (8, 6)])
def test_batch_natural_gradient_matches_oracle(prec, I, J):
    """A ragged batch with the natural gradient, per mixture against the
    oracle."""
    import torch
    from paper_1805_09498_gb300 import ffca
    Ns = [37, 200, 9, 129, 64]
    probs = make_batch(I, J, 3, Ns, seed=70 + I)
    mu = STEP["natural_gradient"]
    refs = [ffa.iterate(q.y, q.v0, q.lam0, q.P0, 3, counter=OpCounter(), p_update="natural_gradient", mu=mu)
            for q in probs]
    y, v, lam, P, Ns_, off = ffca.batch_to_device([q.y for q in probs], [q.v0 for q in probs],
                                                  [q.lam0 for q in probs], [q.P0 for q in probs], prec=prec)
    est = ffca.FastFCABatch(y, v, lam, P, Ns_)
    est.set_p_update("natural_gradient", mu)
    tr = est.iterate(3)
    torch.cuda.synchronize()
    vs = [b[:, :, :Ns_[m]].numpy() for m, b in enumerate(ffca.batch_views(v.double().cpu(), J, 3, off))]
    lam_h, P_h = lam.cpu().numpy(), P.cpu().numpy()
    for m, (q, r) in enumerate(zip(probs, refs)):
        got = (vs[m], lam_h[m], P_h[m], r[3])
        _compare(prec, r, got, q.N, q.F)
    t_ref = np.sum([r[3] for r in refs], axis=0)
    NF = sum(q.N * q.F for q in probs)
    if prec == "fp64":
        assert np.all(np.abs(tr - t_ref) <= 1e-9 * np.abs(t_ref))
    else:
        assert np.all(np.abs(tr - t_ref) <= 1e-5 * NF)
    est.close()


# ------------------------------------------------------------ normal EM
EM_SHAPES = [(1, 2, 3, 41), (2, 3, 4, 50), (3, 3, 5, 137), (4, 3, 3, 301), (3, 6, 2, 123), (2, 1, 3, 77),
             (4, 5, 2, 96), (8, 6, 3, 260), (8, 3, 2, 157), (8, 1, 2, 64)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", EM_SHAPES)
def test_em_iterations_match_oracle(prec, shape):
    """Three iterations of the hybrid with the normal EM update of P (one
    streaming pass per iteration), K = 1, from the perturbed truth; an EM
    step, so L2 does not decrease."""
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=400 + 10 * I + J)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 3, counter=OpCounter(), p_update="em")
    assert np.all(np.diff(ref[3]) >= -1e-9 * np.abs(ref[3][1:]))
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 3, prec, p_update="em")
    _compare(prec, ref, got, N, F)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("I", [2, 3, 4, 8])
def test_em_several_sweeps(prec, I):
    """K = 3 sweeps of the M-step map per iteration (P^{-H} of each
    intermediate P, the W_i of the entering state), on a ragged length with
    NaN in the padding frames."""
    p = make_problem(I, 3, 4, 91, seed=500 + I)
    ref = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, K=3, counter=OpCounter(), p_update="em")
    got = run_gpu(p.y, p.v0, p.lam0, p.P0, 2, prec, K=3, p_update="em", ld=100, pad_value=float("nan"))
    _compare(prec, ref, got, 91, 4)


@pytest.mark.parametrize("I", [2, 4, 8])
def test_em_inversion_count_and_launches(I):
    """(I+1) F K inversions per iteration, as the fixed point; one streaming
    pass per iteration (no pass B launch)."""
    from paper_1805_09498_gb300 import ffca
    p = make_problem(I, 2, 7, 40, seed=6)
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="mixed")
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N, K=2)
    est.set_p_update("em")
    ffca.ffca_timing_read(est.ctx)
    est.iterate(3, trace=False)
    counts = ffca.ffca_timing_read(est.ctx)
    assert est.inversion_count() == 3 * 7 * (I + 1) * 2
    assert counts["estep"][1] == 3 and counts["wcov"][1] == 0 and counts["psolve"][1] == 3
    est.close()


def test_em_graph_replay_and_switch():
    """Two fixed-point iterations, then three EM iterations replayed from a
    captured graph, against the oracle."""
    import torch
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 3, 5, 80, seed=13)
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="fp64")
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N)
    est.set_graph(True)
    est.iterate(2, trace=False)
    est.set_p_update("em")
    est.iterate(3, trace=False)
    torch.cuda.synchronize()
    v, lam, P, _ = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 2, counter=OpCounter())
    ref = ffa.iterate(p.y, v, lam, P, 3, counter=OpCounter(), p_update="em")
    got = (vd[:, :, :N].cpu().numpy(), ld_.cpu().numpy(), Pd.cpu().numpy(), ref[3])
    _compare("fp64", ref, got, N, 5)
    est.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("I,J", [(4, 3), (2, 2), (3, 3), (8, 6)])
def test_batch_em_matches_oracle(prec, I, J):
    """A ragged batch with the normal EM, per mixture against the oracle,
    with the trace (the step's last block sums the problems' L2)."""
    import torch
    from paper_1805_09498_gb300 import ffca
    Ns = [37, 200, 9, 129, 64]
    probs = make_batch(I, J, 3, Ns, seed=90 + I)
    refs = [ffa.iterate(q.y, q.v0, q.lam0, q.P0, 3, counter=OpCounter(), p_update="em") for q in probs]
    y, v, lam, P, Ns_, off = ffca.batch_to_device([q.y for q in probs], [q.v0 for q in probs],
                                                  [q.lam0 for q in probs], [q.P0 for q in probs], prec=prec)
    est = ffca.FastFCABatch(y, v, lam, P, Ns_)
    est.set_p_update("em")
    tr = est.iterate(3)
    torch.cuda.synchronize()
    vs = [b[:, :, :Ns_[m]].numpy() for m, b in enumerate(ffca.batch_views(v.double().cpu(), J, 3, off))]
    lam_h, P_h = lam.cpu().numpy(), P.cpu().numpy()
    for m, (q, r) in enumerate(zip(probs, refs)):
        got = (vs[m], lam_h[m], P_h[m], r[3])
        _compare(prec, r, got, q.N, q.F)
    t_ref = np.sum([r[3] for r in refs], axis=0)
    NF = sum(q.N * q.F for q in probs)
    if prec == "fp64":
        assert np.all(np.abs(tr - t_ref) <= 1e-9 * np.abs(t_ref))
    else:
        assert np.all(np.abs(tr - t_ref) <= 1e-5 * NF)
    est.close()


def test_batch_em_autotune_and_graph():
    """Autotuning with the EM selected times the EM pass on pass A's
    candidates; iterations replayed from a graph afterwards match the oracle
    per mixture (the tuning iterations included)."""
    import torch
    from paper_1805_09498_gb300 import ffca
    Ns = [120, 33, 250]
    probs = make_batch(4, 3, 4, Ns, seed=123)
    y, v, lam, P, Ns_, off = ffca.batch_to_device([q.y for q in probs], [q.v0 for q in probs],
                                                  [q.lam0 for q in probs], [q.P0 for q in probs], prec="fp64")
    est = ffca.FastFCABatch(y, v, lam, P, Ns_, graph=True)
    est.set_p_update("em")
    rounds = 1
    est.autotune(rounds=rounds)
    n_tune = rounds * ffca.lib().ffca_batch_config_count()
    est.iterate(2, trace=False)
    torch.cuda.synchronize()
    vs = [b[:, :, :Ns_[m]].numpy() for m, b in enumerate(ffca.batch_views(v.cpu(), 3, 4, off))]
    for m, q in enumerate(probs):
        r = ffa.iterate(q.y, q.v0, q.lam0, q.P0, n_tune + 2, counter=OpCounter(), p_update="em")
        _compare("fp64", r, (vs[m], lam[m].cpu().numpy(), P[m].cpu().numpy(), r[3]), q.N, q.F)
    est.close()


# ------------------------------------------------------------ Newton's method
def _fpi_then(p, fpi_iters, method, iters, mu, K=1):
    """Oracle: fixed-point iterations to come near a maximum, then `iters`
    iterations with `method` (Newton converges only locally)."""
    v, lam, P, _ = ffa.iterate(p.y, p.v0, p.lam0, p.P0, fpi_iters, counter=OpCounter())
    return (v, lam, P), ffa.iterate(p.y, v, lam, P, iters, K=K, counter=OpCounter(), p_update=method, mu=mu)


def _gpu_from(y, state, iters, prec, method, mu, K=1, N=None):
    return run_gpu(y, *state, iters, prec, K=K, p_update=method, mu=mu)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(1, 2, 3, 41), (2, 3, 4, 150), (3, 3, 5, 237), (4, 3, 3, 301), (3, 6, 2, 223)])
def test_newton_iterations_match_oracle(prec, shape):
    """Six fixed-point iterations (oracle), then three hybrid iterations with
    Newton's method for P (mu = 1) from that state on both sides.  Newton's
    method converges only locally: the cases are ones where the oracle's L2
    rises, so that rounding is not amplified by a diverging step."""
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=600 + 10 * I + J)
    state, ref = _fpi_then(p, 6, "newton", 3, 1.0)
    assert np.all(np.diff(ref[3]) > 0)
    got = _gpu_from(p.y, state, 3, prec, "newton", 1.0)
    _compare(prec, ref, got, N, F)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("I", [2, 3, 4])
def test_newton_several_steps_damped(prec, I):
    """K = 2 damped Newton steps (mu = 0.5) per iteration, after twenty
    fixed-point iterations (at I = 4 six leave the oracle's Newton steps
    lowering L2)."""
    p = make_problem(I, 3, 4, 180, seed=700 + I)
    state, ref = _fpi_then(p, 20, "newton", 2, 0.5, K=2)
    assert np.all(np.diff(ref[3]) > 0)
    got = run_gpu(p.y, *state, 2, prec, K=2, p_update="newton", mu=0.5)
    _compare(prec, ref, got, 180, 4)


def test_newton_inversion_count_and_checks():
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 2, 7, 60, seed=7)
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="fp64")
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N, K=2)
    L = ffca.lib()
    assert L.ffca_set_p_update(est.ctx, 4, 0.0) == 1  # Newton needs a step size > 0
    est.set_p_update("newton", 0.5)
    est.iterate(2, trace=False)
    assert est.inversion_count() == 2 * 7 * 2 * 2
    est.close()
    q = make_problem(8, 6, 2, 40, seed=8, alpha=0.2, kappa=50.0)
    yd, vd, ld_, Pd, N = ffca.to_device(q.y, q.v0, q.lam0, q.P0, prec="mixed")
    e8 = ffca.FastFCA(yd, vd, ld_, Pd, N=N)
    e8.set_p_update("newton", 1.0)
    e8.iterate(1, trace=False)
    assert e8.inversion_count() == 2 * 2
    e8.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("I,J,F,N,fpi,mu,K", [(8, 6, 2, 400, 20, 1.0, 1), (8, 3, 3, 300, 20, 1.0, 1),
                                              (8, 6, 2, 400, 20, 0.5, 2)])
def test_newton_large_array_matches_oracle(prec, I, J, F, N, fpi, mu, K):
    """Newton's method at I = 8 (a CTA per problem, the 128 x 128 system in
    shared memory) after fixed-point iterations, in cases where the oracle's
    L2 rises, against the oracle."""
    p = make_problem(I, J, F, N, seed=600 + 10 * I + J, alpha=0.2, kappa=50.0)
    v, lam, P, _ = ffa.iterate(p.y, p.v0, p.lam0, p.P0, fpi, counter=OpCounter())
    ref = ffa.iterate(p.y, v, lam, P, 3, K=K, counter=OpCounter(), p_update="newton", mu=mu)
    assert np.all(np.diff(ref[3]) > 0)
    got = run_gpu(p.y, v, lam, P, 3, prec, K=K, p_update="newton", mu=mu)
    _compare(prec, ref, got, N, F)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_newton_matches_oracle(prec):
    """A ragged batch: six fixed-point iterations, then two Newton
    iterations, per mixture against the oracle."""
    import torch
    from paper_1805_09498_gb300 import ffca
    I, J = 3, 3
    Ns = [137, 300, 64, 210]
    probs = make_batch(I, J, 3, Ns, seed=140)
    y, v, lam, P, Ns_, off = ffca.batch_to_device([q.y for q in probs], [q.v0 for q in probs],
                                                  [q.lam0 for q in probs], [q.P0 for q in probs], prec=prec)
    est = ffca.FastFCABatch(y, v, lam, P, Ns_)
    est.iterate(6, trace=False)
    est.set_p_update("newton", 1.0)
    tr = est.iterate(2)
    torch.cuda.synchronize()
    vs = [b[:, :, :Ns_[m]].numpy() for m, b in enumerate(ffca.batch_views(v.double().cpu(), J, 3, off))]
    for m, q in enumerate(probs):
        _, r = _fpi_then(q, 6, "newton", 2, 1.0)
        _compare(prec, r, (vs[m], lam[m].cpu().numpy(), P[m].cpu().numpy(), r[3]), q.N, q.F)
    est.close()
