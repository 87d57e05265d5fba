"""GPU parity of the adjoint on batch contexts (ffca_nll_grad and
ffca_wiener_se_grad with ragged mixtures) against the FP64 gradient oracle
applied to each mixture on its own.

Tolerances as for single mixtures (normwise relative error per frequency,
max over f and mixtures): FP64 1e-9 on dv, dlambda, dP and the loss; mixed
1e-4 on the gradients and 1e-5 per point on the loss.
"""
import numpy as np
import pytest

from oracle import adjoint as adj
from paper_1805_09498_gb300.synth import make_problem

from helpers import per_f_relerr

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(par=1e-9, loss_rel=1e-9), "mixed": dict(par=1e-4, loss_tf=1e-5)}
RAGGED = [37, 200, 9, 129, 64]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1805_09498_gb300 import build
    build.build()


def _batch(I, J, F, seed, se):
    probs = [make_problem(I, J, F, max(n, I), seed + 7919 * m, keep_images=se) for m, n in enumerate(RAGGED)]
    return probs


def _run(probs, prec, se):
    import torch
    from paper_1805_09498_gb300 import ffca
    I, J, F = probs[0].I, probs[0].J, probs[0].F
    y, v, lam, P, Ns, off = ffca.batch_to_device([p.y for p in probs], [p.v0 for p in probs],
                                                 [p.lam0 for p in probs], [p.P0 for p in probs], prec=prec)
    est = ffca.FastFCABatch(y, v, lam, P, Ns)
    if se:
        s = torch.zeros(J * I * F * int(off[-1]), dtype=y.dtype)
        for m, blk in enumerate(ffca.batch_views(s, J * I, F, off)):
            blk.view(J, I, F, -1)[..., :Ns[m]] = torch.from_numpy(probs[m].x).to(y.dtype)
        loss, dv, dl, dP = est.wiener_se_grad(s.to(y.device))
    else:
        loss, dv, dl, dP = est.nll_grad()
    torch.cuda.synchronize()
    dvh = dv.double().cpu()
    dvs = [b.numpy() for b in ffca.batch_views(dvh, J, F, off)]
    out = loss, dvs, dl.cpu().numpy(), dP.cpu().numpy(), Ns
    est.close()
    return out


def _check(prec, probs, got, se):
    loss, dvs, dl, dP, Ns = got
    tol = TOL[prec]
    ref_loss = 0.0
    for m, p in enumerate(probs):
        if se:
            ref_loss += adj.wiener_se(p.y, p.x, p.v0, p.lam0, p.P0)
            rv, rl, rP = adj.wiener_se_grad(p.y, p.x, p.v0, p.lam0, p.P0)
        else:
            ref_loss += adj.nll(p.y, p.v0, p.lam0, p.P0)
            rv, rl, rP = adj.nll_grad(p.y, p.v0, p.lam0, p.P0)
        e = dict(v=per_f_relerr(dvs[m][:, :, :Ns[m]], rv, 1), lam=per_f_relerr(dl[m], rl, 0))
        if se and p.I == 1:  # P cancels out of the Wiener estimate: dP vanishes
            assert np.max(np.abs(dP[m])) <= (1e-12 if prec == "fp64" else 1e-5) * p.N
        else:
            e["P"] = per_f_relerr(dP[m], rP, 0)
        for k, x in e.items():
            assert x <= tol["par"], (m, k, x, e)
        # frames beyond N_m: the last vector unit's tail is written as 0, the rest untouched (0 here)
        assert np.all(dvs[m][:, :, Ns[m]:] == 0)
    NF = sum(p.N * p.F for p in probs)
    if prec == "fp64":
        assert abs(loss - ref_loss) <= tol["loss_rel"] * abs(ref_loss), (loss, ref_loss)
    else:
        assert abs(loss - ref_loss) <= tol["loss_tf"] * NF, (loss, ref_loss)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("I,J", [(4, 3), (3, 3), (2, 2), (1, 2), (4, 4), (8, 6)])
def test_batch_nll_gradient_matches_oracle(prec, I, J):
    probs = _batch(I, J, 3, 500 + 10 * I + J, se=False)
    _check(prec, probs, _run(probs, prec, se=False), se=False)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("I,J", [(4, 3), (3, 3), (2, 2), (1, 2), (8, 3)])
def test_batch_wiener_se_gradient_matches_oracle(prec, I, J):
    probs = _batch(I, J, 3, 600 + 10 * I + J, se=True)
    _check(prec, probs, _run(probs, prec, se=True), se=True)


def test_batch_gradients_after_iterations():
    """The gradient of the state the batch iterations left: three hybrid
    iterations, then NLL's gradient, against the oracle at the oracle's
    iterate (FP64)."""
    import torch
    from oracle import fastfca_as as ffa
    from oracle.fastfca_as import OpCounter
    from paper_1805_09498_gb300 import ffca
    probs = _batch(3, 2, 4, 700, se=False)
    y, v, lam, P, Ns, off = ffca.batch_to_device([p.y for p in probs], [p.v0 for p in probs],
                                                 [p.lam0 for p in probs], [p.P0 for p in probs], prec="fp64")
    est = ffca.FastFCABatch(y, v, lam, P, Ns)
    est.iterate(3, trace=False)
    loss, dv, dl, dP = est.nll_grad()
    torch.cuda.synchronize()
    dvs = [b.numpy() for b in ffca.batch_views(dv.cpu(), 2, 4, off)]
    ref_loss = 0.0
    for m, p in enumerate(probs):
        v3, l3, P3, _ = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 3, counter=OpCounter())
        ref_loss += adj.nll(p.y, v3, l3, P3)
        rv, rl, rP = adj.nll_grad(p.y, v3, l3, P3)
        assert per_f_relerr(dvs[m][:, :, :Ns[m]], rv, 1) <= 1e-8
        assert per_f_relerr(dl.cpu().numpy()[m], rl, 0) <= 1e-8
        assert per_f_relerr(dP.cpu().numpy()[m], rP, 0) <= 1e-8
    assert abs(loss - ref_loss) <= 1e-9 * abs(ref_loss)
    est.close()
