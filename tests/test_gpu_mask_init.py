"""GPU parity of the mask-based initialisation (ffca_mask_init; Sec. 5
initialises by mask-based covariance estimation, the steps are the readings
of oracle/mask_init.py) against the FP64 oracle: soft and binary masks,
every compiled I, FP64 and mixed, single mixtures and a ragged batch, masks
with zeros; for one source, where the pencil (R, R) leaves P free, the
unique parts (v and the diagonal form of P^H R P).

Tolerances: FP64 1e-9 normwise per frequency on v, lambda and P; mixed 1e-4
(the covariances are summed in FP64 from the FP32 data on both sides; v is
formed in FP32 on the GPU).
"""
import numpy as np
import pytest

from oracle import mask_init as mi
from paper_1805_09498_gb300.synth import make_batch, make_problem

from helpers import per_f_relerr

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "mixed": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1805_09498_gb300 import build
    build.build()


def soft_masks(p):
    """Masks from the true model: each source's share of the model power,
    v_j tr(Lambda_j) / sum_k v_k tr(Lambda_k)."""
    pw = p.v_true * p.lam_true.sum(axis=2).T[:, :, None]
    return pw / pw.sum(axis=0, keepdims=True)


def binary_masks(p):
    s = soft_masks(p)
    return (s == s.max(axis=0, keepdims=True)).astype(np.float64)


def _run(p, m, prec, sweeps=10, delta=1e-3, ld=None):
    import torch
    from paper_1805_09498_gb300 import ffca
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=prec, ld=ld)
    md = torch.zeros_like(vd)
    md[:, :, :N] = torch.from_numpy(m).to(vd.dtype)
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N)
    est.mask_init(md, sweeps, delta)
    torch.cuda.synchronize()
    out = (vd[:, :, :N].double().cpu().numpy(), ld_.cpu().numpy(), Pd.cpu().numpy(), est)
    # the oracle reads the values the GPU read (FP32 data widened for mixed)
    y_in = yd[:, :, :N].cpu().numpy().astype(np.complex128)
    m_in = md[:, :, :N].double().cpu().numpy()
    return out, y_in, m_in


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("I,J,F,N,kind", [(2, 2, 5, 300, "soft"), (3, 3, 6, 400, "soft"), (4, 3, 4, 500, "binary"),
                                          (3, 5, 3, 350, "soft"), (8, 6, 2, 800, "soft"), (1, 2, 4, 200, "soft")])
def test_matches_oracle(prec, I, J, F, N, kind):
    alpha, kappa = (0.2, 50.0) if I == 8 else (0.3, 10.0)
    p = make_problem(I, J, F, N, seed=800 + 10 * I + J, alpha=alpha, kappa=kappa)
    m = soft_masks(p) if kind == "soft" else binary_masks(p)
    (vg, lg, Pg, est), y_in, m_in = _run(p, m, prec)
    est.close()
    vr, lr, Pr = mi.mask_init(y_in, m_in, sweeps=10, delta=1e-3)
    e = dict(v=per_f_relerr(vg, vr, 1), lam=per_f_relerr(lg, lr, 0), P=per_f_relerr(Pg, Pr, 0))
    print(prec, I, J, kind, e)
    assert max(e.values()) <= TOL[prec], e


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_start_alone_and_ragged_row(prec):
    """No alternations (the GEVD start alone), a padded row with NaN in the
    padding frames (they are not read)."""
    import torch
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 2, 4, 333, seed=9)
    m = soft_masks(p)
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=prec, ld=344)
    yd[:, :, N:] = float("nan")
    md = torch.full_like(vd, float("nan"))
    md[:, :, :N] = torch.from_numpy(m).to(vd.dtype)
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N)
    est.mask_init(md, 0, 1e-3)
    torch.cuda.synchronize()
    vr, lr, Pr = mi.mask_init(yd[:, :, :N].cpu().numpy().astype(np.complex128), md[:, :, :N].double().cpu().numpy(),
                              sweeps=0)
    e = dict(v=per_f_relerr(vd[:, :, :N].double().cpu().numpy(), vr, 1), lam=per_f_relerr(ld_.cpu().numpy(), lr, 0),
             P=per_f_relerr(Pd.cpu().numpy(), Pr, 0))
    assert max(e.values()) <= TOL[prec], e
    est.close()


def test_one_source_unique_parts():
    """J = 1: every generalized eigenvalue of (R, R) is 1, so P is any P with
    P^H R P diagonal; v = max(m, delta) y^H R^{-1} y / I does not depend on
    the choice."""
    p = make_problem(3, 1, 3, 300, seed=4)
    m = np.random.default_rng(5).uniform(0.2, 1.0, (1, 3, 300))
    (vg, lg, Pg, est), y_in, m_in = _run(p, m, "fp64", sweeps=3)
    est.close()
    vr, _, _ = mi.mask_init(y_in, m_in, sweeps=3)
    assert per_f_relerr(vg, vr, 1) < 1e-9
    R = mi.masked_covariances(y_in, m_in)
    M = np.einsum("fai,fjab,fbk->fjik", Pg.conj(), R, Pg)
    off = M - np.einsum("fjii->fji", M)[..., None] * np.eye(3)
    assert np.max(np.abs(off)) < 1e-9 * np.max(np.abs(M))
    assert np.allclose(lg, np.einsum("fjii->fji", M).real, rtol=1e-9)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_oracle(prec):
    """A ragged batch: every mixture initialised from its masks, against the
    oracle per mixture."""
    import torch
    from paper_1805_09498_gb300 import ffca
    I, J, F = 3, 3, 3
    Ns = [150, 37, 420, 96]
    probs = make_batch(I, J, F, Ns, seed=55)
    y, v, lam, P, Ns_, off = ffca.batch_to_device([q.y for q in probs], [q.v0 for q in probs],
                                                  [q.lam0 for q in probs], [q.P0 for q in probs], prec=prec)
    md = torch.ones_like(v)
    views = ffca.batch_views(md, J, F, off)
    for k, q in enumerate(probs):
        views[k][:, :, :q.N] = torch.from_numpy(soft_masks(q)).to(v.dtype)
    est = ffca.FastFCABatch(y, v, lam, P, Ns_)
    est.mask_init(md)
    torch.cuda.synchronize()
    yv = ffca.batch_views(y.cpu(), I, F, off)
    vv = ffca.batch_views(v.double().cpu(), J, F, off)
    mv = ffca.batch_views(md.double().cpu(), J, F, off)
    for k, q in enumerate(probs):
        n = q.N
        vr, lr, Pr = mi.mask_init(yv[k][:, :, :n].numpy().astype(np.complex128), mv[k][:, :, :n].numpy())
        e = dict(v=per_f_relerr(vv[k][:, :, :n].numpy(), vr, 1), lam=per_f_relerr(lam[k].cpu().numpy(), lr, 0),
                 P=per_f_relerr(P[k].cpu().numpy(), Pr, 0))
        assert max(e.values()) <= TOL[prec], (k, e)
    est.close()


def test_initialised_estimation_rises():
    """From the masks' initial state the hybrid iterations raise L2 (the
    monitor of the whole chain: init, then Sec. 4.4)."""
    p = make_problem(3, 3, 8, 600, seed=21)
    (vg, lg, Pg, est), _, _ = _run(p, soft_masks(p), "mixed")
    tr = est.iterate(10)
    est.close()
    assert np.all(np.isfinite(tr)) and tr[-1] > tr[0]


def test_argument_checks():
    import torch
    from paper_1805_09498_gb300 import ffca
    p = make_problem(2, 2, 3, 50, seed=3)
    yd, vd, ld_, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="fp64")
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N)
    md = torch.ones_like(vd)
    L = ffca.lib()
    import ctypes
    for sweeps, delta in [(-1, 1e-3), (1001, 1e-3), (10, 0.0), (10, 2.0), (10, float("nan"))]:
        assert L.ffca_mask_init(est.ctx, ctypes.c_void_p(md.data_ptr()), sweeps, delta) == 1
    assert L.ffca_mask_init(est.ctx, None, 10, 1e-3) == 1
    md[1, 2, :] = 0.0  # an all-zero mask row: no covariance for that source and frequency
    with pytest.raises(ffca.FFCAError):
        est.mask_init(md)
    est.close()
