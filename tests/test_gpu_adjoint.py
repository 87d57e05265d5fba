"""GPU parity of the adjoint kernels (ffca_nll_grad, ffca_wiener_se_grad and
the autograd functions over them) against the FP64 gradient oracle, and
against central finite differences of the oracle's losses.

Tolerances (normwise relative error per frequency, max over f):
    FP64 path:  1e-9 on dv, dlambda, dP; 1e-9 relative on the loss
    mixed path: 1e-4 on dv, dlambda, dP; |dLoss| / (N F) <= 1e-5 per point
    finite differences (FP64, 16-frame slice): 1e-6 relative
"""
import numpy as np
import pytest

from oracle import adjoint as adj
from paper_1805_09498_gb300.synth import make_problem

from helpers import per_f_relerr

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(par=1e-9, loss_rel=1e-9), "mixed": dict(par=1e-4, loss_tf=1e-5)}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1805_09498_gb300 import build
    build.build()


def _device_problem(p, prec):
    import torch
    from paper_1805_09498_gb300 import ffca
    yd, vd, lamd, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=prec)
    s = None
    if p.x is not None:
        cdt = yd.dtype
        s = torch.zeros((p.J, p.I, p.F, yd.shape[2]), dtype=cdt)
        s[..., :N] = torch.from_numpy(p.x).to(cdt)
        s = s.to(yd.device)
    return yd, vd, lamd, Pd, N, s


def _gpu_grads(p, prec, se=False):
    import torch
    from paper_1805_09498_gb300 import ffca
    yd, vd, lamd, Pd, N, s = _device_problem(p, prec)
    est = ffca.FastFCA(yd, vd, lamd, Pd, N=N)
    loss, dv, dl, dP = est.wiener_se_grad(s) if se else est.nll_grad()
    torch.cuda.synchronize()
    out = (loss, dv[:, :, :N].double().cpu().numpy(), dl.cpu().numpy(), dP.cpu().numpy())
    est.close()
    return out


def _compare(prec, p, ref_loss, ref, got, p_zero=False):
    """p_zero: dP vanishes identically (I = 1, squared error: P cancels out
    of the Wiener estimate), so it is checked in absolute terms."""
    loss, gv, gl, gP = got
    rv, rl, rP = ref
    e = dict(v=per_f_relerr(gv, rv, 1), lam=per_f_relerr(gl, rl, 0))
    if p_zero:
        assert np.max(np.abs(gP)) <= (1e-12 if prec == "fp64" else 1e-5) * p.N
    else:
        e["P"] = per_f_relerr(gP, rP, 0)
    tol = TOL[prec]
    for k, x in e.items():
        assert x <= tol["par"], (k, x, e)
    if prec == "fp64":
        assert abs(loss - ref_loss) <= tol["loss_rel"] * abs(ref_loss), (loss, ref_loss)
    else:
        assert abs(loss - ref_loss) <= tol["loss_tf"] * p.N * p.F, (loss, ref_loss)


SHAPES = [(4, 4, 5, 37), (3, 3, 4, 50), (2, 3, 3, 33), (1, 2, 3, 17), (4, 2, 3, 1030), (3, 6, 2, 64),
          (8, 6, 3, 61), (8, 3, 2, 300), (8, 2, 2, 45)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", SHAPES)
def test_nll_gradient_matches_oracle(prec, shape):
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=300 + I * 10 + J)
    got = _gpu_grads(p, prec)
    _compare(prec, p, adj.nll(p.y, p.v0, p.lam0, p.P0), adj.nll_grad(p.y, p.v0, p.lam0, p.P0), got)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", SHAPES)
def test_wiener_se_gradient_matches_oracle(prec, shape):
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=400 + I * 10 + J, keep_images=True)
    got = _gpu_grads(p, prec, se=True)
    _compare(prec, p, adj.wiener_se(p.y, p.x, p.v0, p.lam0, p.P0),
             adj.wiener_se_grad(p.y, p.x, p.v0, p.lam0, p.P0), got, p_zero=(I == 1))


@pytest.mark.parametrize("se", [False, True])
def test_large_array_gradients_match_central_differences(se):
    """I = 8, J = 6 (the large-array shape, eight threads per unit) on a
    16-frame slice: FP64 GPU gradients against central differences of the
    oracle's loss along random directions."""
    p = make_problem(8, 6, 3, 16, seed=78, keep_images=True, alpha=0.2, kappa=50.0)
    loss, gv, gl, gP = _gpu_grads(p, "fp64", se=se)
    if se:
        L = lambda v, lam, P: adj.wiener_se(p.y, p.x, v, lam, P)  # noqa: E731
    else:
        L = lambda v, lam, P: adj.nll(p.y, v, lam, P)  # noqa: E731
    rng = np.random.default_rng(6)
    h = 1e-6
    for _ in range(3):
        dv = p.v0 * rng.standard_normal(p.v0.shape)
        dl = p.lam0 * rng.standard_normal(p.lam0.shape)
        dP = rng.standard_normal(p.P0.shape) + 1j * rng.standard_normal(p.P0.shape)
        fd = (L(p.v0 + h * dv, p.lam0 + h * dl, p.P0 + h * dP)
              - L(p.v0 - h * dv, p.lam0 - h * dl, p.P0 - h * dP)) / (2 * h)
        pred = np.sum(gv * dv) + np.sum(gl * dl) + 2.0 * np.real(np.sum(gP.conj() * dP))
        assert abs(fd - pred) <= 1e-6 * abs(fd), (fd, pred)


@pytest.mark.parametrize("se", [False, True])
def test_gradients_match_central_differences_on_a_16_frame_slice(se):
    """The adjoint workload's shape (I = J = 4, F = 257) on a 16-frame slice:
    FP64 GPU gradients against central differences of the oracle's loss along
    random directions (independent of both gradient codes)."""
    p = make_problem(4, 4, 257, 16, seed=77, keep_images=True)
    loss, gv, gl, gP = _gpu_grads(p, "fp64", se=se)
    if se:
        L = lambda v, lam, P: adj.wiener_se(p.y, p.x, v, lam, P)  # noqa: E731
    else:
        L = lambda v, lam, P: adj.nll(p.y, v, lam, P)  # noqa: E731
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(4):
        dv = p.v0 * rng.standard_normal(p.v0.shape)
        dl = p.lam0 * rng.standard_normal(p.lam0.shape)
        dP = rng.standard_normal(p.P0.shape) + 1j * rng.standard_normal(p.P0.shape)
        fd = (L(p.v0 + h * dv, p.lam0 + h * dl, p.P0 + h * dP)
              - L(p.v0 - h * dv, p.lam0 - h * dl, p.P0 - h * dP)) / (2 * h)
        pred = np.sum(gv * dv) + np.sum(gl * dl) + 2.0 * np.real(np.sum(gP.conj() * dP))
        assert abs(fd - pred) <= 1e-6 * abs(fd), (fd, pred)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_workload_against_oracle(prec):
    """I = J = 4, F = 257, N = 2000 (the adjoint workload), both losses."""
    p = make_problem(4, 4, 257, 2000, seed=3, keep_images=True)
    got = _gpu_grads(p, prec)
    _compare(prec, p, adj.nll(p.y, p.v0, p.lam0, p.P0), adj.nll_grad(p.y, p.v0, p.lam0, p.P0), got)
    got = _gpu_grads(p, prec, se=True)
    _compare(prec, p, adj.wiener_se(p.y, p.x, p.v0, p.lam0, p.P0),
             adj.wiener_se_grad(p.y, p.x, p.v0, p.lam0, p.P0), got)


def test_autograd_functions():
    """loss.backward() through ffca.nll / ffca.wiener_se gives the kernel's
    gradients in torch's convention (2 dL/dP^* for complex P), which also
    equal torch's own autograd of a plain-torch NLL in complex128."""
    import torch
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 2, 4, 40, seed=21, keep_images=True)
    yd, vd, lamd, Pd, N, s = _device_problem(p, "fp64")
    v = vd.clone().requires_grad_(True)
    lam = lamd.clone().requires_grad_(True)
    P = Pd.clone().requires_grad_(True)
    loss = ffca.nll(v, lam, P, yd, N)
    loss.backward()
    # plain torch NLL on the same state
    v2, lam2, P2 = (vd.clone().requires_grad_(True), lamd.clone().requires_grad_(True),
                    Pd.clone().requires_grad_(True))
    y = yd[:, :, :N]
    yt = torch.einsum("fai,afn->ifn", P2.conj(), y)
    sig = torch.einsum("jfn,fji->ifn", v2[:, :, :N], lam2)
    logdet = torch.linalg.slogdet(P2)[1]
    ref = -(-p.I * np.log(np.pi) * N * p.F + 2.0 * N * logdet.sum()
            - torch.sum(torch.log(sig) + yt.abs() ** 2 / sig))
    ref.backward()
    assert abs(loss.item() - ref.item()) <= 1e-9 * abs(ref.item())
    np.testing.assert_allclose(v.grad[:, :, :N].cpu().numpy(), v2.grad[:, :, :N].cpu().numpy(),
                               rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(lam.grad.cpu().numpy(), lam2.grad.cpu().numpy(), rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(P.grad.cpu().numpy(), P2.grad.cpu().numpy(), rtol=1e-8, atol=1e-8)
    # the squared-error function against the oracle, in torch's convention
    v3, lam3, P3 = (vd.clone().requires_grad_(True), lamd.clone().requires_grad_(True),
                    Pd.clone().requires_grad_(True))
    se = ffca.wiener_se(v3, lam3, P3, yd, s, N)
    se.backward()
    rv, rl, rP = adj.wiener_se_grad(p.y, p.x, p.v0, p.lam0, p.P0)
    assert per_f_relerr(v3.grad[:, :, :N].cpu().numpy(), rv, 1) < 1e-9
    assert per_f_relerr(lam3.grad.cpu().numpy(), rl, 0) < 1e-9
    assert per_f_relerr(P3.grad.cpu().numpy(), 2.0 * rP, 0) < 1e-9

