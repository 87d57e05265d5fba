"""The allocation-free entry point, ffca_iterate_noalloc.

Callers such as a real-time audio thread (where cudaMalloc may block and
synchronise the device) or a plugin without an allocator of its own cannot
hand the library a workspace.  ffca_iterate_noalloc runs the same hybrid
iterations with its scratch in a fixed array inside the library image.  These
tests call it through the C ABI and check it against the workspace-based
entry point (ffca_init + ffca_iterate) on two calls in a row, with the
tolerances of the other parity tests.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1805_09498_gb300.synth import make_problem

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


def _desc_for(yd, vd, lamd, Pd, N, prec):
    import torch
    from paper_1805_09498_gb300 import ffca
    I, F, ld = yd.shape
    return ffca.ffca_desc(I=I, J=vd.shape[0], F=F, N=N, ld=ld, K=1,
                          prec=ffca.FFCA_PREC_FP64 if prec == "fp64" else ffca.FFCA_PREC_MIXED,
                          y=yd.data_ptr(), v=vd.data_ptr(), lambda_=lamd.data_ptr(),
                          P=Pd.data_ptr(), workspace=None, workspace_bytes=0,
                          stream=torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_workspace_entry_point(prec):
    import torch
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 3, 9, 1001, seed=21)
    # the existing entry point, two calls of two iterations each
    ya, va, la, Pa, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=prec)
    est = ffca.FastFCA(ya, va, la, Pa, N=N)
    ta = np.concatenate([est.iterate(2)[:-1], est.iterate(2)])
    est.close()
    # the allocation-free entry point on a copy of the same state, two calls in a row
    yb, vb, lb, Pb, _ = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=prec)
    d = _desc_for(yb, vb, lb, Pb, N, prec)
    tb = np.concatenate([ffca.ffca_iterate_noalloc(d, 2)[:-1], ffca.ffca_iterate_noalloc(d, 2)])
    torch.cuda.synchronize()
    tol = TOL[prec]
    for a, b, ax in ((va[:, :, :N], vb[:, :, :N], 1), (la, lb, 0), (Pa, Pb, 0)):
        assert per_f_relerr(b.cpu().numpy(), a.cpu().numpy(), ax) <= tol["par"]
    if prec == "fp64":
        assert np.all(np.abs(tb - ta) <= tol["ll_rel"] * np.abs(ta))
    else:
        assert np.all(np.abs(tb - ta) <= tol["ll_tf"] * N * 9)


def test_noalloc_rejects_problems_beyond_its_scratch():
    """A workspace larger than FFCA_NOALLOC_SCRATCH_BYTES is an argument error."""
    import torch
    from paper_1805_09498_gb300 import ffca
    I, J, F, N = 3, 3, 100000, 4
    y = torch.zeros((I, F, N), dtype=torch.complex64, device="cuda")
    v = torch.ones((J, F, N), dtype=torch.float32, device="cuda")
    lam = torch.ones((F, J, I), dtype=torch.float64, device="cuda")
    P = torch.eye(I, dtype=torch.complex128, device="cuda").repeat(F, 1, 1).contiguous()
    d = _desc_for(y, v, lam, P, N, "mixed")
    assert ffca.ffca_workspace_size(d) > 8 << 20
    st = ffca.lib().ffca_iterate_noalloc(ctypes.byref(d), 1, None)
    assert st == 1
