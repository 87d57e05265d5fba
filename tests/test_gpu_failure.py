"""Failure detection on the GPU without a GPU fault: an injected fault
(ffca_test_fault) makes pass A's producers issue no copies, so the
consumers' bounded waits run out.  The call must return FFCA_ERR_TIMEOUT
within seconds, and the GPU must stay usable: a new context on the same
device then matches the oracle."""
import time

import numpy as np
import pytest

from oracle import fastfca_as as ffa
from oracle.fastfca_as import OpCounter
from paper_1805_09498_gb300.synth import make_problem

from helpers import per_f_relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1805_09498_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_withheld_copies_time_out_and_the_gpu_stays_usable(prec):
    import torch
    from paper_1805_09498_gb300 import ffca
    p = make_problem(3, 3, 4, 200, seed=13)
    yd, vd, lamd, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=prec)
    est = ffca.FastFCA(yd, vd, lamd, Pd, N=N)
    ffca.ffca_test_fault(est.ctx, ffca.FAULT_PASS_A_NO_COPIES)
    t0 = time.time()
    with pytest.raises(ffca.FFCAError) as ei:
        est.iterate(1)  # with the trace: synchronises and returns the latched status
    assert ei.value.status == 5  # FFCA_ERR_TIMEOUT
    assert time.time() - t0 < 60
    est.close()
    torch.cuda.synchronize()  # the context survived

    # a new context on a fresh copy of the state runs normally
    yd, vd, lamd, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=prec)
    est = ffca.FastFCA(yd, vd, lamd, Pd, N=N)
    tr = est.iterate(1)
    torch.cuda.synchronize()
    v_r, l_r, P_r, t_r = ffa.iterate(p.y, p.v0, p.lam0, p.P0, 1, counter=OpCounter())
    tol = 1e-4 if prec == "mixed" else 1e-9
    assert per_f_relerr(vd[:, :, :N].double().cpu().numpy(), v_r, 1) <= tol
    assert per_f_relerr(Pd.cpu().numpy(), P_r, 0) <= tol
    assert np.all(np.abs(tr - t_r) <= (1e-5 * N * 4 if prec == "mixed" else 1e-9 * np.abs(t_r)))
    est.close()


def test_switching_the_fault_off_again():
    """FFCA_FAULT_NONE restores normal launches on a context that has not
    run with the fault; unknown kinds are argument errors."""
    from paper_1805_09498_gb300 import ffca
    p = make_problem(2, 2, 3, 64, seed=14)
    yd, vd, lamd, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="mixed")
    est = ffca.FastFCA(yd, vd, lamd, Pd, N=N)
    ffca.ffca_test_fault(est.ctx, ffca.FAULT_PASS_A_NO_COPIES)
    ffca.ffca_test_fault(est.ctx, ffca.FAULT_NONE)
    assert ffca.lib().ffca_test_fault(est.ctx, 7) == 1
    est.iterate(2)  # raises on any latched status
    est.close()
