"""GPU parity of the conventional FCA EM baseline (Sec. 3.3), called through
the C ABI, against the FP64 oracle of FCA on the same seeded inputs, and its
operation counts against the numbers Sec. 3.4 prints.

Tolerances as for FastFCA-AS: FP64 1e-9 (normwise per frequency) on v and
S_j and relative on L1; mixed 1e-4 on v and S_j, 1e-5 nats per point on L1.
"""
import json
import os

import numpy as np
import pytest

from oracle import fca
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


def run_fca_gpu(y, v, S, iters, prec, ld=None):
    import torch
    from paper_1805_09498_gb300 import ffca
    yd, vd, _, _, N = ffca.to_device(y, v, np.zeros((y.shape[1], v.shape[0], y.shape[0])),
                                     np.zeros((y.shape[1], y.shape[0], y.shape[0]), complex),
                                     prec=prec, ld=ld)
    Sd = torch.from_numpy(np.ascontiguousarray(S)).to("cuda")
    est = ffca.FCA(yd, vd, Sd, N=N)
    tr = est.iterate(iters)
    counts = est.op_counts()
    torch.cuda.synchronize()
    out = (vd[:, :, :N].double().cpu().numpy(), Sd.cpu().numpy(), tr, counts)
    est.close()
    return out


def _check(prec, ref, got, N, F):
    v_r, S_r, t_r = ref
    v_g, S_g, t_g, _ = got
    ev, eS = per_f_relerr(v_g, v_r, 1), per_f_relerr(S_g, S_r, 0)
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert ev <= tol and eS <= tol, (ev, eS)
    if prec == "fp64":
        assert np.all(np.abs(t_g - t_r) <= 1e-9 * np.abs(t_r)), (t_g, t_r)
    else:
        assert np.all(np.abs(t_g - t_r) <= 1e-5 * N * F), (t_g - t_r) / (N * F)


SHAPES = [(3, 3, 5, 37), (2, 3, 4, 50), (1, 2, 3, 17), (4, 2, 3, 41), (3, 1, 2, 33), (3, 3, 3, 1030),
          (4, 4, 2, 77), (2, 6, 2, 64)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", SHAPES)
def test_fca_iterations_match_oracle(prec, shape):
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=300 + I * 10 + J)
    S0 = fca.spatial_from_joint(p.P0, p.lam0)
    ref = fca.iterate(p.y, p.v0, S0, 2, counter=OpCounter())
    got = run_fca_gpu(p.y, p.v0, S0, 2, prec)
    _check(prec, ref, got, N, F)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fca_trajectory_plain_config(prec):
    """20 EM iterations at I = J = 3, F = 257, N = 600; L1 rises (EM)."""
    p = make_problem(3, 3, 257, 600, seed=0)
    S0 = fca.spatial_from_joint(p.P0, p.lam0)
    ref = fca.iterate(p.y, p.v0, S0, 20, counter=OpCounter())
    got = run_fca_gpu(p.y, p.v0, S0, 20, prec)
    _check(prec, ref, got, 600, 257)
    assert np.all(np.diff(got[2]) >= -1e-6 * np.abs(got[2][:-1]))


def test_fca_operation_counts_match_paper():
    """At I = J = 3, N = 249, F = 512 one EM iteration performs the (J+N)F =
    129024 inversions and 2JNF = 764928 multiplications Sec. 3.4 prints."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "op_counts.json")))["fca"]
    p = make_problem(g["I"], g["J"], g["F"], g["N"], seed=12)
    S0 = fca.spatial_from_joint(p.P0, p.lam0)
    got = run_fca_gpu(p.y, p.v0, S0, 1, "fp64")
    assert got[3] == (g["inversions"], g["multiplications"])


def test_fca_and_fastfca_agree_from_joint_state():
    """Started from S_j = P^-H Lambda_j P^-1 the two GPU paths give the same
    first v update and log-likelihood (Sec. 4.1: FastFCA-AS is FCA with
    jointly diagonalisable S_j)."""
    from helpers import run_gpu
    p = make_problem(3, 3, 7, 300, seed=21)
    S0 = fca.spatial_from_joint(p.P0, p.lam0)
    a = run_fca_gpu(p.y, p.v0, S0, 1, "fp64")
    b = run_gpu(p.y, p.v0, p.lam0, p.P0, 1, "fp64")
    assert per_f_relerr(a[0], b[0], 1) <= 1e-10
    assert abs(a[2][0] - b[3][0]) <= 1e-10 * abs(b[3][0])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(8, 6, 3, 37), (8, 2, 2, 300), (8, 6, 2, 1030)])
def test_fca_large_array_matches_oracle(prec, shape):
    """I = 8: the rearranged E/M steps (per-point Hermitian inverse kept, the
    J products per frequency) against the oracle's literal Sec. 3.3 form."""
    I, J, F, N = shape
    p = make_problem(I, J, F, N, seed=600 + J, alpha=0.2, kappa=50.0)
    S0 = fca.spatial_from_joint(p.P0, p.lam0)
    ref = fca.iterate(p.y, p.v0, S0, 2, counter=OpCounter())
    got = run_fca_gpu(p.y, p.v0, S0, 2, prec)
    _check(prec, ref, got, N, F)
    # operations as performed: one inversion of R per point, 2 J products per frequency
    inv, mul = got[3]
    assert inv == 2 * N * F and mul == 2 * 2 * J * F
