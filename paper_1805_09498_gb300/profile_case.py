"""A fixed, small FastFCA-AS run for kernel profiling (e.g. under ncu).

    python -m paper_1805_09498_gb300.profile_case [--N 8000] [--iters 3] [--prec mixed]

Default: I = J = 3, F = 513, N = 8000 frames (y 98 MB + v 49 MB in the mixed
path: larger than the 129 MB L2 together, a few hundred MB on the device),
`iters` hybrid iterations followed by one Wiener pass.  P(f) is drawn with
alpha = 0.3, cond < 10, or alpha = 0.2, cond < 50 for I = 8 (the large-array
workload; `--I 8 --J 6 --N 4000` is that workload at full size, y 131 MB +
v 49 MB).

    python -m paper_1805_09498_gb300.profile_case --batch 16 [--I 4 --J 3 --F 257]

A batch of that many mixtures with lengths uniform in [200, 4000] (the
batched workload's distribution; 16 mixtures: y 263 MB + v 99 MB), `iters`
iterations through the batch API.
"""
from __future__ import annotations

import argparse

from . import build as _build
from . import ffca
from .synth import batch_lengths, make_batch_device, make_problem


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--I", type=int, default=3)
    ap.add_argument("--J", type=int, default=3)
    ap.add_argument("--F", type=int, default=513)
    ap.add_argument("--N", type=int, default=8000)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--prec", choices=("mixed", "fp64"), default="mixed")
    ap.add_argument("--batch", type=int, default=0, help="mixtures of a batch (0: one mixture)")
    a = ap.parse_args()
    alpha, kappa = (0.2, 50.0) if a.I == 8 else (0.3, 10.0)
    import torch
    _build.build()
    if a.batch:
        cdt = torch.complex64 if a.prec == "mixed" else torch.complex128
        Ns = batch_lengths(a.batch, 200, 4000, seed=17)
        y, v, lam, P, Ns, _ = make_batch_device(a.I, a.J, a.F, Ns, seed=23, device="cuda",
                                                alpha=alpha, kappa=kappa, complex_dtype=cdt)
        est = ffca.FastFCABatch(y, v, lam, P, Ns)
        tr = est.iterate(a.iters)
        torch.cuda.synchronize()
        est.close()
        print("profile case done; L2 trace:", tr[0], "->", tr[-1])
        return
    p = make_problem(a.I, a.J, a.F, a.N, seed=0, alpha=alpha, kappa=kappa)
    yd, vd, lamd, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=a.prec)
    est = ffca.FastFCA(yd, vd, lamd, Pd, N=N)
    tr = est.iterate(a.iters)
    est.wiener()
    torch.cuda.synchronize()
    est.close()
    print("profile case done; L2 trace:", tr[0], "->", tr[-1])


if __name__ == "__main__":
    main()
