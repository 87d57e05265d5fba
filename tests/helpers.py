"""Shared test helpers: moving seeded problems to the GPU and error metrics."""
import numpy as np


def per_f_relerr(a, b, f_axis):
    """max over f of ||a_f - b_f|| / ||b_f|| (normwise, per frequency)."""
    a = np.moveaxis(np.asarray(a), f_axis, 0)
    b = np.moveaxis(np.asarray(b), f_axis, 0)
    F = a.shape[0]
    a = a.reshape(F, -1)
    b = b.reshape(F, -1)
    num = np.linalg.norm(a - b, axis=1)
    den = np.linalg.norm(b, axis=1)
    return float(np.max(num / np.maximum(den, 1e-300))) if F else 0.0


def run_gpu(y, v, lam, P, iters, prec, K=1, ld=None, pad_value=None, p_update=None, mu=0.0):
    """Run `iters` iterations through the C-ABI; returns (v, lam, P, trace) as numpy.
    p_update: None (the default fixed point) or a name of ffca.P_UPDATES."""
    import torch
    from paper_1805_09498_gb300 import ffca
    yd, vd, ld_, Pd, N = ffca.to_device(y, v, lam, P, prec=prec, ld=ld)
    if pad_value is not None and yd.shape[2] > N:
        yd[:, :, N:] = pad_value
        vd[:, :, N:] = pad_value
    est = ffca.FastFCA(yd, vd, ld_, Pd, N=N, K=K)
    if p_update is not None:
        est.set_p_update(p_update, mu)
    tr = est.iterate(iters)
    torch.cuda.synchronize()
    out = (vd[:, :, :N].double().cpu().numpy(), ld_.cpu().numpy(), Pd.cpu().numpy(), tr)
    est.close()
    return out
