"""Thin Python binding of libffca.so (argument marshalling only).

The functions keep the C names of include/ffca.h; every step of the
estimation runs in the CUDA library.  PyTorch supplies device memory and the
stream.  There is no fallback: if libffca.so is missing or cannot be loaded
the binding raises.

Typical use (device tensors, mic-planar layouts, ld = padded frame stride):

    est = FastFCA(y, v, lam, P, N=N)          # y [I,F,ld] complex, v [J,F,ld] real
    trace = est.iterate(20)                    # numpy array, iters + 1 values of L2
    out = est.wiener()                         # [J,I,F,ld] complex
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libffca.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "ffca.h")

FFCA_OK = 0
FFCA_PREC_FP64 = 0
FFCA_PREC_MIXED = 1
STATUS_NAMES = {0: "FFCA_OK", 1: "FFCA_ERR_ARG", 2: "FFCA_ERR_CUDA", 3: "FFCA_ERR_NONFINITE",
                4: "FFCA_ERR_SINGULAR", 5: "FFCA_ERR_TIMEOUT", 6: "FFCA_ERR_INTERNAL",
                7: "FFCA_ERR_UNSUPPORTED"}


class FFCAError(RuntimeError):
    def __init__(self, status: int, what: str, frequency: int = -1):
        self.status = status
        self.frequency = frequency
        name = STATUS_NAMES.get(status, str(status))
        extra = f" at frequency {frequency}" if frequency >= 0 else ""
        if status in (2, 6) and _lib is not None:
            detail = _lib.ffca_last_error().decode()
            if detail:
                extra += f" ({detail})"
        super().__init__(f"{what}: {name}{extra}")


class ffca_fca_desc(ctypes.Structure):
    _fields_ = [("I", ctypes.c_int), ("J", ctypes.c_int), ("F", ctypes.c_int),
                ("N", ctypes.c_int), ("ld", ctypes.c_int), ("prec", ctypes.c_int),
                ("y", ctypes.c_void_p), ("v", ctypes.c_void_p), ("S", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("stream", ctypes.c_void_p)]


class ffca_desc(ctypes.Structure):
    _fields_ = [("I", ctypes.c_int), ("J", ctypes.c_int), ("F", ctypes.c_int),
                ("N", ctypes.c_int), ("ld", ctypes.c_int), ("K", ctypes.c_int),
                ("prec", ctypes.c_int),
                ("y", ctypes.c_void_p), ("v", ctypes.c_void_p), ("lambda_", ctypes.c_void_p),
                ("P", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("stream", ctypes.c_void_p)]


class ffca_batch_desc(ctypes.Structure):
    _fields_ = [("I", ctypes.c_int), ("J", ctypes.c_int), ("F", ctypes.c_int),
                ("M", ctypes.c_int), ("K", ctypes.c_int), ("prec", ctypes.c_int),
                ("frame_offset", ctypes.POINTER(ctypes.c_longlong)),
                ("N", ctypes.POINTER(ctypes.c_int)), ("ld", ctypes.c_longlong),
                ("y", ctypes.c_void_p), ("v", ctypes.c_void_p), ("lambda_", ctypes.c_void_p),
                ("P", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("stream", ctypes.c_void_p)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libffca.so (built by paper_1805_09498_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1805_09498_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp, ci, dp = ctypes.c_void_p, ctypes.c_int, P(ctypes.c_double)
    sigs = {
        "ffca_workspace_size": (ctypes.c_size_t, [P(ffca_desc)]),
        "ffca_init": (ci, [P(vp), P(ffca_desc)]),
        "ffca_iterate": (ci, [vp, ci, dp]),
        "ffca_loglik": (ci, [vp, dp]),
        "ffca_wiener": (ci, [vp, vp]),
        "ffca_sync": (ci, [vp]),
        "ffca_error_frequency": (ci, [vp]),
        "ffca_inversion_count": (ci, [vp, P(ctypes.c_ulonglong)]),
        "ffca_upload": (ci, [vp, vp, vp, vp, vp]),
        "ffca_download": (ci, [vp, vp, vp, vp]),
        "ffca_wiener_host": (ci, [vp, vp, vp]),
        "ffca_timing_enable": (ci, [vp, ci]),
        "ffca_timing_read": (ci, [vp, dp, P(ctypes.c_ulonglong)]),
        "ffca_iterate_noalloc": (ci, [P(ffca_desc), ci, dp]),
        "ffca_destroy": (None, [vp]),
        "ffca_nll_grad": (ci, [vp, vp, vp, vp, dp]),
        "ffca_wiener_se_grad": (ci, [vp, vp, vp, vp, vp, dp]),
        "ffca_batch_workspace_size": (ctypes.c_size_t, [P(ffca_batch_desc)]),
        "ffca_batch_init": (ci, [P(vp), P(ffca_batch_desc)]),
        "ffca_batch_iterate": (ci, [vp, ci, dp]),
        "ffca_batch_loglik": (ci, [vp, dp]),
        "ffca_set_graph": (ci, [vp, ci]),
        "ffca_set_p_update": (ci, [vp, ci, ctypes.c_double]),
        "ffca_test_fault": (ci, [vp, ci]),
        "ffca_batch_config_count": (ci, []),
        "ffca_batch_autotune": (ci, [vp, ci, P(ci), P(ci), dp, dp]),
        "ffca_batch_set_config": (ci, [vp, ci, ci]),
        "ffca_batch_destroy": (None, [vp]),
        "ffca_fca_workspace_size": (ctypes.c_size_t, [P(ffca_fca_desc)]),
        "ffca_fca_init": (ci, [P(vp), P(ffca_fca_desc)]),
        "ffca_fca_iterate": (ci, [vp, ci, dp]),
        "ffca_fca_loglik": (ci, [vp, dp]),
        "ffca_fca_op_counts": (ci, [vp, P(ctypes.c_ulonglong), P(ctypes.c_ulonglong)]),
        "ffca_fca_error_frequency": (ci, [vp]),
        "ffca_fca_destroy": (None, [vp]),
        "ffca_stft": (ci, [vp, ci, ctypes.c_longlong, vp, ci, vp]),
        "ffca_istft": (ci, [vp, ci, ci, ci, vp, vp]),
        "ffca_status_str": (ctypes.c_char_p, [ci]),
        "ffca_peak_fp64": (ci, [vp, dp]),
        "ffca_mask_init": (ci, [vp, vp, ci, ctypes.c_double]),
        "ffca_set_resident": (ci, [vp, ci]),
        "ffca_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


# ------------------------------------------------------------ STFT front / back end
STFT_L, STFT_H = 1024, 512
STFT_F = STFT_L // 2 + 1


def stft_frames(S: int) -> int:
    """Frames ffca_stft makes of S samples."""
    return 1 + (S - STFT_L) // STFT_H if S >= STFT_L else 0


def stft(x, ld: int | None = None, stream=None):
    """ffca_stft: x [C, S] float32 CUDA -> (X [C, F, ld] complex64, N)."""
    import torch
    if not x.is_cuda or x.dtype != torch.float32 or x.dim() != 2 or not x.is_contiguous():
        raise ValueError("x must be a contiguous [C, S] float32 CUDA tensor")
    C, S = x.shape
    N = stft_frames(S)
    ld = padded_ld(max(N, 1)) if ld is None else ld
    out = torch.empty((C, STFT_F, ld), dtype=torch.complex64, device=x.device)
    s = stream if stream is not None else torch.cuda.current_stream(x.device)
    st = lib().ffca_stft(x.data_ptr(), C, S, out.data_ptr(), ld, s.cuda_stream)
    if st != 0:
        raise FFCAError(st, "ffca_stft")
    return out, N


def istft(X, N: int, stream=None):
    """ffca_istft: X [C, F, ld] complex64 CUDA (first N frames) -> x [C, (N+1) H] float32."""
    import torch
    if not X.is_cuda or X.dtype != torch.complex64 or X.dim() != 3 or not X.is_contiguous():
        raise ValueError("X must be a contiguous [C, F, ld] complex64 CUDA tensor")
    C, Fb, ld = X.shape
    if Fb != STFT_F:
        raise ValueError(f"X must have {STFT_F} bins")
    out = torch.empty((C, (N + 1) * STFT_H if N else 0), dtype=torch.float32, device=X.device)
    s = stream if stream is not None else torch.cuda.current_stream(X.device)
    st = lib().ffca_istft(X.data_ptr(), C, N, ld, out.data_ptr(), s.cuda_stream)
    if st != 0:
        raise FFCAError(st, "ffca_istft")
    return out


def header_functions() -> list[str]:
    """Names of the functions include/ffca.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ffca_[a-z0-9_]+)\s*\(", text)))


# ------------------------------------------------------------ C-named calls
def ffca_workspace_size(desc: ffca_desc) -> int:
    return int(lib().ffca_workspace_size(ctypes.byref(desc)))


def ffca_init(desc: ffca_desc) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    st = lib().ffca_init(ctypes.byref(ctx), ctypes.byref(desc))
    if st != FFCA_OK:
        raise FFCAError(st, "ffca_init")
    return ctx


def _check(ctx, st, what):
    if st != FFCA_OK:
        raise FFCAError(st, what, lib().ffca_error_frequency(ctx))


def ffca_iterate(ctx, iters: int, trace: bool = True):
    """Returns the L2 trace (numpy, iters + 1) when trace, else None (enqueue only)."""
    if trace:
        buf = np.zeros(iters + 1, dtype=np.float64)
        st = lib().ffca_iterate(ctx, iters, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        _check(ctx, st, "ffca_iterate")
        return buf
    _check(ctx, lib().ffca_iterate(ctx, iters, None), "ffca_iterate")
    return None


def ffca_loglik(ctx) -> float:
    out = ctypes.c_double()
    _check(ctx, lib().ffca_loglik(ctx, ctypes.byref(out)), "ffca_loglik")
    return out.value


def ffca_wiener(ctx, out_ptr: int) -> None:
    _check(ctx, lib().ffca_wiener(ctx, ctypes.c_void_p(out_ptr)), "ffca_wiener")


def ffca_sync(ctx) -> None:
    _check(ctx, lib().ffca_sync(ctx), "ffca_sync")


def ffca_inversion_count(ctx) -> int:
    out = ctypes.c_ulonglong()
    _check(ctx, lib().ffca_inversion_count(ctx, ctypes.byref(out)), "ffca_inversion_count")
    return out.value


def ffca_upload(ctx, y_host=0, v_host=0, lam_host=0, P_host=0) -> None:
    _check(ctx, lib().ffca_upload(ctx, y_host or None, v_host or None, lam_host or None,
                                  P_host or None), "ffca_upload")


def ffca_download(ctx, v_host=0, lam_host=0, P_host=0) -> None:
    _check(ctx, lib().ffca_download(ctx, v_host or None, lam_host or None, P_host or None),
           "ffca_download")


def ffca_wiener_host(ctx, out_dev_ptr: int, out_host_ptr: int) -> None:
    _check(ctx, lib().ffca_wiener_host(ctx, ctypes.c_void_p(out_dev_ptr),
                                       ctypes.c_void_p(out_host_ptr)), "ffca_wiener_host")


KERNEL_KINDS = ("prep", "estep", "loglik", "wcov", "wiener", "psolve", "afinal", "adj", "adj_final", "resident")


def ffca_timing_enable(ctx, enable: bool) -> None:
    _check(ctx, lib().ffca_timing_enable(ctx, int(bool(enable))), "ffca_timing_enable")


def ffca_timing_read(ctx):
    """{kind: (device ms summed, launches)} since the last read."""
    ms = (ctypes.c_double * len(KERNEL_KINDS))()
    n = (ctypes.c_ulonglong * len(KERNEL_KINDS))()
    _check(ctx, lib().ffca_timing_read(ctx, ms, n), "ffca_timing_read")
    return {k: (ms[i], int(n[i])) for i, k in enumerate(KERNEL_KINDS)}


def ffca_iterate_noalloc(desc: ffca_desc, iters: int):
    """Allocation-free iterations (static library scratch); returns the L2 trace."""
    buf = np.zeros(iters + 1, dtype=np.float64)
    st = lib().ffca_iterate_noalloc(ctypes.byref(desc), iters,
                                    buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != FFCA_OK:
        raise FFCAError(st, "ffca_iterate_noalloc")
    return buf


def ffca_destroy(ctx) -> None:
    lib().ffca_destroy(ctx)


def ffca_status_str(status: int) -> str:
    return lib().ffca_status_str(status).decode()


def ffca_mask_init(ctx, masks_ptr: int, sweeps: int = 10, delta: float = 1e-3) -> None:
    _check(ctx, lib().ffca_mask_init(ctx, ctypes.c_void_p(masks_ptr), int(sweeps), float(delta)),
           "ffca_mask_init")


def ffca_peak_fp64(stream=None) -> float:
    """Measured FP64 rate of the current device in GFLOP/s (an FMA-chain
    kernel on every SM, best of three launches); synchronises the stream."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    out = ctypes.c_double(0.0)
    st = lib().ffca_peak_fp64(ctypes.c_void_p(s.cuda_stream), ctypes.byref(out))
    if st != FFCA_OK:
        raise FFCAError(st, "ffca_peak_fp64")
    return out.value


# ------------------------------------------------------------ conventional FCA
def ffca_fca_workspace_size(desc: ffca_fca_desc) -> int:
    return int(lib().ffca_fca_workspace_size(ctypes.byref(desc)))


def ffca_fca_init(desc: ffca_fca_desc) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    st = lib().ffca_fca_init(ctypes.byref(ctx), ctypes.byref(desc))
    if st != FFCA_OK:
        raise FFCAError(st, "ffca_fca_init")
    return ctx


def _check_fca(ctx, st, what):
    if st != FFCA_OK:
        raise FFCAError(st, what, lib().ffca_fca_error_frequency(ctx))


def ffca_fca_iterate(ctx, iters: int, trace: bool = True):
    if trace:
        buf = np.zeros(iters + 1, dtype=np.float64)
        _check_fca(ctx, lib().ffca_fca_iterate(ctx, iters, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                   "ffca_fca_iterate")
        return buf
    _check_fca(ctx, lib().ffca_fca_iterate(ctx, iters, None), "ffca_fca_iterate")
    return None


def ffca_fca_loglik(ctx) -> float:
    out = ctypes.c_double()
    _check_fca(ctx, lib().ffca_fca_loglik(ctx, ctypes.byref(out)), "ffca_fca_loglik")
    return out.value


def ffca_fca_op_counts(ctx):
    inv, mul = ctypes.c_ulonglong(), ctypes.c_ulonglong()
    _check_fca(ctx, lib().ffca_fca_op_counts(ctx, ctypes.byref(inv), ctypes.byref(mul)),
               "ffca_fca_op_counts")
    return inv.value, mul.value


def ffca_fca_destroy(ctx) -> None:
    lib().ffca_fca_destroy(ctx)


def ffca_nll_grad(ctx, dv_ptr: int, dlam_ptr: int, dP_ptr: int) -> float:
    """Gradients of NLL = -L2 into device buffers; returns NLL."""
    out = ctypes.c_double()
    _check(ctx, lib().ffca_nll_grad(ctx, ctypes.c_void_p(dv_ptr), ctypes.c_void_p(dlam_ptr),
                                    ctypes.c_void_p(dP_ptr), ctypes.byref(out)), "ffca_nll_grad")
    return out.value


def ffca_wiener_se_grad(ctx, s_ptr: int, dv_ptr: int, dlam_ptr: int, dP_ptr: int) -> float:
    """Gradients of the Wiener squared error against s into device buffers; returns it."""
    out = ctypes.c_double()
    _check(ctx, lib().ffca_wiener_se_grad(ctx, ctypes.c_void_p(s_ptr), ctypes.c_void_p(dv_ptr),
                                          ctypes.c_void_p(dlam_ptr), ctypes.c_void_p(dP_ptr),
                                          ctypes.byref(out)), "ffca_wiener_se_grad")
    return out.value


def ffca_batch_workspace_size(desc: ffca_batch_desc) -> int:
    return int(lib().ffca_batch_workspace_size(ctypes.byref(desc)))


def ffca_batch_init(desc: ffca_batch_desc) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    st = lib().ffca_batch_init(ctypes.byref(ctx), ctypes.byref(desc))
    if st != FFCA_OK:
        raise FFCAError(st, "ffca_batch_init")
    return ctx


def ffca_batch_iterate(ctx, iters: int, trace: bool = True):
    """Run `iters` iterations of every mixture; the summed L2 trace or None."""
    if trace:
        buf = (ctypes.c_double * (iters + 1))()
        _check(ctx, lib().ffca_batch_iterate(ctx, iters, buf), "ffca_batch_iterate")
        return np.frombuffer(buf, dtype=np.float64).copy()
    _check(ctx, lib().ffca_batch_iterate(ctx, iters, None), "ffca_batch_iterate")
    return None


def ffca_batch_loglik(ctx, M: int) -> np.ndarray:
    buf = (ctypes.c_double * M)()
    _check(ctx, lib().ffca_batch_loglik(ctx, buf), "ffca_batch_loglik")
    return np.frombuffer(buf, dtype=np.float64).copy()


def ffca_batch_config_count() -> int:
    return int(lib().ffca_batch_config_count())


def ffca_batch_autotune(ctx, rounds: int = 1):
    """Tune the batch's partitions on real iterations; returns
    (cand_a, cand_b, ms_a[], ms_b[])."""
    n = ffca_batch_config_count()
    ca, cb = ctypes.c_int(), ctypes.c_int()
    ma, mb = (ctypes.c_double * n)(), (ctypes.c_double * n)()
    _check(ctx, lib().ffca_batch_autotune(ctx, rounds, ctypes.byref(ca), ctypes.byref(cb), ma, mb),
           "ffca_batch_autotune")
    return ca.value, cb.value, list(ma), list(mb)


def ffca_batch_set_config(ctx, cand_a: int, cand_b: int) -> None:
    _check(ctx, lib().ffca_batch_set_config(ctx, cand_a, cand_b), "ffca_batch_set_config")


def ffca_set_graph(ctx, enable: bool) -> None:
    _check(ctx, lib().ffca_set_graph(ctx, 1 if enable else 0), "ffca_set_graph")


# Updates of P (ffca_p_update): the fixed point of Eq. FPI, or the gradient
# methods of Sec. 4.6 with step size mu.
P_UPDATES = {"fixed_point": 0, "gradient": 1, "natural_gradient": 2, "em": 3, "newton": 4}


def ffca_set_p_update(ctx, method: str, mu: float = 0.0) -> None:
    if method not in P_UPDATES:
        raise ValueError(f"unknown update of P {method!r}; one of {sorted(P_UPDATES)}")
    _check(ctx, lib().ffca_set_p_update(ctx, P_UPDATES[method], float(mu)), "ffca_set_p_update")


# Injected faults (tests of failure detection; see ffca_test_fault).
FAULT_NONE, FAULT_PASS_A_NO_COPIES = 0, 1


def ffca_test_fault(ctx, kind: int) -> None:
    _check(ctx, lib().ffca_test_fault(ctx, int(kind)), "ffca_test_fault")


def ffca_batch_destroy(ctx) -> None:
    lib().ffca_batch_destroy(ctx)


# ------------------------------------------------------------ torch wrapper
def padded_ld(N: int) -> int:
    """Smallest frame stride the library accepts (>= N, multiple of 4)."""
    return (N + 3) // 4 * 4


class FastFCA:
    """FastFCA-AS estimation state on one GPU, borrowed from torch tensors.

    y   [I, F, ld] complex64 (mixed precision) or complex128 (FP64), CUDA
    v   [J, F, ld] float32 / float64 (matching y), updated in place
    lam [F, J, I] float64, updated in place
    P   [F, I, I] complex128, updated in place
    N   frames actually used (default ld)
    """

    def __init__(self, y, v, lam, P, N: int | None = None, K: int = 1, stream=None):
        import torch
        if not y.is_cuda:
            raise ValueError("FastFCA needs CUDA tensors")
        if y.dtype == torch.complex64:
            prec, vdt = FFCA_PREC_MIXED, torch.float32
        elif y.dtype == torch.complex128:
            prec, vdt = FFCA_PREC_FP64, torch.float64
        else:
            raise TypeError("y must be complex64 or complex128")
        if v.dtype != vdt or lam.dtype != torch.float64 or P.dtype != torch.complex128:
            raise TypeError("dtypes: v matches y's precision, lam float64, P complex128")
        for t in (y, v, lam, P):
            if not t.is_contiguous():
                raise ValueError("tensors must be contiguous")
        I, F, ld = y.shape
        J = v.shape[0]
        if v.shape != (J, F, ld) or lam.shape != (F, J, I) or P.shape != (F, I, I):
            raise ValueError("inconsistent shapes")
        self.I, self.J, self.F, self.ld = I, J, F, ld
        self.N = ld if N is None else int(N)
        self.prec = prec
        self.y, self.v, self.lam, self.P = y, v, lam, P
        s = stream if stream is not None else torch.cuda.current_stream(y.device)
        self.stream = s
        d = ffca_desc(I=I, J=J, F=F, N=self.N, ld=ld, K=K, prec=prec,
                      y=y.data_ptr(), v=v.data_ptr(), lambda_=lam.data_ptr(), P=P.data_ptr(),
                      workspace=None, workspace_bytes=0, stream=s.cuda_stream)
        nbytes = ffca_workspace_size(d)
        if nbytes == 0 and F > 0:
            raise FFCAError(1, "ffca_workspace_size (invalid shape or CUDA failure: "
                               + lib().ffca_last_error().decode() + ")")
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=y.device)
        d.workspace = self.workspace.data_ptr()
        d.workspace_bytes = nbytes
        self.desc = d
        self.ctx = ffca_init(d)

    def iterate(self, iters: int, trace: bool = True):
        return ffca_iterate(self.ctx, iters, trace)

    def set_graph(self, enable: bool = True):
        """Replay iterate() calls from a CUDA graph (with a trace too, for
        fewer than 4096 iterations and without the resident form)."""
        ffca_set_graph(self.ctx, enable)

    def set_p_update(self, method: str = "fixed_point", mu: float = 0.0):
        """Update of P in later iterations: "fixed_point" (Eq. FPI),
        "gradient", "natural_gradient" or "newton" (Sec. 4.6) with step size
        mu, or "em" (the normal EM of Sec. 4.6; mu unused)."""
        ffca_set_p_update(self.ctx, method, mu)

    def loglik(self) -> float:
        return ffca_loglik(self.ctx)

    def set_resident(self, enable: bool = True):
        """Iterations with each problem resident on chip (ffca_set_resident)."""
        _check(self.ctx, lib().ffca_set_resident(self.ctx, 1 if enable else 0), "ffca_set_resident")

    def mask_init(self, masks, sweeps: int = 10, delta: float = 1e-3):
        """Initialise v, lam and P in place from time-frequency masks (a device
        tensor of v's shape and dtype), ffca_mask_init."""
        if masks.shape != self.v.shape or masks.dtype != self.v.dtype or not masks.is_contiguous():
            raise ValueError("masks must be a contiguous tensor of v's shape and dtype")
        ffca_mask_init(self.ctx, masks.data_ptr(), sweeps, delta)

    def wiener(self, out=None):
        import torch
        if out is None:
            out = torch.empty((self.J, self.I, self.F, self.ld), dtype=self.y.dtype,
                              device=self.y.device)
        ffca_wiener(self.ctx, out.data_ptr())
        return out

    def sync(self):
        ffca_sync(self.ctx)

    def nll_grad(self):
        """(NLL, dv, dlam, dPc) at the current state; dPc = dNLL/dP^*."""
        import torch
        dv = torch.zeros_like(self.v)
        dlam = torch.empty_like(self.lam)
        dP = torch.empty_like(self.P)
        loss = ffca_nll_grad(self.ctx, dv.data_ptr(), dlam.data_ptr(), dP.data_ptr())
        return loss, dv, dlam, dP

    def wiener_se_grad(self, s):
        """(SE, dv, dlam, dPc) of sum |x^ - s|^2 at the current state;
        s [J, I, F, ld] complex of y's dtype."""
        import torch
        if s.dtype != self.y.dtype or s.shape != (self.J, self.I, self.F, self.ld) or not s.is_contiguous():
            raise ValueError("s must be a contiguous [J, I, F, ld] tensor of y's dtype")
        dv = torch.zeros_like(self.v)
        dlam = torch.empty_like(self.lam)
        dP = torch.empty_like(self.P)
        loss = ffca_wiener_se_grad(self.ctx, s.data_ptr(), dv.data_ptr(), dlam.data_ptr(), dP.data_ptr())
        return loss, dv, dlam, dP

    def inversion_count(self) -> int:
        return ffca_inversion_count(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            ffca_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def to_device(problem_y, v, lam, P, prec: str = "mixed", device="cuda", ld: int | None = None):
    """Copy numpy arrays (mic-planar, unpadded) into padded CUDA tensors of
    the precision's types.  Returns (y, v, lam, P, N)."""
    import torch
    I, F, N = problem_y.shape
    J = v.shape[0]
    ld = padded_ld(N) if ld is None else ld
    cdt, rdt = (torch.complex64, torch.float32) if prec == "mixed" else (torch.complex128, torch.float64)
    yt = torch.zeros((I, F, ld), dtype=cdt)
    yt[:, :, :N] = torch.from_numpy(np.ascontiguousarray(problem_y)).to(cdt)
    vt = torch.ones((J, F, ld), dtype=rdt)
    vt[:, :, :N] = torch.from_numpy(np.ascontiguousarray(v)).to(rdt)
    return (yt.to(device), vt.to(device),
            torch.from_numpy(np.ascontiguousarray(lam, dtype=np.float64)).to(device),
            torch.from_numpy(np.ascontiguousarray(P, dtype=np.complex128)).to(device), N)


def batch_offsets(Ns) -> np.ndarray:
    """Row-length offsets of mixtures of Ns frames, each row padded to a
    multiple of 4 (frame_offset of ffca_batch_desc)."""
    off = np.zeros(len(Ns) + 1, dtype=np.int64)
    off[1:] = np.cumsum([padded_ld(int(n)) for n in Ns])
    return off


def batch_views(t, rows: int, F: int, offsets):
    """The per-mixture blocks [rows, F, ld_m] of a batch tensor (views)."""
    out = []
    for m in range(len(offsets) - 1):
        o, ldm = int(offsets[m]), int(offsets[m + 1] - offsets[m])
        out.append(t[rows * F * o: rows * F * (o + ldm)].view(rows, F, ldm))
    return out


def batch_to_device(ys, vs, lams, Ps, prec: str = "mixed", device="cuda", pad_value=None):
    """Pack per-mixture numpy arrays (y [I,F,N_m], v [J,F,N_m], lam [F,J,I],
    P [F,I,I]) into the mixture-major batch layout on the device: flat y and
    v holding the blocks [I,F,ld_m] and [J,F,ld_m] one after another.
    Returns (y, v, lam, P, Ns, offsets); padding frames hold pad_value
    (0 / 1 by default for y / v)."""
    import torch
    Ns = [int(y.shape[2]) for y in ys]
    off = batch_offsets(Ns)
    I, F = ys[0].shape[:2]
    J = vs[0].shape[0]
    ld = int(off[-1])
    cdt, rdt = (torch.complex64, torch.float32) if prec == "mixed" else (torch.complex128, torch.float64)
    yt = torch.zeros(I * F * ld, dtype=cdt)
    vt = torch.ones(J * F * ld, dtype=rdt)
    if pad_value is not None:
        yt.fill_(pad_value)
        vt.fill_(pad_value)
    for m, (yb, vb) in enumerate(zip(batch_views(yt, I, F, off), batch_views(vt, J, F, off))):
        yb[:, :, :Ns[m]] = torch.from_numpy(np.ascontiguousarray(ys[m])).to(cdt)
        vb[:, :, :Ns[m]] = torch.from_numpy(np.ascontiguousarray(vs[m])).to(rdt)
    lam = torch.from_numpy(np.ascontiguousarray(np.stack(lams), dtype=np.float64))
    P = torch.from_numpy(np.ascontiguousarray(np.stack(Ps), dtype=np.complex128))
    return yt.to(device), vt.to(device), lam.to(device), P.to(device), Ns, off


class FastFCABatch:
    """FastFCA-AS estimation of M independent mixtures of uneven length in
    one set of launches, borrowed from torch tensors.

    y   flat complex64 / complex128: the blocks [I, F, ld_m] of the mixtures
        one after another (ld_m = offsets[m+1] - offsets[m], first Ns[m] used)
    v   flat real (matching y): the blocks [J, F, ld_m], updated in place
    lam [M, F, J, I] float64, P [M, F, I, I] complex128, updated in place
    I, J, F are given (the flat arrays do not carry them).
    """

    def __init__(self, y, v, lam, P, Ns, offsets=None, K: int = 1, stream=None, graph=False):
        import torch
        if not y.is_cuda:
            raise ValueError("FastFCABatch needs CUDA tensors")
        if y.dtype == torch.complex64:
            prec, vdt = FFCA_PREC_MIXED, torch.float32
        elif y.dtype == torch.complex128:
            prec, vdt = FFCA_PREC_FP64, torch.float64
        else:
            raise TypeError("y must be complex64 or complex128")
        if v.dtype != vdt or lam.dtype != torch.float64 or P.dtype != torch.complex128:
            raise TypeError("dtypes: v matches y's precision, lam float64, P complex128")
        for t in (y, v, lam, P):
            if not t.is_contiguous():
                raise ValueError("tensors must be contiguous")
        M = len(Ns)
        if lam.dim() != 4 or P.dim() != 4 or lam.shape[0] != M or P.shape[0] != M:
            raise ValueError("lam [M, F, J, I] and P [M, F, I, I] expected")
        _, F, J, I = lam.shape
        self.Ns = np.asarray(Ns, dtype=np.int32)
        self.offsets = batch_offsets(Ns) if offsets is None else np.asarray(offsets, dtype=np.int64)
        ld = int(self.offsets[-1])
        if y.dim() != 1 or v.dim() != 1 or y.numel() < I * F * ld or v.numel() < J * F * ld \
                or P.shape != (M, F, I, I):
            raise ValueError("inconsistent shapes")
        self.I, self.J, self.F, self.M, self.ld = I, J, F, M, ld
        self.y, self.v, self.lam, self.P = y, v, lam, P
        s = stream if stream is not None else torch.cuda.current_stream(y.device)
        self.stream = s
        self._off = (ctypes.c_longlong * (M + 1))(*[int(x) for x in self.offsets])
        self._n = (ctypes.c_int * M)(*[int(x) for x in self.Ns])
        d = ffca_batch_desc(I=I, J=J, F=F, M=M, K=K, prec=prec, frame_offset=self._off, N=self._n,
                            ld=ld, y=y.data_ptr(), v=v.data_ptr(), lambda_=lam.data_ptr(),
                            P=P.data_ptr(), workspace=None, workspace_bytes=0,
                            stream=s.cuda_stream)
        nbytes = ffca_batch_workspace_size(d)
        if nbytes == 0:
            raise FFCAError(1, "ffca_batch_workspace_size (invalid batch or CUDA failure: "
                               + lib().ffca_last_error().decode() + ")")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=y.device)
        d.workspace = self.workspace.data_ptr()
        d.workspace_bytes = nbytes
        self.desc = d
        self.ctx = ffca_batch_init(d)
        if graph:
            ffca_set_graph(self.ctx, True)

    def iterate(self, iters: int, trace: bool = True):
        return ffca_batch_iterate(self.ctx, iters, trace)

    def set_p_update(self, method: str = "fixed_point", mu: float = 0.0):
        """Update of P in later iterations (as FastFCA.set_p_update)."""
        ffca_set_p_update(self.ctx, method, mu)

    def nll_grad(self):
        """(NLL summed over the mixtures, dv, dlam, dPc) at the current state,
        in the batch layouts of v, lam and P; dPc = dNLL/dP^*."""
        import torch
        dv = torch.zeros_like(self.v)
        dlam = torch.empty_like(self.lam)
        dP = torch.empty_like(self.P)
        loss = ffca_nll_grad(self.ctx, dv.data_ptr(), dlam.data_ptr(), dP.data_ptr())
        return loss, dv, dlam, dP

    def wiener_se_grad(self, s):
        """(SE summed over the mixtures, dv, dlam, dPc) of sum |x^ - s|^2;
        s flat, in the layout of wiener()'s output, of y's dtype."""
        import torch
        if s.dtype != self.y.dtype or s.numel() != self.J * self.I * self.F * self.ld or not s.is_contiguous():
            raise ValueError("s must be a contiguous tensor in the batch Wiener layout of y's dtype")
        dv = torch.zeros_like(self.v)
        dlam = torch.empty_like(self.lam)
        dP = torch.empty_like(self.P)
        loss = ffca_wiener_se_grad(self.ctx, s.data_ptr(), dv.data_ptr(), dlam.data_ptr(), dP.data_ptr())
        return loss, dv, dlam, dP

    def loglik(self) -> np.ndarray:
        """L2 of every mixture (host array of M values)."""
        return ffca_batch_loglik(self.ctx, self.M)

    def set_resident(self, enable: bool = True):
        """Iterations with each problem resident on chip (ffca_set_resident)."""
        _check(self.ctx, lib().ffca_set_resident(self.ctx, 1 if enable else 0), "ffca_set_resident")

    def mask_init(self, masks, sweeps: int = 10, delta: float = 1e-3):
        """Initialise every mixture's v, lam and P in place from masks in the
        batch layout of v (ffca_mask_init)."""
        if masks.shape != self.v.shape or masks.dtype != self.v.dtype or not masks.is_contiguous():
            raise ValueError("masks must be a contiguous tensor of v's shape and dtype")
        ffca_mask_init(self.ctx, masks.data_ptr(), sweeps, delta)

    def wiener(self, out=None):
        """Multichannel Wiener filter of every mixture: flat [J I F ld] of y's
        dtype, mixture m's block [J, I, F, ld_m] at element J I F offsets[m]
        (batch_views(out, J * I, F, offsets) gives the blocks)."""
        import torch
        if out is None:
            out = torch.empty(self.J * self.I * self.F * self.ld, dtype=self.y.dtype, device=self.y.device)
        ffca_wiener(self.ctx, out.data_ptr())
        return out

    def autotune(self, rounds: int = 1):
        """Pick the fastest work partition of each pass on real iterations
        (rounds x ffca_batch_config_count() of them, advancing the estimate)."""
        return ffca_batch_autotune(self.ctx, rounds)

    def set_config(self, cand_a: int, cand_b: int):
        ffca_batch_set_config(self.ctx, cand_a, cand_b)

    def sync(self):
        ffca_sync(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            ffca_batch_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FCA:
    """Conventional FCA EM state on one GPU, borrowed from torch tensors.

    y [I, F, ld] complex64 / complex128 (CUDA), v [J, F, ld] float32 / float64
    (in place), S [F, J, I, I] complex128 Hermitian positive definite (in place).
    """

    def __init__(self, y, v, S, N: int | None = None, stream=None):
        import torch
        if y.dtype == torch.complex64:
            prec, vdt = FFCA_PREC_MIXED, torch.float32
        elif y.dtype == torch.complex128:
            prec, vdt = FFCA_PREC_FP64, torch.float64
        else:
            raise TypeError("y must be complex64 or complex128")
        if v.dtype != vdt or S.dtype != torch.complex128:
            raise TypeError("dtypes: v matches y's precision, S complex128")
        I, F, ld = y.shape
        J = v.shape[0]
        if v.shape != (J, F, ld) or S.shape != (F, J, I, I):
            raise ValueError("inconsistent shapes")
        self.y, self.v, self.S = y, v, S
        self.N = ld if N is None else int(N)
        s = stream if stream is not None else torch.cuda.current_stream(y.device)
        d = ffca_fca_desc(I=I, J=J, F=F, N=self.N, ld=ld, prec=prec, y=y.data_ptr(),
                          v=v.data_ptr(), S=S.data_ptr(), workspace=None, workspace_bytes=0,
                          stream=s.cuda_stream)
        nbytes = ffca_fca_workspace_size(d)
        if nbytes == 0 and F > 0:
            raise FFCAError(1, "ffca_fca_workspace_size")
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=y.device)
        d.workspace = self.workspace.data_ptr()
        d.workspace_bytes = nbytes
        self.desc = d
        self.ctx = ffca_fca_init(d)

    def iterate(self, iters: int, trace: bool = True):
        return ffca_fca_iterate(self.ctx, iters, trace)

    def loglik(self) -> float:
        return ffca_fca_loglik(self.ctx)

    def op_counts(self):
        return ffca_fca_op_counts(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            ffca_fca_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ autograd
def _autograd_functions():
    import torch

    def _state(y, v, lam, P, N):
        # the library borrows contiguous detached copies; the iteration state
        # of other contexts is not touched
        return FastFCA(y, v.detach().contiguous().clone(), lam.detach().contiguous().clone(),
                       P.detach().contiguous().clone(), N=N)

    class NLL(torch.autograd.Function):
        """NLL(v, lam, P) = -L2 (Eq. L2) on fixed data y; backward runs the
        adjoint kernel (posteriors recomputed)."""

        @staticmethod
        def forward(ctx, v, lam, P, y, N):
            est = _state(y, v, lam, P, N)
            loss, dv, dlam, dP = est.nll_grad()
            est.close()
            ctx.save_for_backward(dv, dlam, dP)
            return torch.tensor(loss, dtype=torch.float64, device=y.device)

        @staticmethod
        def backward(ctx, g):
            dv, dlam, dP = ctx.saved_tensors
            # torch's gradient of a real loss in a complex input is 2 dL/dz^*
            return g.to(dv.dtype) * dv, g * dlam, 2.0 * g * dP, None, None

    class WienerSE(torch.autograd.Function):
        """sum |x^_j - s_j|^2 of the Wiener estimate (Eq. MMSE0) against s."""

        @staticmethod
        def forward(ctx, v, lam, P, y, s, N):
            est = _state(y, v, lam, P, N)
            loss, dv, dlam, dP = est.wiener_se_grad(s)
            est.close()
            ctx.save_for_backward(dv, dlam, dP)
            return torch.tensor(loss, dtype=torch.float64, device=y.device)

        @staticmethod
        def backward(ctx, g):
            dv, dlam, dP = ctx.saved_tensors
            return g.to(dv.dtype) * dv, g * dlam, 2.0 * g * dP, None, None, None

    return NLL, WienerSE


_AUTOGRAD = None


def nll(v, lam, P, y, N=None):
    """Differentiable NLL = -L2 (Eq. L2) of (v, lam, P) on fixed data y
    (layouts of FastFCA).  The gradients come from the adjoint kernel; they
    are computed with the forward value (one streaming pass)."""
    global _AUTOGRAD
    if _AUTOGRAD is None:
        _AUTOGRAD = _autograd_functions()
    return _AUTOGRAD[0].apply(v, lam, P, y, N)


def wiener_se(v, lam, P, y, s, N=None):
    """Differentiable sum |x^_j - s_j|^2 of the Wiener estimate against the
    reference images s [J, I, F, ld]."""
    global _AUTOGRAD
    if _AUTOGRAD is None:
        _AUTOGRAD = _autograd_functions()
    return _AUTOGRAD[1].apply(v, lam, P, y, s, N)
