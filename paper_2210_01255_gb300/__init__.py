"""Spectral Ewald summation of Stokes potentials on NVIDIA GB300 -- Python binding of libse.

This module only marshals arguments to the C ABI declared in include/se.h; every step of
the computation runs in the CUDA kernels of libse (paper_2210_01255_gb300/csrc). There is
no CPU fallback: if the library is missing or no GPU is present, calls raise.

Method: Bagge & Tornberg, "Fast Ewald summation for Stokes flow with arbitrary
periodicity" (Sec. 2-4).
"""
import ctypes
import os

from . import build as _build

STOKESLET, ROTLET, STRESSLET, HARMONIC_FIELD, HARMONIC = 1, 2, 4, 8, 16
WIN_GAUSSIAN, WIN_KB, WIN_PKB = 0, 1, 2
FP64, FP32 = 0, 1
PART_REAL, PART_FOURIER, PART_CORR, PART_ALL = 1, 2, 4, 7
FLAG_TC_GRIDDING = 1  # se_opts.flags: FP32 gridding (P <= 16) on the tensor cores (tcgen05)
FLAG_TEST_TIMEOUT = 2  # se_opts.flags, testing aid: the tensor-core gridding's bounded waits give up at once
FLAG_REAL_BLOCKS = 4  # se_opts.flags: real-space sum with the dense-block path (k_real_blk)
FLAG_FFT_SIZES = 8  # se_opts.flags: grid extents rounded up to FFT-friendly (7-smooth) sizes
FLAG_SPLIT_POLY = 16  # se_opts.flags: D = 0 biharmonic split into (B_R - p) + p, p of degree 6
FLAG_FFT_TIMED = 32  # se_opts.flags: D = 0 extended grid sizes chosen among FFT-friendly ones by timing
KERNELS = {"stokeslet": STOKESLET, "rotlet": ROTLET, "stresslet": STRESSLET,
           "stokeslet+stresslet": STOKESLET | STRESSLET, "harmonic_field": HARMONIC_FIELD,
           "harmonic": HARMONIC}


def out_comps(kernel):
    """Output components per target and RHS: 1 for the harmonic potential, 3 otherwise."""
    return 1 if KERNELS.get(kernel, kernel) == HARMONIC else 3
WINDOWS = {"gaussian": WIN_GAUSSIAN, "kb": WIN_KB, "pkb": WIN_PKB}

SE_OK = 0
_STATUS = {0: "ok", -1: "invalid argument", -2: "coordinate out of range", -3: "out of memory",
           -4: "CUDA error", -5: "cuFFT error", -6: "device wait timed out", -7: "unsupported request",
           -8: "request exceeds a fixed capacity"}


class SeError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s: %s (%d)" % (where, _STATUS.get(code, "unknown"), code))
        self.code = code


class se_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("f_M", ctypes.c_int), ("lambda_", ctypes.c_double),
                ("Mext", ctypes.c_int * 3), ("s0", ctypes.c_double), ("s_star", ctypes.c_double),
                ("kbar_star", ctypes.c_int), ("tol_abs", ctypes.c_double), ("Q", ctypes.c_double),
                ("kernel_mask", ctypes.c_int), ("stream", ctypes.c_void_p), ("flags", ctypes.c_int),
                ("n_rc", ctypes.c_double), ("P_margin", ctypes.c_int), ("tile", ctypes.c_int)]


class se_info(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("R", ctypes.c_double), ("s0", ctypes.c_double),
                ("s_star", ctypes.c_double), ("dL", ctypes.c_double * 3), ("n", ctypes.c_int * 3),
                ("m", ctypes.c_int * 3), ("kbar_star", ctypes.c_int), ("P", ctypes.c_int),
                ("times_ms", ctypes.c_float * 8), ("launches", ctypes.c_int), ("scale_modes", ctypes.c_longlong)]


# every symbol declared in include/se.h, with its ctypes signature
_P = ctypes.c_void_p
_D3 = ctypes.POINTER(ctypes.c_double)
_I3 = ctypes.POINTER(ctypes.c_int)
SIGNATURES = {
    "se_opts_default": (ctypes.c_int, [ctypes.POINTER(se_opts)]),
    "se_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _D3, ctypes.c_double,
                                      ctypes.c_double, _I3, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(se_opts)]),
    "se_autotune": (ctypes.c_int, [ctypes.c_int, _D3, ctypes.c_int, ctypes.c_double, ctypes.c_longlong,
                                   ctypes.c_double, ctypes.POINTER(se_opts), _D3, _D3, _I3, _I3]),
    "se_autotune_timed": (ctypes.c_int, [ctypes.c_int, _D3, ctypes.c_int, ctypes.c_double, ctypes.c_longlong,
                                         _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                         ctypes.POINTER(se_opts), _D3, _D3, _I3, _I3, _D3]),
    "se_eval": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_longlong, _P, _P, ctypes.c_int,
                               ctypes.c_longlong, _P, _P]),
    "se_eval_parts": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, _P, _P,
                                     ctypes.c_int, ctypes.c_longlong, _P, _P]),
    "se_eval_host": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_longlong, _P, _P, ctypes.c_int,
                                    ctypes.c_longlong, _P, _P]),
    "se_get_info": (ctypes.c_int, [_P, ctypes.POINTER(se_info)]),
    "se_debug_grid": (ctypes.c_int, [_P, _P, ctypes.c_ulonglong]),
    "se_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "se_sync": (ctypes.c_int, [_P]),
    "se_destroy": (None, [_P]),
    "se_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "se_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P), _I3,
                                       ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                       _I3, ctypes.POINTER(_P)]),
    "se_batch_launch": (ctypes.c_int, [_P]),
    "se_plan": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _D3, ctypes.c_double, ctypes.c_double, _I3,
                               ctypes.c_int, ctypes.c_int, ctypes.POINTER(se_opts)]),
    "se_eval_batch": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _I3, ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(_P), ctypes.POINTER(_P), _I3, ctypes.POINTER(_P)]),
    "se_batch_destroy": (None, [_P]),
    "se_eval_group": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), _P, _P,
                                     ctypes.c_int, _P]),
    "se_real_noalloc": (ctypes.c_int, [ctypes.c_int, _D3, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_longlong, _P, _P, _P, _P]),
}

_lib = None


def lib(build_if_missing=True):
    """Load libse (building it first if needed). Raises if it cannot be loaded."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libse is not built (%s); run paper_2210_01255_gb300.build.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code, where):
    if code != SE_OK:
        raise SeError(code, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------ same-name thin wrappers

def se_opts_default():
    o = se_opts()
    check(lib().se_opts_default(ctypes.byref(o)), "se_opts_default")
    return o


def se_plan_create(periodicity, box, xi, rc, M, P, window, opts=None):
    h = ctypes.c_void_p()
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    m = (ctypes.c_int * 3)(*[int(v) for v in M])
    check(lib().se_plan_create(ctypes.byref(h), int(periodicity), b, float(xi), float(rc), m, int(P),
                               int(window), ctypes.byref(opts) if opts is not None else None),
          "se_plan_create")
    return h


def se_autotune(periodicity, box, kernel_mask, Q, N, tol_rel, opts=None, xi=0.0):
    o = opts if opts is not None else se_opts_default()
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    x = ctypes.c_double(float(xi))
    rc = ctypes.c_double()
    M = (ctypes.c_int * 3)()
    P = ctypes.c_int()
    check(lib().se_autotune(int(periodicity), b, int(kernel_mask), float(Q), int(N), float(tol_rel),
                            ctypes.byref(o), ctypes.byref(x), ctypes.byref(rc), M, ctypes.byref(P)),
          "se_autotune")
    return dict(xi=x.value, rc=rc.value, M=list(M), P=P.value, opts=o)


def se_autotune_timed(periodicity, box, kernel_mask, Q, src, strengths, n_rhs, tol_rel, window="pkb",
                      opts=None, prec="fp32", stream=None):
    """Parameters chosen by timing candidate plans on the given device arrays (src (N, 3)
    float64, strengths (n_rhs, N, c) in the precision prec); returns se_autotune's dict plus
    the measured time per evaluation "ms"."""
    import torch
    o = opts if opts is not None else se_opts_default()
    o.prec = FP32 if prec in ("fp32", FP32) else FP64
    if stream is None:
        stream = torch.cuda.current_stream()
    o.stream = ctypes.c_void_p(stream.cuda_stream)
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    x = ctypes.c_double()
    rc = ctypes.c_double()
    M = (ctypes.c_int * 3)()
    P = ctypes.c_int()
    ms = ctypes.c_double()
    k = KERNELS.get(kernel_mask, kernel_mask)
    src = src.contiguous()
    strengths = strengths.contiguous()  # kept alive by this name until the call returns
    check(lib().se_autotune_timed(int(periodicity), b, int(k), float(Q), src.shape[0], _ptr(src),
                                  _ptr(strengths), int(n_rhs), float(tol_rel),
                                  WINDOWS.get(window, window), ctypes.byref(o), ctypes.byref(x),
                                  ctypes.byref(rc), M, ctypes.byref(P), ctypes.byref(ms)),
          "se_autotune_timed")
    return dict(xi=x.value, rc=rc.value, M=list(M), P=P.value, opts=o, ms=ms.value)


def se_eval_parts(plan, kernel_mask, parts_mask, src, strengths, n_rhs, tgt, u):
    n_src = src.shape[0]
    n_tgt = 0 if tgt is None else tgt.shape[0]
    check(lib().se_eval_parts(plan, int(kernel_mask), int(parts_mask), n_src, _ptr(src), _ptr(strengths),
                              int(n_rhs), n_tgt, _ptr(tgt), _ptr(u)), "se_eval_parts")


def se_eval(plan, kernel_mask, src, strengths, n_rhs, tgt, u):
    se_eval_parts(plan, kernel_mask, PART_ALL, src, strengths, n_rhs, tgt, u)


def se_eval_host(plan, kernel_mask, src, strengths, n_rhs, tgt, u):
    """src, strengths, tgt, u: contiguous numpy arrays (host)."""
    n_src = src.shape[0]
    n_tgt = 0 if tgt is None else tgt.shape[0]
    p = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)
    check(lib().se_eval_host(plan, int(kernel_mask), n_src, p(src), p(strengths), int(n_rhs), n_tgt,
                             p(tgt), p(u)), "se_eval_host")


def se_get_info(plan):
    i = se_info()
    check(lib().se_get_info(plan, ctypes.byref(i)), "se_get_info")
    return i


def se_debug_grid(plan, host_array):
    check(lib().se_debug_grid(plan, ctypes.c_void_p(host_array.ctypes.data), host_array.nbytes),
          "se_debug_grid")


def se_set_timing(plan, on):
    check(lib().se_set_timing(plan, int(bool(on))), "se_set_timing")


def se_sync(plan):
    check(lib().se_sync(plan), "se_sync")


def se_destroy(plan):
    lib().se_destroy(plan)


def se_real_noalloc(periodicity, box, xi, rc, kernel_mask, prec, src, strengths, u, stream=None):
    """Allocation-free real-space sum (star form, one RHS) into u; see include/se.h."""
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    check(lib().se_real_noalloc(int(periodicity), b, float(xi), float(rc), int(kernel_mask), int(prec),
                                src.shape[0], _ptr(src), _ptr(strengths), _ptr(u),
                                None if stream is None else ctypes.c_void_p(stream.cuda_stream)),
          "se_real_noalloc")


def se_batch_create(plans, kernel_masks, srcs, strengths, n_rhs, us):
    """Record the evaluations of several configurations (star form) into one CUDA graph.
    plans: handles sharing one non-default stream; srcs / strengths / us: torch device tensors."""
    n = len(plans)
    h = ctypes.c_void_p()
    arr = lambda t, vals: (t * n)(*vals)
    check(lib().se_batch_create(ctypes.byref(h), n, arr(ctypes.c_void_p, [p.value for p in plans]),
                                arr(ctypes.c_int, [int(k) for k in kernel_masks]),
                                arr(ctypes.c_longlong, [int(s.shape[0]) for s in srcs]),
                                arr(ctypes.c_void_p, [s.data_ptr() for s in srcs]),
                                arr(ctypes.c_void_p, [f.data_ptr() for f in strengths]),
                                arr(ctypes.c_int, [int(r) for r in n_rhs]),
                                arr(ctypes.c_void_p, [u.data_ptr() for u in us])), "se_batch_create")
    return h


def se_eval_batch(plans, kernel_masks, srcs, strengths, n_rhs, us):
    """Evaluate several independent configurations (star form) in one call, each on its
    plan's stream. plans: handles; srcs / strengths / us: torch device tensors."""
    n = len(plans)
    arr = lambda t, vals: (t * n)(*vals)
    check(lib().se_eval_batch(arr(ctypes.c_void_p, [p.value for p in plans]), n,
                              arr(ctypes.c_int, [int(KERNELS.get(k, k)) for k in kernel_masks]),
                              arr(ctypes.c_longlong, [int(s.shape[0]) for s in srcs]),
                              arr(ctypes.c_void_p, [s.data_ptr() for s in srcs]),
                              arr(ctypes.c_void_p, [f.data_ptr() for f in strengths]),
                              arr(ctypes.c_int, [int(r) for r in n_rhs]),
                              arr(ctypes.c_void_p, [u.data_ptr() for u in us])), "se_eval_batch")


def se_eval_group(plan, kernel_mask, n_src, src, strengths, n_rhs, u):
    """Several independent configurations on one plan in one evaluation (star form). n_src:
    the configurations' point counts; src (sum n_src, 3), strengths (per configuration an
    [n_rhs][N_c][c] block, concatenated) and u (per configuration an [n_rhs][N_c][out] block,
    concatenated): contiguous torch device tensors (or raw device addresses)."""
    n = len(n_src)
    ptr = lambda t: ctypes.c_void_p(t if isinstance(t, int) else t.data_ptr())
    check(lib().se_eval_group(plan, int(KERNELS.get(kernel_mask, kernel_mask)), n,
                              (ctypes.c_longlong * n)(*[int(v) for v in n_src]), ptr(src), ptr(strengths),
                              int(n_rhs), ptr(u)), "se_eval_group")


def se_batch_launch(batch):
    check(lib().se_batch_launch(batch), "se_batch_launch")


def se_batch_destroy(batch):
    lib().se_batch_destroy(batch)


def se_status_str(code):
    return lib().se_status_str(int(code)).decode()


# -------------------------------------------------------------- convenience wrapper

class Plan:
    """A plan bound to torch's current CUDA stream (memory via torch, compute via libse)."""

    def __init__(self, periodicity, box, xi, rc, M, P, window="pkb", prec="fp64", opts=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libse needs a CUDA GPU")
        o = opts if opts is not None else se_opts_default()
        o.prec = FP32 if prec in ("fp32", FP32) else FP64
        if stream is None:
            stream = torch.cuda.current_stream()
        o.stream = ctypes.c_void_p(stream.cuda_stream)
        self.stream = stream
        self.dtype = torch.float32 if o.prec == FP32 else torch.float64
        self.periodicity = periodicity
        self.handle = se_plan_create(periodicity, box, xi, rc, M, P,
                                     WINDOWS.get(window, window), o)

    def evaluate(self, kernel, x, f, targets=None, parts=PART_ALL, out=None):
        """x: (N,3) float64 cuda; f: (n_rhs, N, c) or (N, c) in the plan dtype; returns u."""
        import torch
        k = KERNELS.get(kernel, kernel)
        single = f.dim() == 2
        f3 = f.unsqueeze(0) if single else f
        n_rhs = f3.shape[0]
        nt = x.shape[0] if targets is None else targets.shape[0]
        if out is None:
            out = torch.empty((n_rhs, nt, out_comps(k)), dtype=self.dtype, device=x.device)
        se_eval_parts(self.handle, k, parts, x.contiguous(), f3.contiguous(), n_rhs,
                      None if targets is None else targets.contiguous(), out)
        return out[0] if single else out

    def info(self):
        return se_get_info(self.handle)

    def sync(self):
        se_sync(self.handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.se_destroy(h)
            self.handle = None
