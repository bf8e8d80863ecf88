"""Thin ctypes binding over ``libfmm_gb300.so`` (the C ABI declared in include/fmm.h).

Argument marshalling only: every step of the multiply runs in the library's
CUDA kernels.  PyTorch supplies device memory (the workspace, and the operand
tensors a caller passes in) and the current CUDA stream.  Importing this
module loads the library and raises if it has not been built: there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

FMM_OK = 0
FMM_ERR_INVALID_ARG = 1
FMM_ERR_UNSUPPORTED = 6
FMM_ERR_TIMEOUT = 7
STATUS_NAMES = {0: "FMM_OK", 1: "FMM_ERR_INVALID_ARG", 2: "FMM_ERR_ALIGNMENT", 3: "FMM_ERR_SHAPE_MISMATCH",
                4: "FMM_ERR_OOM", 5: "FMM_ERR_CUDA", 6: "FMM_ERR_UNSUPPORTED", 7: "FMM_ERR_TIMEOUT",
                8: "FMM_ERR_NO_DEVICE", 9: "FMM_ERR_WORKSPACE"}
PRECISIONS = {"fp32": 0, "tf32": 1, "bf16x3": 2, "fp16x3": 3}
ODD = {"pad": 0, "peel": 1, "tile": 2, "auto": 3}
PLANNERS = {"fixed": 0, "exhaustive": 1, "mlp": 2}
ALGOS = {"winograd": 0, "classical": 1}


class FmmError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = f"{where}: {STATUS_NAMES.get(status, status)}"
        try:
            detail = _lib.fmm_last_error().decode()
            if detail:
                msg += f" ({detail})"
        except Exception:
            pass
        super().__init__(msg)


class Options(C.Structure):
    _fields_ = [("depth", C.c_int), ("cutoff", C.c_int), ("leaf_tile", C.c_int), ("precision", C.c_int),
                ("odd", C.c_int), ("planner", C.c_int), ("algo", C.c_int), ("host_operands", C.c_int),
                ("refine_fp64", C.c_int), ("fuse_last", C.c_int), ("host_copy", C.c_int)]


def _load():
    path = _build.LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -m paper_1205_2927_gb300.build)")
    lib = C.CDLL(path)
    i64, vp, sz = C.c_int64, C.c_void_p, C.c_size_t
    lib.fmm_options_default.argtypes = [C.POINTER(Options)]
    lib.fmm_options_default.restype = C.c_int
    lib.fmm_plan.argtypes = [C.POINTER(vp), i64, i64, i64, i64, i64, i64, C.POINTER(Options), vp, sz,
                             C.POINTER(sz), vp]
    lib.fmm_plan.restype = C.c_int
    lib.fmm_gemm.argtypes = [vp, C.c_float, vp, vp, C.c_float, vp, vp]
    lib.fmm_gemm.restype = C.c_int
    lib.fmm_gemm_batched.argtypes = [C.c_int, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(vp),
                                     C.POINTER(i64), C.POINTER(vp), C.POINTER(i64), C.POINTER(vp),
                                     C.POINTER(i64), C.POINTER(C.c_float), C.POINTER(C.c_float),
                                     C.POINTER(Options), vp, sz, C.POINTER(sz), vp]
    lib.fmm_gemm_batched.restype = C.c_int
    lib.fmm_free.argtypes = [vp]
    lib.fmm_free.restype = None
    lib.fmm_status_string.argtypes = [C.c_int]
    lib.fmm_status_string.restype = C.c_char_p
    lib.fmm_last_error.argtypes = []
    lib.fmm_last_error.restype = C.c_char_p
    lib.fmm_get_device_status.argtypes = [vp]
    lib.fmm_get_device_status.restype = C.c_int
    lib.fmm_plan_info.argtypes = [vp] + [C.POINTER(C.c_int)] * 5
    lib.fmm_plan_info.restype = C.c_int
    lib.fmm_plan_fuse_last.argtypes = [vp, C.POINTER(C.c_int)]
    lib.fmm_plan_fuse_last.restype = C.c_int
    lib.fmm_plan_host_copy.argtypes = [vp, C.POINTER(C.c_int)]
    lib.fmm_plan_host_copy.restype = C.c_int
    lib.fmm_plan_profile.argtypes = [vp, C.c_int]
    lib.fmm_plan_profile.restype = C.c_int
    lib.fmm_plan_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), C.POINTER(i64), C.POINTER(i64)]
    lib.fmm_plan_profile_read.restype = C.c_int
    lib.fmm_plan_phase_bytes.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.fmm_plan_phase_bytes.restype = C.c_int
    lib.fmm_wait_selftest.argtypes = [vp, i64, vp]
    lib.fmm_wait_selftest.restype = C.c_int
    lib.fmm_residual.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, vp, vp, sz, C.POINTER(sz), C.c_int, vp]
    lib.fmm_residual.restype = C.c_int
    lib.fmm_gemm_static.argtypes = [i64, i64, i64, C.c_float, vp, i64, vp, i64, C.c_float, vp, i64, vp]
    lib.fmm_gemm_static.restype = C.c_int
    lib.fmm_gemm_static_status.argtypes = [vp]
    lib.fmm_gemm_static_status.restype = C.c_int
    lib.fmm_tensor_peak.argtypes = [C.c_int, i64, vp, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
    lib.fmm_tensor_peak.restype = C.c_int
    return lib


_lib = _load()


def library():
    return _lib


def _check(status, where):
    if status != FMM_OK:
        raise FmmError(status, where)


HOST_COPY = {"default": 0, "engine": 1, "sm": 2}


def options(depth=-1, cutoff=2048, leaf_tile=0, precision="fp32", odd="auto", planner="fixed",
            algo="winograd", host_operands=0, refine_fp64=0, fuse_last=0, host_copy="default") -> Options:
    o = Options()
    _check(_lib.fmm_options_default(C.byref(o)), "fmm_options_default")
    o.depth, o.cutoff, o.leaf_tile = depth, cutoff, leaf_tile
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.odd = ODD[odd] if isinstance(odd, str) else int(odd)
    o.planner = PLANNERS[planner] if isinstance(planner, str) else int(planner)
    o.algo = ALGOS[algo] if isinstance(algo, str) else int(algo)
    o.host_operands, o.refine_fp64 = host_operands, refine_fp64
    o.fuse_last = int(fuse_last)
    o.host_copy = HOST_COPY[host_copy] if isinstance(host_copy, str) else int(host_copy)
    return o


def _ld(t):
    """Leading dimension (row stride, elements) of a 2-D row-major operand; an
    empty operand is never read, so any valid value will do (numpy-backed empty
    tensors carry stride 0)."""
    return max(t.stride(0), 1) if t.numel() > 0 else max(t.shape[1], 1)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------------ same names as the C ABI

def fmm_plan(M, N, K, lda, ldb, ldc, opt=None, workspace=None, workspace_bytes=0, stream=None, query_only=False):
    """Returns (plan_handle or None, workspace_needed)."""
    need = C.c_size_t(0)
    if query_only:
        _check(_lib.fmm_plan(None, M, N, K, lda, ldb, ldc, C.byref(opt) if opt else None, None, 0,
                             C.byref(need), None), "fmm_plan(query)")
        return None, need.value
    h = C.c_void_p()
    _check(_lib.fmm_plan(C.byref(h), M, N, K, lda, ldb, ldc, C.byref(opt) if opt else None,
                         C.c_void_p(workspace), workspace_bytes, C.byref(need), _stream_ptr(stream)),
           "fmm_plan")
    return h, need.value


def fmm_gemm(plan, alpha, A_ptr, B_ptr, beta, C_ptr, stream=None):
    _check(_lib.fmm_gemm(plan, C.c_float(alpha), C.c_void_p(A_ptr), C.c_void_p(B_ptr), C.c_float(beta),
                         C.c_void_p(C_ptr), _stream_ptr(stream)), "fmm_gemm")


def fmm_free(plan):
    _lib.fmm_free(plan)


def fmm_get_device_status(plan):
    return _lib.fmm_get_device_status(plan)


def fmm_plan_info(plan):
    vals = [C.c_int() for _ in range(5)]
    _check(_lib.fmm_plan_info(plan, *[C.byref(v) for v in vals]), "fmm_plan_info")
    return dict(zip(("depth", "leaf_tile", "precision", "odd", "algo"), [v.value for v in vals]))


def fmm_plan_host_copy(plan):
    """1: the plan's next call moves host operands with the copy engines, 2: with
    SM loads and stores, 0: device-resident plan."""
    m = C.c_int()
    _check(_lib.fmm_plan_host_copy(plan, C.byref(m)), "fmm_plan_host_copy")
    return m.value


def fmm_plan_fuse_last(plan):
    f = C.c_int()
    _check(_lib.fmm_plan_fuse_last(plan, C.byref(f)), "fmm_plan_fuse_last")
    return bool(f.value)


def fmm_plan_profile(plan, enable=True):
    _check(_lib.fmm_plan_profile(plan, int(bool(enable))), "fmm_plan_profile")


def fmm_plan_profile_read(plan):
    v = [C.c_double() for _ in range(3)] + [C.c_int64(), C.c_int64()]
    _check(_lib.fmm_plan_profile_read(plan, *[C.byref(x) for x in v]), "fmm_plan_profile_read")
    return dict(pre_ms=v[0].value, leaf_ms=v[1].value, post_ms=v[2].value, launches=v[3].value, calls=v[4].value)


def fmm_residual(A, B, Cm, x, fp64=False, stream=None):
    """Freivalds residual r = Cm x - A (B x) of device tensors (row-major, unit
    column stride; x: N float32 entries); returns r (M float64 entries, device)."""
    import torch
    M, K = A.shape
    N = B.shape[1]
    need = C.c_size_t(0)
    _check(_lib.fmm_residual(M, N, K, None, _ld(A), None, _ld(B), None,
                             _ld(Cm), None, None, None, 0, C.byref(need), int(fp64), None),
           "fmm_residual(query)")
    ws = torch.empty(max(need.value, 256), dtype=torch.uint8, device=A.device)
    r = torch.empty(M, dtype=torch.float64, device=A.device)
    _check(_lib.fmm_residual(M, N, K, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B),
                             Cm.data_ptr(), _ld(Cm), x.data_ptr(), r.data_ptr(), ws.data_ptr(),
                             ws.numel(), C.byref(need), int(fp64), _stream_ptr(stream)), "fmm_residual")
    return r


def _check_static_operands(A, B, Cm):
    """Shape, dtype, device and layout checks of fmm_gemm_static's tensors, made
    before any call into the library: M, N, K are taken from A and B, so a short
    B or a small C would otherwise be read or written past its end."""
    import torch
    for name, t in (("A", A), ("B", B), ("C", Cm)):
        if t.dim() != 2:
            raise ValueError(f"fmm_gemm_static: {name} must be a 2-D tensor")
    M, K = A.shape
    if B.shape[0] != K:
        raise ValueError(f"fmm_gemm_static: B has {B.shape[0]} rows, A has {K} columns")
    if tuple(Cm.shape) != (M, B.shape[1]):
        raise ValueError(f"fmm_gemm_static: C is {tuple(Cm.shape)}, expected {(M, B.shape[1])}")
    for name, t in (("A", A), ("B", B), ("C", Cm)):
        if t.dtype != torch.float32:
            raise TypeError(f"fmm_gemm_static: {name} must be float32, got {t.dtype}")
        if not t.is_cuda:
            raise ValueError(f"fmm_gemm_static: {name} must be a CUDA tensor")
        if t.shape[0] > 0 and t.shape[1] > 1 and t.stride(1) != 1:
            raise ValueError(f"fmm_gemm_static: {name} must have unit column stride")


def fmm_gemm_static(A, B, Cm, alpha=1.0, beta=0.0, stream=None):
    """Cm <- alpha A B + beta Cm through the allocation-free entry point (device
    float32 tensors, row-major, unit column stride; M, N, K <= 1024)."""
    _check_static_operands(A, B, Cm)
    M, K = A.shape
    N = B.shape[1]
    _check(_lib.fmm_gemm_static(M, N, K, float(alpha), A.data_ptr(), _ld(A), B.data_ptr(),
                                _ld(B), float(beta), Cm.data_ptr(), _ld(Cm),
                                _stream_ptr(stream)), "fmm_gemm_static")
    return Cm


def fmm_gemm_static_status(stream=None):
    """Device status of the last fmm_gemm_static call (synchronises `stream`)."""
    return _lib.fmm_gemm_static_status(_stream_ptr(stream))


def fmm_tensor_peak(kind="tf32", batches=20000, seed=1, stream=None):
    """Tensor-pipe rate of this GPU in TFLOP/s (measurement helper): back-to-back
    tcgen05.mma of the leaf kernel's shape on shared-memory tiles filled with
    uniform random values.  Returns (tflops, ms of the timed launch)."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    fill = (torch.rand(16384, generator=g) * 2 - 1).cuda()
    tf, ms = C.c_double(), C.c_double()
    _check(_lib.fmm_tensor_peak({"tf32": 0, "bf16": 1}[kind], int(batches), fill.data_ptr(), C.byref(tf),
                                C.byref(ms), _stream_ptr(stream)), "fmm_tensor_peak")
    return tf.value, ms.value


def fmm_plan_phase_bytes(plan):
    pre, post = C.c_double(), C.c_double()
    _check(_lib.fmm_plan_phase_bytes(plan, C.byref(pre), C.byref(post)), "fmm_plan_phase_bytes")
    return dict(pre_bytes=pre.value, post_bytes=post.value)


# ------------------------------------------------------------------ convenience over torch tensors

class Plan:
    """A plan plus the workspace it owns (a torch uint8 device tensor)."""

    def __init__(self, M, N, K, lda=None, ldb=None, ldc=None, device=None, stream=None, **opt_kwargs):
        import torch
        self.M, self.N, self.K = int(M), int(N), int(K)
        self.lda = int(lda if lda is not None else max(K, 1))
        self.ldb = int(ldb if ldb is not None else max(N, 1))
        self.ldc = int(ldc if ldc is not None else max(N, 1))
        self.opt = options(**opt_kwargs)
        _, need = fmm_plan(self.M, self.N, self.K, self.lda, self.ldb, self.ldc, self.opt, query_only=True)
        self.workspace_bytes = need
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
        self.handle, _ = fmm_plan(self.M, self.N, self.K, self.lda, self.ldb, self.ldc, self.opt,
                                  self.workspace.data_ptr(), self.workspace.numel(), stream)
        self.info = fmm_plan_info(self.handle)
        self.info["fuse_last"] = fmm_plan_fuse_last(self.handle)

    def __call__(self, A, B, C=None, alpha=1.0, beta=0.0, stream=None):
        import torch
        if C is None:
            C = (torch.empty((self.M, self.ldc), dtype=torch.float32).pin_memory() if self.opt.host_operands
                 else torch.empty((self.M, self.ldc), dtype=torch.float32, device=A.device))[:, : self.N]
        for t in (A, B, C):
            assert t.dtype == torch.float32
            assert t.is_cuda or (self.opt.host_operands and t.is_pinned()), \
                "operands must be CUDA tensors (or pinned host tensors with host_operands=1)"
        fmm_gemm(self.handle, alpha, A.data_ptr(), B.data_ptr(), beta, C.data_ptr(), stream)
        return C

    def device_status(self):
        return fmm_get_device_status(self.handle)

    def profile(self, enable=True):
        fmm_plan_profile(self.handle, enable)

    def profile_read(self):
        return fmm_plan_profile_read(self.handle)

    def host_copy(self):
        """How the next call moves host operands: "engine", "sm" or None (device plan)."""
        return {0: None, 1: "engine", 2: "sm"}[fmm_plan_host_copy(self.handle)]

    def wait_selftest(self, limit_ns=20_000_000, stream=None):
        """Run the device-wait failure path once (see fmm_wait_selftest)."""
        _check(_lib.fmm_wait_selftest(self.handle, int(limit_ns), _stream_ptr(stream)), "fmm_wait_selftest")

    def phase_bytes(self):
        """Algorithmic bytes of the last call's addition phases (pre_bytes, post_bytes)."""
        return fmm_plan_phase_bytes(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fmm_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def matmul(A, B, depth=-1, precision="fp32", **kw):
    """C = A @ B for contiguous float32 CUDA tensors via a one-off plan."""
    M, K = A.shape
    N = B.shape[1]
    p = Plan(M, N, K, _ld(A), _ld(B), N, depth=depth, precision=precision, **kw)
    return p(A, B)


# ------------------------------------------------------------------ batched

def _batched_argtypes():
    i64p, vpp = C.POINTER(C.c_int64), C.POINTER(C.c_void_p)
    fp = C.POINTER(C.c_float)
    common = [C.c_int, i64p, i64p, i64p, vpp, i64p, vpp, i64p, vpp, i64p, fp, fp, C.POINTER(Options),
              C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t), C.c_void_p]
    _lib.fmm_batched_plan.argtypes = [C.POINTER(C.c_void_p)] + common
    _lib.fmm_batched_plan.restype = C.c_int
    _lib.fmm_batched_run.argtypes = [C.c_void_p, C.c_void_p]
    _lib.fmm_batched_run.restype = C.c_int
    _lib.fmm_batched_free.argtypes = [C.c_void_p]
    _lib.fmm_batched_free.restype = None
    _lib.fmm_batched_info.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    _lib.fmm_batched_info.restype = C.c_int
    _lib.fmm_batched_classes.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    _lib.fmm_batched_classes.restype = C.c_int


_batched_argtypes()


class BatchedPlan:
    """Batched products C_i = alpha_i A_i B_i + beta_i C_i over lists of 2-D float32
    CUDA tensors (row-major, unit column stride).  run() only launches kernels,
    so it can be captured in a CUDA graph."""

    def __init__(self, As, Bs, Cs, alpha=1.0, beta=0.0, stream=None, **opt_kwargs):
        import torch
        n = len(As)
        self.count = n
        self._keep = (list(As), list(Bs), list(Cs))
        i64 = C.c_int64 * n
        vp = C.c_void_p * n
        f = C.c_float * n
        al = [alpha] * n if not isinstance(alpha, (list, tuple)) else alpha
        be = [beta] * n if not isinstance(beta, (list, tuple)) else beta
        self._arrs = (i64(*[a.shape[0] for a in As]), i64(*[b.shape[1] for b in Bs]), i64(*[a.shape[1] for a in As]),
                      vp(*[a.data_ptr() for a in As]), i64(*[_ld(a) for a in As]),
                      vp(*[b.data_ptr() for b in Bs]), i64(*[_ld(b) for b in Bs]),
                      vp(*[c.data_ptr() for c in Cs]), i64(*[_ld(c) for c in Cs]),
                      f(*al), f(*be))
        self.opt = options(**opt_kwargs)
        need = C.c_size_t(0)
        _check(_lib.fmm_batched_plan(None, n, *self._arrs, C.byref(self.opt), None, 0, C.byref(need), None),
               "fmm_batched_plan(query)")
        self.workspace = torch.empty(max(need.value, 256), dtype=torch.uint8, device=As[0].device if n else "cuda")
        self.handle = C.c_void_p()
        _check(_lib.fmm_batched_plan(C.byref(self.handle), n, *self._arrs, C.byref(self.opt),
                                     C.c_void_p(self.workspace.data_ptr()), self.workspace.numel(), C.byref(need),
                                     _stream_ptr(stream)), "fmm_batched_plan")

    def run(self, stream=None):
        _check(_lib.fmm_batched_run(self.handle, _stream_ptr(stream)), "fmm_batched_run")

    def info(self):
        d = (C.c_int * max(self.count, 1))()
        t, l = C.c_int64(), C.c_int64()
        _check(_lib.fmm_batched_info(self.handle, d, C.byref(t), C.byref(l)), "fmm_batched_info")
        cl = (C.c_int * max(self.count, 1))()
        nc, tile = C.c_int(), C.c_int()
        _check(_lib.fmm_batched_classes(self.handle, cl, C.byref(nc), C.byref(tile)), "fmm_batched_classes")
        return dict(depths=list(d)[: self.count], total_tiles=t.value, launches=l.value,
                    classes=list(cl)[: self.count], nclasses=nc.value, leaf_tile=tile.value)

    def close(self):
        if getattr(self, "handle", None):
            _lib.fmm_batched_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ remaining C-ABI names

def fmm_options_default():
    """The library's default options (depth -1, cut-off 2048, FP32, PAD, FIXED, Winograd)."""
    o = Options()
    _check(_lib.fmm_options_default(C.byref(o)), "fmm_options_default")
    return o


def fmm_status_string(status):
    return _lib.fmm_status_string(int(status)).decode()


def fmm_last_error():
    return _lib.fmm_last_error().decode()


def fmm_wait_selftest(plan, limit_ns=20_000_000, stream=None):
    _check(_lib.fmm_wait_selftest(plan, int(limit_ns), _stream_ptr(stream)), "fmm_wait_selftest")


def fmm_batched_plan(As, Bs, Cs, alpha=1.0, beta=0.0, stream=None, **opt_kwargs):
    """Plan for the batched products C_i = alpha_i A_i B_i + beta_i C_i (a BatchedPlan)."""
    return BatchedPlan(As, Bs, Cs, alpha=alpha, beta=beta, stream=stream, **opt_kwargs)


def fmm_batched_run(bplan, stream=None):
    bplan.run(stream)


def fmm_batched_info(bplan):
    return bplan.info()


def fmm_batched_classes(bplan):
    i = bplan.info()
    return dict(classes=i["classes"], nclasses=i["nclasses"], leaf_tile=i["leaf_tile"])


def fmm_batched_free(bplan):
    bplan.close()


def fmm_gemm_batched(As, Bs, Cs, alpha=1.0, beta=0.0, stream=None, **opt_kwargs):
    """One-shot batched call (plan, run on `stream`, release the host state)."""
    import torch
    n = len(As)
    i64, vp, f = C.c_int64 * n, C.c_void_p * n, C.c_float * n
    al = [alpha] * n if not isinstance(alpha, (list, tuple)) else alpha
    be = [beta] * n if not isinstance(beta, (list, tuple)) else beta
    arrs = (i64(*[a.shape[0] for a in As]), i64(*[b.shape[1] for b in Bs]), i64(*[a.shape[1] for a in As]),
            vp(*[a.data_ptr() for a in As]), i64(*[_ld(a) for a in As]),
            vp(*[b.data_ptr() for b in Bs]), i64(*[_ld(b) for b in Bs]),
            vp(*[c.data_ptr() for c in Cs]), i64(*[_ld(c) for c in Cs]), f(*al), f(*be))
    opt = options(**opt_kwargs)
    need = C.c_size_t(0)
    _check(_lib.fmm_gemm_batched(n, *arrs, C.byref(opt), None, 0, C.byref(need), None), "fmm_gemm_batched(query)")
    ws = torch.empty(max(need.value, 256), dtype=torch.uint8, device=As[0].device if n else "cuda")
    _check(_lib.fmm_gemm_batched(n, *arrs, C.byref(opt), C.c_void_p(ws.data_ptr()), ws.numel(), C.byref(need),
                                 _stream_ptr(stream)), "fmm_gemm_batched")
    return ws   # the device tables live in the workspace until the launch has run


# ------------------------------------------------------------------ planner / cost model

NPARAM = 4673


def _planner_argtypes():
    vp, i64, sz = C.c_void_p, C.c_int64, C.c_size_t
    ip, fp = C.POINTER(C.c_int), C.POINTER(C.c_float)
    _lib.fmm_autotune.argtypes = [i64, i64, i64, C.POINTER(Options), vp, vp, vp, vp, sz, C.POINTER(sz), ip, ip, fp,
                                  ip, C.c_int, vp]
    _lib.fmm_autotune.restype = C.c_int
    _lib.fmm_plan_features.argtypes = [i64, i64, i64, C.c_int, C.c_int, C.c_int, fp]
    _lib.fmm_plan_features.restype = C.c_int
    _lib.fmm_mlp_forward.argtypes = [vp, vp, vp, C.c_int, vp]
    _lib.fmm_mlp_forward.restype = C.c_int
    _lib.fmm_mlp_train_step.argtypes = [vp, vp, vp, C.c_int, C.c_float, vp, vp, C.c_int, vp, sz, C.POINTER(sz), vp,
                                        vp, vp]
    _lib.fmm_mlp_train_step.restype = C.c_int
    _lib.fmm_set_cost_model.argtypes = [fp, fp, fp]
    _lib.fmm_set_cost_model.restype = C.c_int


_planner_argtypes()


def fmm_autotune(M, N, K, A, B, Cmat, reps=1, stream=None, **opt_kwargs):
    """Time every candidate plan on device tensors A, B, C (C is overwritten).
    Returns a list of (depth, leaf_tile, milliseconds)."""
    import torch
    opt = options(**opt_kwargs)
    need = C.c_size_t(0)
    n = C.c_int(0)
    _check(_lib.fmm_autotune(M, N, K, C.byref(opt), None, None, None, None, 0, C.byref(need), None, None, None,
                             C.byref(n), reps, None), "fmm_autotune(query)")
    ws = torch.empty(max(need.value, 256), dtype=torch.uint8, device=A.device)
    d, t, ms = (C.c_int * 16)(), (C.c_int * 16)(), (C.c_float * 16)()
    _check(_lib.fmm_autotune(M, N, K, C.byref(opt), A.data_ptr(), B.data_ptr(), Cmat.data_ptr(), ws.data_ptr(),
                             ws.numel(), C.byref(need), d, t, ms, C.byref(n), reps, _stream_ptr(stream)),
           "fmm_autotune")
    return [(d[i], t[i], ms[i]) for i in range(n.value)]


def fmm_plan_features(M, N, K, depth, leaf_tile, precision=0):
    out = (C.c_float * 6)()
    _check(_lib.fmm_plan_features(M, N, K, depth, leaf_tile, precision, out), "fmm_plan_features")
    return list(out)


def fmm_mlp_forward(params, X, Y, stream=None):
    _check(_lib.fmm_mlp_forward(params.data_ptr(), X.data_ptr(), Y.data_ptr(), X.shape[0], _stream_ptr(stream)),
           "fmm_mlp_forward")


def fmm_mlp_train_step(params, m, v, step, lr, X, T, workspace, grad_out=None, loss_out=None, stream=None):
    _check(_lib.fmm_mlp_train_step(params.data_ptr(), m.data_ptr(), v.data_ptr(), step, lr, X.data_ptr(),
                                   T.data_ptr(), X.shape[0], workspace.data_ptr(), workspace.numel(), None,
                                   grad_out.data_ptr() if grad_out is not None else None,
                                   loss_out.data_ptr() if loss_out is not None else None, _stream_ptr(stream)),
           "fmm_mlp_train_step")


def mlp_workspace_bytes(batch):
    need = C.c_size_t(0)
    _check(_lib.fmm_mlp_train_step(None, None, None, 1, 0.0, None, None, batch, None, 0, C.byref(need), None, None,
                                   None), "fmm_mlp_train_step(query)")
    return need.value


def fmm_set_cost_model(params=None, mean=None, std=None):
    if params is None:
        _check(_lib.fmm_set_cost_model(None, None, None), "fmm_set_cost_model")
        return
    P = (C.c_float * NPARAM)(*[float(x) for x in params])
    Mn = (C.c_float * 6)(*[float(x) for x in mean])
    Sd = (C.c_float * 6)(*[float(x) for x in std])
    _check(_lib.fmm_set_cost_model(P, Mn, Sd), "fmm_set_cost_model")
