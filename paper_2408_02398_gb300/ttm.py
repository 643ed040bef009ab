"""Python binding of libttm (include/ttm.h): argument marshalling only.

Every function keeps the name of the C entry point it calls and takes
PyTorch tensors for device buffers (PyTorch provides device memory and
streams; every computation runs in the library's CUDA kernels). The library
must have been built (``paper_2408_02398_gb300.build.build()``); importing
this module without it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libttm.so")

TTM_OK = 0
STATUS = {0: "TTM_OK", 1: "TTM_E_INVALID_ARG", 2: "TTM_E_SHAPE", 3: "TTM_E_UNSUPPORTED", 4: "TTM_E_OOM",
          5: "TTM_E_CUDA", 6: "TTM_E_TIMEOUT", 7: "TTM_E_INTERNAL"}
TTM_PREC_FP32, TTM_PREC_FP16_SPECTRA, TTM_PREC_BF16_SPECTRA = 0, 1, 2
TTM_MAX_PLAIN, TTM_MAX_MLP_WARM = 0, 1
TTM_LOCALSUM_FP64, TTM_LOCALSUM_DF64 = 0, 1
TTM_MLP_FP32, TTM_MLP_BF16 = 0, 1
TTM_BATCH_AUTOTUNE, TTM_BATCH_LOCALSUM_DF64 = 1, 2

# every symbol include/ttm.h declares
EXPORTS = ["ttm_default_params", "ttm_ctx_create", "ttm_ctx_destroy", "ttm_ctx_set_wait_limit", "ttm_ctx_device_status", "ttm_last_error", "ttm_num_components",
           "ttm_version", "ttm_rotation_set", "ttm_build_tensor_field", "ttm_plan_create", "ttm_plan_destroy",
           "ttm_plan_components", "ttm_plan_valid_box", "ttm_correlate", "ttm_plan_copy_w", "ttm_peak_map",
           "ttm_find_peaks", "tm_correlate", "ttm_plan_enable_timing", "ttm_plan_stage_times", "ttm_num_stages",
           "ttm_stage_name", "ttm_kernel_launches", "ttm_plan_set_localsum",
           "ttm_find_peaks_noalloc", "ttm_plan_fallback_count", "ttm_mlp_num_params", "ttm_mlp_create",
           "ttm_mlp_destroy", "ttm_mlp_inputs", "ttm_mlp_get_params", "ttm_mlp_set_params", "ttm_mlp_forward",
           "ttm_mlp_loss_grad", "ttm_mlp_train", "ttm_mlp_set_precision", "ttm_mlp_infer", "ttm_mlp_make_pairs", "ttm_mlp_save",
           "ttm_mlp_load", "ttm_plan_create_padded", "ttm_autotune_shape", "ttm_autotune_entries",
           "ttm_autotune_save", "ttm_autotune_load", "ttm_batch_create", "ttm_batch_run", "ttm_batch_work_shape",
           "ttm_batch_destroy", "ttm_refine_peaks", "ttm_slab_ranges", "ttm_merge_peaks", "ttm_blocked_peaks",
           "ttm_blocked_create", "ttm_blocked_run", "ttm_blocked_destroy"]


class TTMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(code, str(code)), msg))
        self.code = code


class ttm_field_params(C.Structure):
    _fields_ = [("order_n", C.c_int), ("dprime", C.c_int), ("mask_radius", C.c_double),
                ("mask_soft_width", C.c_double), ("filter_a", C.c_double), ("n_rot_base", C.c_int64),
                ("cube_symmetrize", C.c_int)]


_lib = None
_vp = C.c_void_p
_i = C.c_int
_i64 = C.c_int64
_d = C.c_double


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libttm.so is not built (run paper_2408_02398_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        sig = {
            "ttm_default_params": (None, [C.POINTER(ttm_field_params)]),
            "ttm_ctx_create": (_i, [_i, C.POINTER(_vp)]),
            "ttm_ctx_destroy": (None, [_vp]),
            "ttm_ctx_set_wait_limit": (_i, [_vp, _i64]),
            "ttm_ctx_device_status": (_i, [_vp, _vp]),
            "ttm_last_error": (C.c_char_p, [_vp]),
            "ttm_num_components": (_i, [_i, _i]),
            "ttm_version": (C.c_char_p, []),
            "ttm_rotation_set": (_i, [_i64, _i, _vp]),
            "ttm_build_tensor_field": (_i, [_vp, _vp, _i, _i, _i, C.POINTER(ttm_field_params), _vp, _vp]),
            "ttm_plan_create": (_i, [_vp, _vp, _i, _i, _i, C.POINTER(ttm_field_params), _i, _i, _i, _i,
                                     C.POINTER(_vp)]),
            "ttm_plan_destroy": (None, [_vp]),
            "ttm_plan_components": (_i, [_vp]),
            "ttm_plan_valid_box": (None, [_vp, C.POINTER(_i)]),
            "ttm_correlate": (_i, [_vp, _vp, _vp, _vp]),
            "ttm_plan_copy_w": (_i, [_vp, _vp, _vp]),
            "ttm_peak_map": (_i, [_vp, _vp, _i, _vp, _vp, _vp, _vp, _vp]),
            "ttm_find_peaks": (_i, [_vp, _vp, _i, _d, _vp, _vp, C.POINTER(_i), _vp]),
            "tm_correlate": (_i, [_vp, _vp, _i, _i, _i, _vp, _i, _i, _i, C.POINTER(ttm_field_params), _vp, _i64,
                                  _vp, _vp, _vp]),
            "ttm_plan_enable_timing": (_i, [_vp, _i]),
            "ttm_plan_stage_times": (_i, [_vp, _vp, _i]),
            "ttm_num_stages": (_i, []),
            "ttm_stage_name": (C.c_char_p, [_i]),
            "ttm_kernel_launches": (C.c_uint64, []),
            "ttm_plan_set_localsum": (_i, [_vp, _i]),
            "ttm_find_peaks_noalloc": (_i, [_vp, _vp, _i, _i, _i, _vp, _i, _d, _vp, _vp, C.POINTER(_i), _vp]),
            "ttm_plan_fallback_count": (_i, [_vp, C.POINTER(_i64), _vp]),
            "ttm_refine_peaks": (_i, [_vp, _vp, _vp, _vp, _i, _d, _vp, _vp, _vp, _vp]),
            "ttm_slab_ranges": (_i, [_i, _i, _i, _vp, _i]),
            "ttm_merge_peaks": (_i, [_i64, _vp, _vp, _i, _i, _i, _i, _d, _vp, _vp]),
            "ttm_blocked_create": (_i, [_vp, _vp, _i, _i, _i, _vp, _i, _i, _i, _i, C.POINTER(_vp)]),
            "ttm_blocked_run": (_i, [_vp, _vp, _i, _i, _d, _vp, _vp, _vp, _vp]),
            "ttm_blocked_destroy": (None, [_vp]),
            "ttm_blocked_peaks": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp, _i, _i, _i, _i, _i, _i, _d, _vp, _vp,
                                       C.POINTER(_i), _vp]),
            "ttm_mlp_num_params": (_i64, [_i]),
            "ttm_mlp_create": (_i, [_vp, _i, C.c_uint64, C.POINTER(_vp)]),
            "ttm_mlp_destroy": (None, [_vp]),
            "ttm_mlp_inputs": (_i, [_vp]),
            "ttm_mlp_get_params": (_i, [_vp, _vp]),
            "ttm_mlp_set_params": (_i, [_vp, _vp]),
            "ttm_mlp_forward": (_i, [_vp, _vp, _i64, _vp, _vp]),
            "ttm_mlp_loss_grad": (_i, [_vp, _vp, _vp, _i64, _vp, C.POINTER(_d), _vp]),
            "ttm_mlp_train": (_i, [_vp, _vp, _vp, _i64, _i, _i, C.c_float, C.c_uint64, C.POINTER(_d), _vp]),
            "ttm_mlp_infer": (_i, [_vp, _vp, _i64, _vp, _vp]),
            "ttm_mlp_set_precision": (_i, [_vp, _i]),
            "ttm_mlp_make_pairs": (_i, [_vp, _vp, _i, _i64, _vp, _vp, _i64, _vp, _vp, _vp]),
            "ttm_mlp_save": (_i, [_vp, C.c_char_p]),
            "ttm_mlp_load": (_i, [_vp, C.c_char_p, C.POINTER(_vp)]),
            "ttm_plan_create_padded": (_i, [_vp, _vp, _i, _i, _i, C.POINTER(ttm_field_params), _i, _i, _i, _i, _i,
                                            _i, _i, C.POINTER(_vp)]),
            "ttm_autotune_shape": (_i, [_vp, _i, _i, _i, _vp]),
            "ttm_autotune_entries": (_i, [_vp]),
            "ttm_autotune_save": (_i, [_vp, C.c_char_p]),
            "ttm_autotune_load": (_i, [_vp, C.c_char_p]),
            "ttm_batch_create": (_i, [_vp, C.POINTER(ttm_field_params), _i, _i, _i, _i, _vp, _i, _vp, _i, _vp, _i,
                                      _i, C.POINTER(_vp)]),
            "ttm_batch_run": (_i, [_vp, _vp]),
            "ttm_batch_work_shape": (_i, [_vp, _i, _vp]),
            "ttm_batch_destroy": (None, [_vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# ------------------------------------------------------------ marshalling --

def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _dev(t, dtype, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError("%s must be a contiguous CUDA %s tensor" % (name, dtype))
    return t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _check(code, ctx=None):
    if code != TTM_OK:
        msg = lib().ttm_last_error(ctx).decode() if ctx else ""
        raise TTMError(code, msg)


def params(order_n=4, mask_radius=16.0, dprime=3, mask_soft_width=0.0, filter_a=0.2, n_rot_base=2048,
           cube_symmetrize=True) -> ttm_field_params:
    p = ttm_field_params()
    lib().ttm_default_params(C.byref(p))
    p.order_n, p.dprime, p.mask_radius = order_n, dprime, float(mask_radius)
    p.mask_soft_width, p.filter_a = float(mask_soft_width), float(filter_a)
    p.n_rot_base, p.cube_symmetrize = int(n_rot_base), int(bool(cube_symmetrize))
    return p


# -------------------------------------------------------- entry points --

def ttm_num_components(order_n: int, dprime: int = 3) -> int:
    return lib().ttm_num_components(order_n, dprime)


def ttm_version() -> str:
    return lib().ttm_version().decode()


def ttm_rotation_set(n_base: int, cube: bool = True) -> np.ndarray:
    q = np.zeros((n_base * (24 if cube else 1), 4))
    _check(lib().ttm_rotation_set(n_base, int(cube), q.ctypes.data))
    return q


class Context:
    """ttm_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        h = _vp()
        code = lib().ttm_ctx_create(device, C.byref(h))
        if code != TTM_OK:
            raise TTMError(code, "ttm_ctx_create(%d)" % device)
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            lib().ttm_ctx_destroy(self.h)
            self.h = None

    __del__ = close

    def check(self, code):
        _check(code, self.h)


def ttm_ctx_create(device: int = 0) -> Context:
    return Context(device)


def ttm_ctx_set_wait_limit(ctx: Context, polls: int):
    ctx.check(lib().ttm_ctx_set_wait_limit(ctx.h, int(polls)))


def ttm_ctx_device_status(ctx: Context, stream=None):
    """Raises TTMError (code TTM_E_TIMEOUT) if a bounded device wait of the
    context expired since the last check; synchronises the stream."""
    ctx.check(lib().ttm_ctx_device_status(ctx.h, _stream(stream)))


def ttm_build_tensor_field(ctx: Context, d_tmpl, p: ttm_field_params, d_field, stream=None):
    import torch
    tz, ty, tx = d_tmpl.shape
    ctx.check(lib().ttm_build_tensor_field(ctx.h, _dev(d_tmpl, torch.float32, "d_tmpl"), tz, ty, tx, C.byref(p),
                                           _dev(d_field, torch.float64, "d_field"), _stream(stream)))


class Plan:
    """ttm_plan: a tensor field bound to one tomogram shape."""

    def __init__(self, ctx: Context, d_field, p: ttm_field_params, shape, precision=TTM_PREC_FP32,
                 work_shape=None):
        import torch
        K, tz, ty, tx = d_field.shape
        if K != ttm_num_components(p.order_n, p.dprime):
            raise ValueError("the field has %d components; order %d, d' = %d needs %d"
                             % (K, p.order_n, p.dprime, ttm_num_components(p.order_n, p.dprime)))
        Z, Y, X = shape
        Zw, Yw, Xw = shape if work_shape is None else work_shape
        h = _vp()
        ctx.check(lib().ttm_plan_create_padded(ctx.h, _dev(d_field, torch.float64, "d_field"), tz, ty, tx,
                                               C.byref(p), Z, Y, X, Zw, Yw, Xw, precision, C.byref(h)))
        self.h, self.ctx, self.K = h, ctx, lib().ttm_plan_components(h)
        self.tomo_shape = (Z, Y, X)
        self.shape = (Zw, Yw, Xw)   # working grid: the layout of every map
        self.tshape = (tz, ty, tx)
        self.params = p

    def close(self):
        if getattr(self, "h", None):
            lib().ttm_plan_destroy(self.h)
            self.h = None

    __del__ = close

    def valid_box(self):
        b = (C.c_int * 6)()
        lib().ttm_plan_valid_box(self.h, b)
        return tuple(b)


def ttm_plan_create(ctx, d_field, p, shape, precision=TTM_PREC_FP32) -> Plan:
    return Plan(ctx, d_field, p, shape, precision)


def ttm_correlate(plan: Plan, d_tomo, d_C, stream=None):
    import torch
    plan.ctx.check(lib().ttm_correlate(plan.h, _dev(d_tomo, torch.float32, "d_tomo"),
                                       _dev(d_C, torch.float32, "d_C"), _stream(stream)))


def ttm_plan_set_localsum(plan: Plan, mode: int):
    plan.ctx.check(lib().ttm_plan_set_localsum(plan.h, int(mode)))


def ttm_plan_copy_w(plan: Plan, d_w, stream=None):
    import torch
    plan.ctx.check(lib().ttm_plan_copy_w(plan.h, _dev(d_w, torch.float32, "d_w"), _stream(stream)))


def ttm_peak_map(plan: Plan, d_C, d_score, d_orient, d_frob=None, mode=TTM_MAX_PLAIN, mlp=None, stream=None):
    """Score, orientation and Frobenius maps on the plan's working grid;
    d_orient holds d' components per voxel: (u_x, u_y, u_z) for d' = 3, the
    unit quaternion (w, x, y, z) for d' = 4."""
    import torch
    if mlp is not None and mode == TTM_MAX_PLAIN:
        mode = TTM_MAX_MLP_WARM
    V = int(np.prod(plan.shape))
    if d_C.numel() < plan.K * V or d_score.numel() < V or d_orient.numel() < plan.params.dprime * V or \
            (d_frob is not None and d_frob.numel() < V):
        raise ValueError("map buffers are smaller than the plan's working grid needs")
    plan.ctx.check(lib().ttm_peak_map(plan.h, _dev(d_C, torch.float32, "d_C"), mode,
                                      None if mlp is None else mlp.h,
                                      _dev(d_score, torch.float32, "d_score"),
                                      _dev(d_orient, torch.float32, "d_orient"),
                                      None if d_frob is None else _dev(d_frob, torch.float32, "d_frob"),
                                      _stream(stream)))


def ttm_plan_fallback_count(plan: Plan, stream=None) -> int:
    n = C.c_int64(0)
    plan.ctx.check(lib().ttm_plan_fallback_count(plan.h, C.byref(n), _stream(stream)))
    return n.value


# ------------------------------------------------------ learned warm start --

def ttm_mlp_num_params(n_inputs: int) -> int:
    return lib().ttm_mlp_num_params(n_inputs)


class Mlp:
    """ttm_mlp: the warm-start network K -> 128 -> 128 -> 3 on one device."""

    def __init__(self, ctx: Context, n_inputs: int = 0, seed: int = 0, handle=None):
        self.ctx = ctx
        if handle is None:
            h = _vp()
            ctx.check(lib().ttm_mlp_create(ctx.h, n_inputs, seed, C.byref(h)))
            handle = h
        self.h = handle
        self.K = lib().ttm_mlp_inputs(self.h)
        self.num_params = lib().ttm_mlp_num_params(self.K)

    def close(self):
        if getattr(self, "h", None):
            lib().ttm_mlp_destroy(self.h)
            self.h = None

    __del__ = close

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.num_params, dtype=np.float32)
        self.ctx.check(lib().ttm_mlp_get_params(self.h, p.ctypes.data))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.num_params
        self.ctx.check(lib().ttm_mlp_set_params(self.h, p.ctypes.data))

    def forward(self, d_X, d_U, stream=None):
        import torch
        self.ctx.check(lib().ttm_mlp_forward(self.h, _dev(d_X, torch.float32, "d_X"), d_X.shape[0],
                                             _dev(d_U, torch.float32, "d_U"), _stream(stream)))

    def set_precision(self, mode: int):
        """TTM_MLP_FP32 (default) or TTM_MLP_BF16 products in forward, loss_grad and train."""
        self.ctx.check(lib().ttm_mlp_set_precision(self.h, int(mode)))

    def infer(self, d_X, d_U, stream=None):
        import torch
        self.ctx.check(lib().ttm_mlp_infer(self.h, _dev(d_X, torch.float32, "d_X"), d_X.shape[0],
                                           _dev(d_U, torch.float32, "d_U"), _stream(stream)))

    def loss_grad(self, d_X, d_U, d_grad, stream=None) -> float:
        import torch
        L = C.c_double(0)
        self.ctx.check(lib().ttm_mlp_loss_grad(self.h, _dev(d_X, torch.float32, "d_X"),
                                               _dev(d_U, torch.float32, "d_U"), d_X.shape[0],
                                               _dev(d_grad, torch.float32, "d_grad"), C.byref(L), _stream(stream)))
        return L.value

    def train(self, d_X, d_U, epochs=20, batch=4096, lr=1e-3, seed=0, stream=None) -> float:
        import torch
        L = C.c_double(0)
        self.ctx.check(lib().ttm_mlp_train(self.h, _dev(d_X, torch.float32, "d_X"),
                                           _dev(d_U, torch.float32, "d_U"), d_X.shape[0], epochs, batch,
                                           float(lr), seed, C.byref(L), _stream(stream)))
        return L.value

    def save(self, path: str):
        self.ctx.check(lib().ttm_mlp_save(self.h, path.encode()))

    @classmethod
    def load(cls, ctx: Context, path: str) -> "Mlp":
        h = _vp()
        ctx.check(lib().ttm_mlp_load(ctx.h, path.encode(), C.byref(h)))
        return cls(ctx, handle=h)


def ttm_mlp_make_pairs(ctx: Context, d_C, order_n: int, d_orient, d_idx, d_X, d_U, stream=None):
    import torch
    V = d_C[0].numel()
    ctx.check(lib().ttm_mlp_make_pairs(ctx.h, _dev(d_C, torch.float32, "d_C"), order_n, V,
                                       _dev(d_orient, torch.float32, "d_orient"), _dev(d_idx, torch.int64, "d_idx"),
                                       d_idx.shape[0], _dev(d_X, torch.float32, "d_X"),
                                       _dev(d_U, torch.float32, "d_U"), _stream(stream)))


# -------------------------------------------------- autotuner and batches --

def ttm_autotune_shape(ctx: Context, shape) -> tuple:
    out = (C.c_int * 3)()
    ctx.check(lib().ttm_autotune_shape(ctx.h, int(shape[0]), int(shape[1]), int(shape[2]), out))
    return tuple(out)


def ttm_autotune_entries(ctx: Context) -> int:
    return lib().ttm_autotune_entries(ctx.h)


def ttm_autotune_save(ctx: Context, path: str):
    ctx.check(lib().ttm_autotune_save(ctx.h, path.encode()))


def ttm_autotune_load(ctx: Context, path: str):
    ctx.check(lib().ttm_autotune_load(ctx.h, path.encode()))


class ttm_batch_tomo(C.Structure):
    _fields_ = [("d_tomo", _vp), ("Z", _i), ("Y", _i), ("X", _i)]


class ttm_batch_item(C.Structure):
    _fields_ = [("tomo", _i), ("tmpl", _i), ("d_score", _vp), ("d_orient", _vp), ("d_frob", _vp)]


class Batch:
    """ttm_batch: (tomogram, template) pairs in one captured CUDA graph.
    tomos: CUDA float32 [Z][Y][X] tensors; fields: CUDA float64 [K][t][t][t]
    tensors; items: (tomo, tmpl, d_score, d_orient, d_frob or None) with
    maps on the tomogram grid (only the valid box is written)."""

    def __init__(self, ctx: Context, p: ttm_field_params, fields, tomos, items, n_branches=4,
                 flags=TTM_BATCH_AUTOTUNE):
        import torch
        self.ctx = ctx
        self._keep = (list(fields), list(tomos), list(items))
        tz, ty, tx = fields[0].shape[1:]
        fptr = (C.c_void_p * len(fields))(*[_dev(f, torch.float64, "field") for f in fields])
        tarr = (ttm_batch_tomo * len(tomos))(*[ttm_batch_tomo(_dev(t, torch.float32, "tomo"), *t.shape)
                                              for t in tomos])
        iarr = (ttm_batch_item * len(items))(*[
            ttm_batch_item(a, b, _dev(s, torch.float32, "d_score"), _dev(o, torch.float32, "d_orient"),
                           None if f is None else _dev(f, torch.float32, "d_frob")) for a, b, s, o, f in items])
        h = _vp()
        ctx.check(lib().ttm_batch_create(ctx.h, C.byref(p), tz, ty, tx, len(fields), fptr, len(tomos), tarr,
                                         len(items), iarr, n_branches, flags, C.byref(h)))
        self.h = h

    def run(self, stream=None):
        self.ctx.check(lib().ttm_batch_run(self.h, _stream(stream)))

    def work_shape(self, i: int) -> tuple:
        out = (C.c_int * 3)()
        self.ctx.check(lib().ttm_batch_work_shape(self.h, i, out))
        return tuple(out)

    def close(self):
        if getattr(self, "h", None):
            lib().ttm_batch_destroy(self.h)
            self.h = None

    __del__ = close


def ttm_find_peaks(plan: Plan, d_map, P: int, min_dist: float, stream=None):
    import torch
    idx = np.zeros(max(P, 1), dtype=np.int64)
    val = np.zeros(max(P, 1), dtype=np.float32)
    n = C.c_int(0)
    plan.ctx.check(lib().ttm_find_peaks(plan.h, _dev(d_map, torch.float32, "d_map"), P, float(min_dist),
                                        idx.ctypes.data, val.ctypes.data, C.byref(n), _stream(stream)))
    return idx[:n.value], val[:n.value]


def ttm_refine_peaks(plan: Plan, d_tmpl, d_orient, peaks, r_s: float = 3.0, stream=None):
    """TTM-ref (Alg. 3): refined linear indices, rotations (w, x, y, z) and
    LNCC values of the peaks (linear indices on the plan's working grid)."""
    import torch
    pk = np.ascontiguousarray(peaks, dtype=np.int64)
    P = int(pk.size)
    if d_orient.numel() < 4 * int(np.prod(plan.shape)):
        raise ValueError("d_orient must hold the [4][Z][Y][X] quaternion map")
    idx = np.zeros(max(P, 1), dtype=np.int64)
    quat = np.zeros((max(P, 1), 4), dtype=np.float32)
    lncc = np.zeros(max(P, 1), dtype=np.float32)
    plan.ctx.check(lib().ttm_refine_peaks(plan.h, _dev(d_tmpl, torch.float32, "d_tmpl"),
                                          _dev(d_orient, torch.float32, "d_orient"), pk.ctypes.data, P,
                                          float(r_s), idx.ctypes.data, quat.ctypes.data, lncc.ctypes.data,
                                          _stream(stream)))
    return idx[:P], quat[:P], lncc[:P]


def ttm_slab_ranges(Z: int, tz: int, slab_z: int) -> np.ndarray:
    """Block processing's z-slab table: rows (o0, o1, m0, m1, i0, i1)."""
    n = lib().ttm_slab_ranges(int(Z), int(tz), int(slab_z), None, 0)
    if n < 0:
        raise ValueError("bad slab arguments")
    out = np.zeros((max(n, 1), 6), dtype=np.int32)
    lib().ttm_slab_ranges(int(Z), int(tz), int(slab_z), out.ctypes.data, n)
    return out[:n]


def ttm_merge_peaks(idx, val, shape, P: int, min_dist: float):
    """Merge Peaks: (value desc, index asc) order, greedy exclusion at min_dist."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    val = np.ascontiguousarray(val, dtype=np.float32)
    Z, Y, X = shape
    oi = np.zeros(max(P, 1), dtype=np.int64)
    ov = np.zeros(max(P, 1), dtype=np.float32)
    n = lib().ttm_merge_peaks(idx.size, idx.ctypes.data, val.ctypes.data, Z, Y, X, int(P), float(min_dist),
                              oi.ctypes.data, ov.ctypes.data)
    if n < 0:
        raise ValueError("bad merge arguments")
    return oi[:n], ov[:n]


def ttm_blocked_peaks(ctx: Context, d_field, p: ttm_field_params, tomo, slab_z: int, P: int, min_dist: float,
                      map_kind: int = 0, stream=None):
    """Block processing (Sec. 3.4) of a host tomogram (float32 numpy array)."""
    import torch
    tomo = np.ascontiguousarray(tomo, dtype=np.float32)
    Z, Y, X = tomo.shape
    K, tz, ty, tx = d_field.shape
    idx = np.zeros(max(P, 1), dtype=np.int64)
    val = np.zeros(max(P, 1), dtype=np.float32)
    n = C.c_int(0)
    ctx.check(lib().ttm_blocked_peaks(ctx.h, _dev(d_field, torch.float64, "d_field"), tz, ty, tx, C.byref(p),
                                      tomo.ctypes.data, Z, Y, X, int(slab_z), int(map_kind), int(P),
                                      float(min_dist), idx.ctypes.data, val.ctypes.data, C.byref(n),
                                      _stream(stream)))
    return idx[:n.value], val[:n.value]


class Blocked:
    """ttm_blocked: block processing (Sec. 3.4) kept across tomograms of one shape."""

    def __init__(self, ctx: Context, d_field, p: ttm_field_params, shape, slab_z: int):
        import torch
        K, tz, ty, tx = d_field.shape
        Z, Y, X = shape
        h = _vp()
        ctx.check(lib().ttm_blocked_create(ctx.h, _dev(d_field, torch.float64, "d_field"), tz, ty, tx, C.byref(p),
                                           Z, Y, X, int(slab_z), C.byref(h)))
        self.h, self.ctx, self.shape = h, ctx, (Z, Y, X)

    def run(self, tomo, P: int, min_dist: float, map_kind: int = 0, stream=None):
        """tomo: float32 host array (numpy, or a pinned CPU tensor for
        copies that overlap the kernels)."""
        if hasattr(tomo, "data_ptr"):
            if tuple(tomo.shape) != self.shape or not tomo.is_contiguous():
                raise ValueError("tomogram shape or layout differs from the session's")
            ptr = tomo.data_ptr()
        else:
            tomo = np.ascontiguousarray(tomo, dtype=np.float32)
            if tomo.shape != self.shape:
                raise ValueError("tomogram shape differs from the session's")
            ptr = tomo.ctypes.data
        idx = np.zeros(max(P, 1), dtype=np.int64)
        val = np.zeros(max(P, 1), dtype=np.float32)
        n = C.c_int(0)
        self.ctx.check(lib().ttm_blocked_run(self.h, ptr, int(map_kind), int(P), float(min_dist), idx.ctypes.data,
                                             val.ctypes.data, C.byref(n), _stream(stream)))
        return idx[:n.value], val[:n.value]

    def close(self):
        if getattr(self, "h", None):
            lib().ttm_blocked_destroy(self.h)
            self.h = None

    __del__ = close


def ttm_find_peaks_noalloc(ctx: Context, d_map, box, P: int, min_dist: float, stream=None):
    """Allocation-free Find Peaks over box (z0, z1, y0, y1, x0, x1) of d_map."""
    import torch
    Z, Y, X = d_map.shape
    b = (C.c_int * 6)(*[int(v) for v in box])
    idx = np.zeros(max(P, 1), dtype=np.int64)
    val = np.zeros(max(P, 1), dtype=np.float32)
    n = C.c_int(0)
    ctx.check(lib().ttm_find_peaks_noalloc(ctx.h, _dev(d_map, torch.float32, "d_map"), Z, Y, X, b, P,
                                           float(min_dist), idx.ctypes.data, val.ctypes.data, C.byref(n),
                                           _stream(stream)))
    return idx[:n.value], val[:n.value]


def tm_correlate(ctx: Context, d_tomo, d_tmpl, p: ttm_field_params, quats: np.ndarray, d_best, d_best_idx,
                 stream=None):
    import torch
    Z, Y, X = d_tomo.shape
    tz, ty, tx = d_tmpl.shape
    q = np.ascontiguousarray(quats, dtype=np.float64).reshape(-1, 4)
    ctx.check(lib().tm_correlate(ctx.h, _dev(d_tomo, torch.float32, "d_tomo"), Z, Y, X,
                                 _dev(d_tmpl, torch.float32, "d_tmpl"), tz, ty, tx, C.byref(p), q.ctypes.data,
                                 q.shape[0], _dev(d_best, torch.float32, "d_best"),
                                 _dev(d_best_idx, torch.int32, "d_best_idx"), _stream(stream)))


def ttm_plan_enable_timing(plan: Plan, on: bool = True):
    plan.ctx.check(lib().ttm_plan_enable_timing(plan.h, int(on)))


def ttm_plan_stage_times(plan: Plan) -> dict:
    n = lib().ttm_num_stages()
    ms = np.zeros(n)
    plan.ctx.check(lib().ttm_plan_stage_times(plan.h, ms.ctypes.data, n))
    return {lib().ttm_stage_name(i).decode(): float(ms[i]) for i in range(n)}


def ttm_kernel_launches() -> int:
    return int(lib().ttm_kernel_launches())


# ------------------------------------------------------------ pipeline --

class Matcher:
    """Convenience: one template, one tomogram shape, device buffers for the
    whole hot path (C, score, orientation, Frobenius)."""

    def __init__(self, ctx: Context, template, p: ttm_field_params, shape, device="cuda"):
        import torch
        self.ctx, self.p = ctx, p
        t = torch.as_tensor(np.ascontiguousarray(template, dtype=np.float32), device=device)
        K = ttm_num_components(p.order_n, p.dprime)
        self.field = torch.empty((K,) + tuple(t.shape), dtype=torch.float64, device=device)
        ttm_build_tensor_field(ctx, t, p, self.field)
        torch.cuda.synchronize()
        self.plan = Plan(ctx, self.field, p, shape)
        Z, Y, X = shape
        self.C = torch.empty((K, Z, Y, X), dtype=torch.float32, device=device)
        self.score = torch.empty((Z, Y, X), dtype=torch.float32, device=device)
        self.orient = torch.empty((p.dprime, Z, Y, X), dtype=torch.float32, device=device)
        self.frob = torch.empty((Z, Y, X), dtype=torch.float32, device=device)

    def run(self, d_tomo, stream=None, mlp=None):
        ttm_correlate(self.plan, d_tomo, self.C, stream)
        ttm_peak_map(self.plan, self.C, self.score, self.orient, self.frob, mlp=mlp, stream=stream)
        return self.score, self.orient, self.frob
