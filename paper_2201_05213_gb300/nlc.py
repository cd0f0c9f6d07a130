"""Python binding of the nlc C ABI (include/nlc.h): argument marshalling only.

Each ``nlc_*`` function here calls the C function of the same name in
libnlc.so, passing raw device pointers of torch CUDA tensors (PyTorch only
provides device memory and streams).  Every step of compression,
decompression and training runs in the library's CUDA kernels; there is no
CPU fallback: if the library or a GPU is missing, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libnlc.so")
_lib = None
_lock = threading.Lock()

NLC_OK = 0
NLC_ERR_ARG = 1
NLC_ERR_CAPACITY = 2
NLC_ERR_CORRUPT = 3
NLC_ERR_WEIGHTS = 4
NLC_ERR_CUDA = 5
NLC_ERR_TIMEOUT = 6
NLC_ERR_UNSUPPORTED = 7

NLC_FP32, NLC_BF16, NLC_BF16_SHEARED = 0, 1, 2
NLC_SCHED_RASTER, NLC_SCHED_WAVEFRONT, NLC_SCHED_SEQUENTIAL = 0, 1, 2
NLC_LAYOUT_UNIT, NLC_LAYOUT_ROW = 0, 1

EXPORTS = [
    "nlc_last_error", "nlc_abi_version", "nlc_num_weights", "nlc_create", "nlc_destroy",
    "nlc_get_weights", "nlc_set_weights", "nlc_weight_hash", "nlc_sync_status", "nlc_set_tuning",
    "nlc_compress_bound", "nlc_compress", "nlc_decompress", "nlc_forward", "nlc_tables",
    "nlc_rans_encode", "nlc_rans_decode", "nlc_train_step", "nlc_loss_grad",
    "nlc_compress_noalloc", "nlc_decode_profile",
    "nlc_plan_decode", "nlc_plan_run", "nlc_plan_tune", "nlc_plan_destroy",
    "nlc_decode_step_times", "nlc_measure_mufu", "nlc_backward", "nlc_load_weights",
    "nlc_sample", "nlc_set_wait_limits",
]


class NLCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nlc error {code}: {msg}")
        self.code = code


class nlc_model_cfg(C.Structure):
    _fields_ = [("h", C.c_int32), ("C", C.c_int32), ("n_res", C.c_int32), ("K", C.c_int32),
                ("precision", C.c_int32)]


class nlc_image(C.Structure):
    _fields_ = [("data", C.c_void_p), ("H", C.c_int32), ("W", C.c_int32)]


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Loads libnlc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise NLCError(NLC_ERR_CUDA, f"{_LIB_PATH} is missing: run build() first")
            L = C.CDLL(_LIB_PATH)
            p, i, i32, i64, sz, f = C.c_void_p, C.c_int, C.c_int32, C.c_int64, C.c_size_t, C.c_float
            L.nlc_last_error.restype = C.c_char_p
            L.nlc_abi_version.restype = i
            L.nlc_num_weights.restype = sz
            L.nlc_num_weights.argtypes = [p]
            L.nlc_create.argtypes = [p, p, sz, p]
            L.nlc_destroy.argtypes = [p]
            L.nlc_get_weights.argtypes = [p, p, sz]
            L.nlc_set_weights.argtypes = [p, p, sz]
            L.nlc_weight_hash.argtypes = [p, p]
            L.nlc_sync_status.argtypes = [p, p]
            L.nlc_set_tuning.argtypes = [p, i, i]
            L.nlc_compress_bound.argtypes = [p, p, i, i, i, p]
            L.nlc_compress.argtypes = [p, p, i, i, i, p, sz, p, p]
            L.nlc_decompress.argtypes = [p, p, p, p, i, i, i, i, p]
            L.nlc_forward.argtypes = [p, p, i, i, p, p, p]
            L.nlc_tables.argtypes = [p, p, p, i64, p, p]
            L.nlc_rans_encode.argtypes = [p, p, p, i, p, i64, p, p]
            L.nlc_rans_decode.argtypes = [p, p, i64, p, p, p, i, p, p]
            L.nlc_train_step.argtypes = [p, p, i, i, i, f, p, p]
            L.nlc_loss_grad.argtypes = [p, p, i, i, i, p, p, p]
            L.nlc_compress_noalloc.argtypes = [p, p, i, i, i, p, sz, p, p]
            L.nlc_decode_profile.argtypes = [p, i, p]
            L.nlc_plan_decode.argtypes = [p, p, i, i, i, i, p]
            L.nlc_plan_run.argtypes = [p, p, p, p]
            L.nlc_plan_tune.argtypes = [p, p, p, i, p, p, p]
            L.nlc_plan_destroy.argtypes = [p]
            L.nlc_decode_step_times.argtypes = [p, p, i64]
            L.nlc_measure_mufu.argtypes = [i, p, p, p]
            L.nlc_backward.argtypes = [p, p, i, i, i, p, p, p]
            L.nlc_load_weights.argtypes = [p, p, sz, p]
            L.nlc_sample.argtypes = [p, p, i, i, C.c_uint64, i, p]
            L.nlc_set_wait_limits.argtypes = [p, C.c_uint32, C.c_uint32]
            for name in EXPORTS:
                getattr(L, name).restype = getattr(L, name).restype or i
            L.nlc_last_error.restype = C.c_char_p
            L.nlc_num_weights.restype = sz
            _lib = L
    return _lib


def _check(rc):
    if rc != NLC_OK:
        raise NLCError(rc, load().nlc_last_error().decode())
    return rc


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        return None
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _images(imgs):
    arr = (nlc_image * max(len(imgs), 1))()
    for k, t in enumerate(imgs):
        H, W = int(t.shape[0]), int(t.shape[1])
        arr[k] = nlc_image(t.data_ptr() if H * W > 0 else None, H, W)
    return arr


def _cfg(h, C_, n_res, K, precision):
    return nlc_model_cfg(h, C_, n_res, K, precision)


# ---------------------------------------------------------------- same names

def nlc_abi_version():
    return load().nlc_abi_version()


def nlc_num_weights(h, C_, n_res, K, precision=NLC_FP32):
    cfg = _cfg(h, C_, n_res, K, precision)
    return int(load().nlc_num_weights(C.byref(cfg)))


def nlc_create(h, C_, n_res, K, precision, weights):
    cfg = _cfg(h, C_, n_res, K, precision)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    ctx = C.c_void_p()
    _check(load().nlc_create(C.byref(cfg), _ptr(w), w.size, C.byref(ctx)))
    return ctx


def nlc_destroy(ctx):
    return _check(load().nlc_destroy(ctx))


def nlc_get_weights(ctx, n):
    w = np.zeros(n, dtype=np.float32)
    _check(load().nlc_get_weights(ctx, _ptr(w), n))
    return w


def nlc_set_weights(ctx, weights):
    w = np.ascontiguousarray(weights, dtype=np.float32)
    return _check(load().nlc_set_weights(ctx, _ptr(w), w.size))


def nlc_weight_hash(ctx):
    h = C.c_uint64(0)
    _check(load().nlc_weight_hash(ctx, C.byref(h)))
    return h.value


def nlc_sync_status(ctx, stream=None):
    """Returns the device status code (0 = OK) and clears it; does not raise."""
    return load().nlc_sync_status(ctx, _stream(stream))


def nlc_decode_profile(ctx, enable, read=True):
    """Enables/disables decoder phase profiling; returns the 16 counters (or None)."""
    out = np.zeros(16, dtype=np.uint64) if read else None
    _check(load().nlc_decode_profile(ctx, int(enable), _ptr(out) if read else None))
    return out


def nlc_decode_step_times(ctx, times):
    """times: int64 CUDA tensor receiving the decoder's step end times (ns), or None."""
    if times is None:
        return _check(load().nlc_decode_step_times(ctx, None, 0))
    return _check(load().nlc_decode_step_times(ctx, _ptr(times), int(times.numel())))


def nlc_set_tuning(ctx, px_per_cta, max_ctas=0):
    return _check(load().nlc_set_tuning(ctx, int(px_per_cta), int(max_ctas)))


def nlc_compress_bound(sizes, patch, layout):
    n = len(sizes)
    H = np.array([s[0] for s in sizes] or [0], dtype=np.int32)
    W = np.array([s[1] for s in sizes] or [0], dtype=np.int32)
    out = C.c_size_t(0)
    _check(load().nlc_compress_bound(_ptr(H), _ptr(W), n, patch, layout, C.byref(out)))
    return out.value


def nlc_compress(ctx, imgs, patch, layout, out, offsets, stream=None):
    """imgs: list of (H, W, 3) uint8 CUDA tensors; out: uint8 CUDA buffer;
    offsets: (n+1,) int64 CUDA tensor written with the container offsets."""
    arr = _images(imgs)
    return _check(load().nlc_compress(ctx, arr, len(imgs), patch, layout, _ptr(out),
                                      out.numel(), _ptr(offsets), _stream(stream)))


def nlc_compress_noalloc(ctx, imgs, patch, layout, out, offsets, stream=None):
    """nlc_compress with the library's fixed device scratch instead of its
    workspace: the call itself allocates no device memory."""
    arr = _images(imgs)
    return _check(load().nlc_compress_noalloc(ctx, arr, len(imgs), patch, layout, _ptr(out),
                                              out.numel(), _ptr(offsets), _stream(stream)))


NLC_NOALLOC_SCRATCH_BYTES = 32 << 20


def nlc_decompress(ctx, data, offsets, outs, patch, layout, schedule, stream=None):
    arr = _images(outs)
    return _check(load().nlc_decompress(ctx, _ptr(data), _ptr(offsets), arr, len(outs), patch,
                                        layout, schedule, _stream(stream)))


def nlc_plan_decode(ctx, outs, patch, layout, schedule):
    """Plan for decoding into the (H, W, 3) uint8 CUDA tensors outs (kept by
    the caller for the plan's lifetime)."""
    arr = _images(outs)
    plan = C.c_void_p()
    _check(load().nlc_plan_decode(ctx, arr, len(outs), patch, layout, schedule, C.byref(plan)))
    return plan


def nlc_plan_run(plan, data, offsets, stream=None):
    return _check(load().nlc_plan_run(plan, _ptr(data), _ptr(offsets), _stream(stream)))


def nlc_plan_tune(plan, data, offsets, reps=2, stream=None):
    """Returns (px_per_cta, ms per decode) of the fastest setting."""
    ppc, ms = C.c_int(0), C.c_float(0)
    _check(load().nlc_plan_tune(plan, _ptr(data), _ptr(offsets), int(reps), _stream(stream),
                                C.byref(ppc), C.byref(ms)))
    return ppc.value, ms.value


def nlc_plan_destroy(plan):
    return _check(load().nlc_plan_destroy(plan))


def nlc_forward(ctx, imgs, patch, params=None, bits=None, stream=None):
    arr = _images(imgs)
    return _check(load().nlc_forward(ctx, arr, len(imgs), patch, _ptr(params), _ptr(bits),
                                     _stream(stream)))


def nlc_tables(ctx, params, pixels, cum, stream=None):
    n = int(pixels.shape[0])
    return _check(load().nlc_tables(ctx, _ptr(params), _ptr(pixels), n, _ptr(cum),
                                    _stream(stream)))


def nlc_rans_encode(start, freq, sym_off, out, stride, lens, stream=None):
    return _check(load().nlc_rans_encode(_ptr(start), _ptr(freq), _ptr(sym_off),
                                         int(lens.numel()), _ptr(out), int(stride), _ptr(lens),
                                         _stream(stream)))


def nlc_rans_decode(ctx, data, stride, lens, cum, sym_off, sym, stream=None):
    return _check(load().nlc_rans_decode(ctx, _ptr(data), int(stride), _ptr(lens), _ptr(cum),
                                         _ptr(sym_off), int(lens.numel()), _ptr(sym),
                                         _stream(stream)))


def nlc_train_step(ctx, batch, lr, stream=None, want_loss=True):
    N, H, W, _ = batch.shape
    loss = C.c_float(0)
    _check(load().nlc_train_step(ctx, _ptr(batch), N, H, W, float(lr),
                                 C.byref(loss) if want_loss else None, _stream(stream)))
    return loss.value if want_loss else None


def nlc_loss_grad(ctx, batch, loss, grad, stream=None):
    N, H, W, _ = batch.shape
    return _check(load().nlc_loss_grad(ctx, _ptr(batch), N, H, W, _ptr(loss), _ptr(grad),
                                       _stream(stream)))


def nlc_measure_mufu(iters=20000, stream=None):
    """(MUFU ops/s, kernel ms) of the ex2 + rcp pair at full occupancy."""
    r, ms = C.c_double(0), C.c_double(0)
    _check(load().nlc_measure_mufu(int(iters), _stream(stream), C.byref(r), C.byref(ms)))
    return r.value, ms.value


def nlc_backward(ctx, batch, dparams, dweights, stream=None):
    """Weight gradient (dweights, device) of sum(dparams * outputs) over the
    N x H x W x 3 uint8 batch (dparams: N H W x 10K FP32, device)."""
    N_, H, W, _ = batch.shape
    _check(load().nlc_backward(ctx, _ptr(batch), N_, H, W, _ptr(dparams), _ptr(dweights),
                               _stream(stream)))


def nlc_load_weights(ctx, weights, stream=None):
    """Weights from a device FP32 tensor (asynchronous)."""
    _check(load().nlc_load_weights(ctx, _ptr(weights), int(weights.numel()), _stream(stream)))


def nlc_sample(ctx, outs, patch, seed, schedule, stream=None):
    """Draws len(outs) images from the model into the uint8 CUDA tensors outs."""
    arr, n = _images(outs), len(outs)
    _check(load().nlc_sample(ctx, arr, n, patch, int(seed) & 0xFFFFFFFFFFFFFFFF, schedule,
                             _stream(stream)))


def nlc_set_wait_limits(ctx, grid_polls=0, mma_polls=0):
    """Polls of the decoder's bounded waits before a timeout (0 = defaults)."""
    _check(load().nlc_set_wait_limits(ctx, int(grid_polls), int(mma_polls)))
