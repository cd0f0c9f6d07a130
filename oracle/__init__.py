"""CPU oracle for the parallel local-autoregressive compressor (test infrastructure).

ONLY the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  It shares no code with the CUDA
library: the arithmetic lives in ``nlc_oracle.c`` (scalar FP64 C) and in
``schedule.py`` (plain Python); this module only loads the C file with ctypes
and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nlc_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

MQ = 65280


def build(force: bool = False) -> str:
    """Compile nlc_oracle.c with gcc (no vector intrinsics, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i, l, p = C.c_double, C.c_int, C.c_long, C.c_void_p
            L.orc_num_weights.restype = l
            L.orc_num_weights.argtypes = [i, i, i, i]
            L.orc_sigmoid.restype = d
            L.orc_sigmoid.argtypes = [d]
            L.orc_log_bin_mass.restype = d
            L.orc_log_bin_mass.argtypes = [d, d, i]
            L.orc_quantise_cdf.argtypes = [p, p]
            L.orc_pixel_tables.argtypes = [i, p, i, i, p]
            L.orc_pixel_bits.restype = d
            L.orc_pixel_bits.argtypes = [i, p, i, i, i]
            L.orc_channel_prob.restype = d
            L.orc_channel_prob.argtypes = [i, p, i, i, i, i]
            L.orc_num_units.argtypes = [i, i, i]
            L.orc_forward_image.argtypes = [i, i, i, i, p, p, i, i, i, p]
            L.orc_forward_pixels.argtypes = [i, i, i, i, p, p, i, i, i, i, p, p, p]
            L.orc_image_bits.argtypes = [i, i, i, i, p, p, i, i, i, p]
            u64 = C.c_uint64
            L.orc_splitmix64.restype = u64
            L.orc_splitmix64.argtypes = [u64, u64]
            L.orc_sample_u16.restype = C.c_uint32
            L.orc_sample_u16.argtypes = [u64, i, i, i, i]
            L.orc_sample_image.argtypes = [i, i, i, i, p, i, i, i, u64, i, p]
            L.orc_rans_encode.restype = l
            L.orc_rans_encode.argtypes = [l, p, p, p, l]
            L.orc_rans_decode.argtypes = [p, l, l, p, p]
            L.orc_num_streams.argtypes = [i, i, i, i]
            L.orc_encode_image.restype = l
            L.orc_encode_image.argtypes = [i, i, i, i, p, p, i, i, i, i, p, l, p, p, p]
            L.orc_decode_image.argtypes = [i, i, i, i, p, p, p, i, i, i, i, p]
            L.orc_nll_grad.restype = d
            L.orc_nll_grad.argtypes = [i, i, i, i, p, p, i, i, i, p]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _w64(w):
    return np.ascontiguousarray(np.asarray(w, dtype=np.float64))


def num_weights(h, C_, R, K):
    return int(lib().orc_num_weights(h, C_, R, K))


def sigmoid(z):
    return float(lib().orc_sigmoid(float(z)))


def log_bin_mass(m, ls, v):
    """log P(v) of one logistic component (location m, log-scale ls)."""
    return float(lib().orc_log_bin_mass(float(m), float(ls), int(v)))


def quantise_cdf(F):
    """F: 257 CDF values (F[0]=0, F[256]=1) -> cum[257] uint32."""
    F = np.ascontiguousarray(np.asarray(F, dtype=np.float64))
    assert F.shape == (257,)
    cum = np.zeros(257, dtype=np.uint32)
    lib().orc_quantise_cdf(_ptr(F), _ptr(cum))
    return cum


def pixel_tables(K, params, r, g):
    """cum[3][257] of one pixel's R, G|r, B|r,g coding distributions."""
    p = _w64(params)
    cum = np.zeros((3, 257), dtype=np.uint32)
    lib().orc_pixel_tables(K, _ptr(p), int(r), int(g), _ptr(cum))
    return cum


def pixel_bits(K, params, r, g, b):
    p = _w64(params)
    return float(lib().orc_pixel_bits(K, _ptr(p), int(r), int(g), int(b)))


def channel_prob(K, params, ch, r, g, v):
    p = _w64(params)
    return float(lib().orc_channel_prob(K, _ptr(p), int(ch), int(r), int(g), int(v)))


def num_units(H, W, patch):
    return int(lib().orc_num_units(H, W, patch))


def num_streams(H, W, patch, layout):
    return int(lib().orc_num_streams(H, W, patch, layout))


def forward_image(cfg, w, img, patch=0):
    """Network outputs [H][W][10K] (FP64) of every pixel of img (H,W,3 uint8)."""
    h, C_, R, K = cfg
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W, _ = img.shape
    out = np.zeros((H, W, 10 * K), dtype=np.float64)
    w = _w64(w)
    lib().orc_forward_image(h, C_, R, K, _ptr(w), _ptr(img), H, W, patch, _ptr(out))
    return out


def forward_pixels(cfg, w, img, ys, xs, patch=0):
    """Network outputs [n][10K] of the pixels (ys[q], xs[q]) of img."""
    h, C_, R, K = cfg
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W, _ = img.shape
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    out = np.zeros((len(ys), 10 * K), dtype=np.float64)
    w = _w64(w)
    lib().orc_forward_pixels(h, C_, R, K, _ptr(w), _ptr(img), H, W, patch, len(ys), _ptr(ys),
                             _ptr(xs), _ptr(out))
    return out


def image_bits(cfg, w, img, patch=0):
    """Model code length -log2 p (bits) of every pixel of img, [H][W] FP64."""
    h, C_, R, K = cfg
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W, _ = img.shape
    out = np.zeros((H, W), dtype=np.float64)
    w = _w64(w)
    lib().orc_image_bits(h, C_, R, K, _ptr(w), _ptr(img), H, W, patch, _ptr(out))
    return out


def _bits_task(args):
    cfg, w, img = args
    return float(image_bits(cfg, w, img).sum())


def batch_bits_parallel(cfg, w, imgs, patch, n_proc=None, units=None):
    """Total model bits of the coding units of a batch, one spawned process per
    host core (safe beside a CUDA context).  A unit's bits equal those of its
    sub-image coded as a whole image (the context is zero outside the unit).
    units: list of (image index, y0, x0, Hu, Wu), default every unit of every
    image under the P x P partition (P = patch, 0 = whole images)."""
    import multiprocessing as mp

    if units is None:
        units = []
        for k, im in enumerate(imgs):
            H, W = im.shape[:2]
            P = patch if patch > 0 else max(H, W)
            for y in range(0, H, P):
                for x in range(0, W, P):
                    units.append((k, y, x, min(P, H - y), min(P, W - x)))
    tasks = [(cfg, _w64(w), np.ascontiguousarray(imgs[k][y:y + hu, x:x + wu]))
             for k, y, x, hu, wu in units]
    n_proc = n_proc or os.cpu_count() or 1
    build()
    with mp.get_context("spawn").Pool(min(n_proc, max(1, len(tasks)))) as pool:
        parts = pool.map(_bits_task, tasks, chunksize=1)
    return float(sum(parts)), sum(t[2].shape[0] * t[2].shape[1] for t in tasks)


def splitmix64(seed, k):
    """Output k (0, 1, ...) of SplitMix64 seeded with seed."""
    return int(lib().orc_splitmix64(int(seed) & (2 ** 64 - 1), int(k)))


def sample_u16(seed, n, y, x, c):
    """The sampler's uniform 16-bit value of channel c of pixel (y, x) of image n."""
    return int(lib().orc_sample_u16(int(seed) & (2 ** 64 - 1), n, y, x, c))


def sample_image(cfg, w, H, W, patch=0, seed=0, n=0):
    """Image n of a batch drawn from the model in raster order (H, W, 3 uint8)."""
    h, C_, R, K = cfg
    img = np.zeros((H, W, 3), dtype=np.uint8)
    w = _w64(w)
    lib().orc_sample_image(h, C_, R, K, _ptr(w), H, W, patch, int(seed) & (2 ** 64 - 1), n,
                           _ptr(img))
    return img


def rans_encode(start, freq):
    """One rANS stream (bytes, decoder order) for symbols given by (start, freq)."""
    start = np.ascontiguousarray(start, dtype=np.uint32)
    freq = np.ascontiguousarray(freq, dtype=np.uint32)
    n = len(start)
    cap = 2 * n + 4
    out = np.zeros(cap, dtype=np.uint8)
    m = lib().orc_rans_encode(n, _ptr(start), _ptr(freq), _ptr(out), cap)
    assert m >= 0
    return out[:m].copy()


def rans_decode(words, cum_tables):
    """Decode len(cum_tables) symbols; returns (symbols, ok)."""
    words = np.ascontiguousarray(words, dtype=np.uint8)
    cum = np.ascontiguousarray(cum_tables, dtype=np.uint32)
    n = cum.shape[0]
    sym = np.zeros(n, dtype=np.int32)
    rc = lib().orc_rans_decode(_ptr(words), len(words), n, _ptr(cum), _ptr(sym))
    return sym, rc == 0


def encode_image(cfg, w, img, patch=0, layout=1):
    """Raster-order encode. Returns (bytes uint8, lens int32[n_streams], bits_model, bits_quant)."""
    h, C_, R, K = cfg
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W, _ = img.shape
    ns = num_streams(H, W, patch, layout)
    cap = 6 * H * W + 4 * ns
    words = np.zeros(cap, dtype=np.uint8)
    lens = np.zeros(ns, dtype=np.int32)
    bm = C.c_double(0)
    bq = C.c_double(0)
    w = _w64(w)
    n = lib().orc_encode_image(h, C_, R, K, _ptr(w), _ptr(img), H, W, patch, layout, _ptr(words),
                               cap, _ptr(lens), C.byref(bm), C.byref(bq))
    assert n >= 0
    return words[:n].copy(), lens, bm.value, bq.value


def decode_image(cfg, w, words, lens, H, W, patch=0, layout=1):
    """Raster-order decode. Returns (img, ok)."""
    h, C_, R, K = cfg
    words = np.ascontiguousarray(words, dtype=np.uint8)
    lens = np.ascontiguousarray(lens, dtype=np.int32)
    img = np.zeros((H, W, 3), dtype=np.uint8)
    w = _w64(w)
    rc = lib().orc_decode_image(h, C_, R, K, _ptr(w), _ptr(words), _ptr(lens), H, W, patch, layout,
                                _ptr(img))
    return img, rc == 0


def nll_grad(cfg, w, imgs, grad=True):
    """Mean bits/dim of imgs (N,H,W,3) and its gradient (FP64) w.r.t. the weights."""
    h, C_, R, K = cfg
    imgs = np.ascontiguousarray(imgs, dtype=np.uint8)
    N, H, W, _ = imgs.shape
    w = _w64(w)
    g = np.zeros(len(w), dtype=np.float64) if grad else None
    v = lib().orc_nll_grad(h, C_, R, K, _ptr(w), _ptr(imgs), N, H, W,
                           _ptr(g) if grad else None)
    return (v, g) if grad else v
