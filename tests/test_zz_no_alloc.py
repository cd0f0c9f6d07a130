"""The allocation-free compression entry point (nlc_compress_noalloc).

Some callers cannot call cudaMalloc when they compress (a framework
allocator owns the device memory, or a real-time thread cannot take
cudaMalloc's synchronisation), so the library offers a compress call whose
scratch is a fixed device array instead of the context's workspace.  This
file is collected last; its test must pass alone in a fresh process and after
every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2201_05213_gb300 import nlc as N

from gpu_util import DEV, ensure_built, images, make_codec, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _compress(fn, codec, dimgs, patch, layout, cap):
    out = torch.full((cap,), 0xAB, dtype=torch.uint8, device=DEV)
    offs = torch.zeros(len(dimgs) + 1, dtype=torch.int64, device=DEV)
    torch.cuda.synchronize()
    fn(codec.ctx, dimgs, patch, layout, out, offs)
    assert N.nlc_sync_status(codec.ctx) == N.NLC_OK
    return out, offs


@pytest.mark.parametrize("prec,patch,layout", [(N.NLC_BF16, 32, N.NLC_LAYOUT_ROW),
                                               (N.NLC_FP32, 0, N.NLC_LAYOUT_UNIT)])
def test_noalloc_matches_compress_twice(prec, patch, layout):
    sizes = [(70, 90), (33, 17), (64, 64)]
    cap = N.nlc_compress_bound(sizes, patch, layout)
    batches = [[to_dev(i) for i in images(30 + call, sizes)] for call in range(2)]
    # A first call on another context loads the library's kernels and its
    # scratch array on this device, so that what follows measures the calls.
    warm, _ = make_codec((3, 32, 2, 10), prec, seed=21, scale=1.5)
    _compress(N.nlc_compress_noalloc, warm, batches[0], patch, layout, cap)
    warm.close()
    # A fresh context has an empty workspace: two calls in a row on it must
    # leave the device's free memory unchanged (no allocation anywhere).
    codec, _ = make_codec((3, 32, 2, 10), prec, seed=21, scale=1.5)
    outs = [torch.full((cap,), 0xAB, dtype=torch.uint8, device=DEV) for _ in range(2)]
    offs = [torch.zeros(len(sizes) + 1, dtype=torch.int64, device=DEV) for _ in range(2)]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for call in range(2):
        N.nlc_compress_noalloc(codec.ctx, batches[call], patch, layout, outs[call], offs[call])
        assert N.nlc_sync_status(codec.ctx) == N.NLC_OK
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory moved by {free0 - free1} bytes"
    # then the allocating entry point on the same context, same inputs
    for call in range(2):
        ref, ref_offs = _compress(N.nlc_compress, codec, batches[call], patch, layout, cap)
        assert torch.equal(offs[call], ref_offs)
        end = int(ref_offs[-1])
        assert torch.equal(outs[call][:end], ref[:end])
        dec = codec.decompress(outs[call], offs[call], sizes, patch, layout,
                               N.NLC_SCHED_WAVEFRONT if layout == N.NLC_LAYOUT_ROW
                               else N.NLC_SCHED_SEQUENTIAL)
        for a, b in zip(dec, batches[call]):
            assert torch.equal(a, b)


def test_noalloc_rejects_batches_beyond_its_scratch():
    codec, _ = make_codec((1, 16, 0, 2), N.NLC_FP32, seed=22)
    # 1400 x 1400 pixels need about 23.5 MB of staging plus 11.8 MB of stream bytes
    big = torch.zeros((1400, 1400, 3), dtype=torch.uint8, device=DEV)
    out = torch.zeros(16, dtype=torch.uint8, device=DEV)
    offs = torch.zeros(2, dtype=torch.int64, device=DEV)
    with pytest.raises(N.NLCError) as e:
        N.nlc_compress_noalloc(codec.ctx, [big], 0, 1, out, offs)
    assert e.value.code == N.NLC_ERR_CAPACITY
    assert b"scratch" in N.load().nlc_last_error()
    assert N.nlc_sync_status(codec.ctx) == N.NLC_OK
