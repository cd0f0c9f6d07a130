"""End-to-end parity of the CUDA codec through the C ABI.

Decoded pixels must equal the input bit for bit under every schedule
(Section 4: sequential, wavefront and patch decoding give the same result),
code lengths must match the oracle's model (|delta bpd| <= 0.01 FP32,
<= 0.03 BF16) and the bytes must be within 32 bits per stream of the
tables' ideal length; malformed inputs must be reported, not decoded
silently.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_05213_gb300 import codec as CD
from paper_2201_05213_gb300 import nlc as N
from paper_2201_05213_gb300 import synth

from gpu_util import DEV, ensure_built, images, make_codec, to_dev

pytestmark = pytest.mark.gpu

SCHEDS = [N.NLC_SCHED_WAVEFRONT, N.NLC_SCHED_RASTER, N.NLC_SCHED_SEQUENTIAL]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _round_trip(codec, imgs, patch, layout, scheds=SCHEDS):
    dimgs = [to_dev(i) for i in imgs]
    data, offs = codec.compress(dimgs, patch, layout)
    sizes = [i.shape[:2] for i in imgs]
    for sch in scheds:
        if layout == N.NLC_LAYOUT_UNIT and sch == N.NLC_SCHED_WAVEFRONT:
            continue
        outs = codec.decompress(data, offs, sizes, patch, layout, sch)
        for a, b in zip(outs, imgs):
            assert np.array_equal(a.cpu().numpy(), b), (patch, layout, sch)
    return data, offs


@pytest.mark.parametrize("prec,cfg", [(N.NLC_FP32, (3, 32, 2, 10)), (N.NLC_BF16, (3, 64, 2, 10)),
                                      (N.NLC_FP32, (1, 16, 1, 4)), (N.NLC_BF16, (2, 32, 1, 10))])
@pytest.mark.parametrize("patch,layout", [(0, 1), (16, 1), (0, 0), (13, 0)])
def test_round_trip_all_schedules(prec, cfg, patch, layout):
    codec, _ = make_codec(cfg, prec, seed=5, scale=2.0)
    imgs = images(11, [(33, 41), (16, 16), (1, 7), (9, 1), (2, 2), (20, 3)])
    _round_trip(codec, imgs, patch, layout)


@pytest.mark.parametrize("prec,cfg", [(N.NLC_FP32, (3, 32, 2, 10)), (N.NLC_BF16, (2, 32, 1, 10))])
def test_round_trip_with_non_finite_network_outputs(prec, cfg):
    # head biases set to NaN / +-inf make those outputs non-finite for every
    # pixel (a logit, locations, a log-scale, a coupling coefficient): the
    # tables stay valid, so the codec still round-trips
    h, C, R, K = cfg
    w = synth.xavier_weights(h, C, R, K, seed=7) * np.float32(2.0)
    bH = w[len(w) - 10 * K:]
    bH[3] = np.nan                # logit of component 3
    bH[K + 2] = np.nan            # R location of component 2
    bH[2 * K + 5] = np.inf        # G location of component 5
    bH[4 * K + 1] = np.inf        # R log-scale of component 1
    bH[5 * K + 4] = -np.inf       # G log-scale of component 4
    bH[7 * K + 6] = np.nan        # a coupling coefficient of component 6
    bH[9 * K + 8] = -np.inf
    codec = CD.Codec(h, C, R, K, prec, w)
    imgs = images(21, [(19, 23), (8, 8)])
    _round_trip(codec, imgs, 0, 1, [N.NLC_SCHED_WAVEFRONT, N.NLC_SCHED_SEQUENTIAL])


def test_decode_profile_runs_the_instrumented_build():
    # profiling switches decodes to the instrumented decoder (a plan made
    # before it was switched on runs it too); its counters fill, and both
    # builds decode the same pixels
    codec, _ = make_codec((3, 64, 2, 10), N.NLC_BF16, seed=5)
    imgs = images(31, [(64, 80), (40, 40)])
    dimgs = [to_dev(i) for i in imgs]
    data, offs = codec.compress(dimgs, 32, 1)
    sizes = [i.shape[:2] for i in imgs]
    plan = codec.plan(sizes, 32, 1)

    def same(outs):
        for a, b in zip(outs, imgs):
            assert np.array_equal(a.cpu().numpy(), b)

    plan.run(data, offs)
    codec.check()
    same(plan.outs)
    N.nlc_decode_profile(codec.ctx, 1, read=False)
    for o in plan.outs:
        o.zero_()
    plan.run(data, offs)
    codec.check()
    same(plan.outs)
    cnt = N.nlc_decode_profile(codec.ctx, 0)  # read, clear, switch off
    T = 32 + 31 * 4  # the largest unit's steps: 32 x 32 patches, h = 3
    assert int(cnt[7]) == T and int(cnt[6]) >= 1
    assert all(int(cnt[i]) > 0 for i in (0, 2, 3, 8, 9, 12, 13, 14, 15))
    same(codec.decompress(data, offs, sizes, 32, 1))
    assert int(N.nlc_decode_profile(codec.ctx, 0)[3]) == 0  # off: nothing recorded


def test_edge_cases():
    codec, _ = make_codec((3, 32, 2, 10), N.NLC_FP32, seed=6)
    # empty batch
    data, offs = codec.compress([], 0, 1) if False else (None, None)
    out = torch.zeros(16, dtype=torch.uint8, device=DEV)
    offs = torch.zeros(1, dtype=torch.int64, device=DEV)
    N.nlc_compress(codec.ctx, [], 0, 1, out, offs)
    assert N.nlc_sync_status(codec.ctx) == N.NLC_OK
    assert int(offs[0]) == 0
    N.nlc_decompress(codec.ctx, out, offs, [], 0, 1, N.NLC_SCHED_WAVEFRONT)
    # zero-sized images next to real ones; h >= W; single pixel
    imgs = [np.zeros((0, 5, 3), np.uint8)] + images(12, [(1, 1), (5, 2), (3, 3)])
    dimgs = [to_dev(i) for i in imgs]
    data, offs = codec.compress(dimgs, 0, 1)
    outs = codec.decompress(data, offs, [i.shape[:2] for i in imgs], 0, 1)
    for a, b in zip(outs, imgs):
        assert np.array_equal(a.cpu().numpy(), b)


@pytest.mark.parametrize("prec", [N.NLC_FP32, N.NLC_BF16])
@pytest.mark.parametrize("tuning", [(1, 0), (8, 0), (4096, 0), (8, 1), (1, 3)])
def test_decoder_work_split(prec, tuning):
    # many pixels per CTA (several tiles per step), one CTA, odd grids
    cfg = (3, 32, 2, 10)
    codec, _ = make_codec(cfg, prec, seed=7, scale=2.0)
    N.nlc_set_tuning(codec.ctx, *tuning)
    imgs = images(13, [(70, 300), (31, 17), (64, 64)])
    _round_trip(codec, imgs, 0, 1, [N.NLC_SCHED_WAVEFRONT])


def test_deterministic_and_batch_independent():
    # O12: the encoder's tables of a pixel do not depend on its tile position
    codec, _ = make_codec((3, 64, 2, 10), N.NLC_BF16, seed=8, scale=2.0)
    imgs = images(14, [(30, 50), (17, 9), (40, 40)])
    d1, o1 = codec.compress([to_dev(i) for i in imgs], 0, 1)
    d2, o2 = codec.compress([to_dev(i) for i in imgs], 0, 1)
    assert torch.equal(o1, o2) and torch.equal(d1[: int(o1[-1])], d2[: int(o2[-1])])
    rev = imgs[::-1]
    d3, o3 = codec.compress([to_dev(i) for i in rev], 0, 1)
    a = d1.cpu().numpy()
    b = d3.cpu().numpy()
    o1n, o3n = o1.cpu().numpy(), o3.cpu().numpy()
    for k in range(3):
        r = 2 - k
        assert np.array_equal(a[o1n[k]:o1n[k + 1]], b[o3n[r]:o3n[r + 1]])


@pytest.mark.parametrize("prec,tol", [(N.NLC_FP32, 0.01), (N.NLC_BF16, 0.03)])
def test_code_length_matches_oracle(prec, tol):
    cfg = (3, 32, 2, 10) if prec == N.NLC_FP32 else (3, 64, 2, 10)
    codec, w = make_codec(cfg, prec, seed=9)
    imgs = images(15, [(40, 48), (24, 24)])
    dims = sum(3 * i.shape[0] * i.shape[1] for i in imgs)
    dimgs = [to_dev(i) for i in imgs]
    _, bits = codec.forward(dimgs, 0, params=False, bits=True)
    gpu_bpd = float(bits.double().sum()) / dims
    ref_bits = 0.0
    for im in imgs:
        P = O.forward_image(cfg, w, im).reshape(-1, 10 * cfg[3])
        pix = im.reshape(-1, 3)
        ref_bits += sum(O.pixel_bits(cfg[3], P[q], *pix[q]) for q in range(len(pix)))
    assert abs(gpu_bpd - ref_bits / dims) <= tol, (gpu_bpd, ref_bits / dims)
    # actual bytes: within 32 bits per stream (+ headers) of the tables' ideal length
    data, offs = codec.compress(dimgs, 0, 1)
    P, _ = codec.forward(dimgs, 0)
    pix = torch.cat([t.reshape(-1, 3) for t in dimgs])
    cum = codec.tables(P, pix)
    ideal = CD.ideal_bits_from_tables(cum, pix)
    nstreams = sum(i.shape[0] for i in imgs)
    payload = int(offs[-1]) - sum(32 + _len_width(*i.shape[:2], 0, 1) * i.shape[0] for i in imgs)
    assert 8 * payload <= ideal + 32 * nstreams + 8 * 16 * len(imgs)
    assert 8 * payload >= ideal - 1


def test_malformed_input_is_reported():
    codec, w = make_codec((2, 16, 1, 4), N.NLC_FP32, seed=10, scale=2.0)
    imgs = images(16, [(20, 30), (12, 12)])
    dimgs = [to_dev(i) for i in imgs]
    data, offs = codec.compress(dimgs, 0, 1)
    sizes = [i.shape[:2] for i in imgs]
    # flipped payload byte: reported or at least not silently equal
    bad = data.clone()
    pos = int(offs[0]) + 32 + 4 * 20 + 40
    bad[pos] ^= 0x5A
    outs = codec.decompress(bad, offs, sizes, 0, 1, check=False)
    code = N.nlc_sync_status(codec.ctx)
    assert code == N.NLC_ERR_CORRUPT or not np.array_equal(outs[0].cpu().numpy(), imgs[0])
    # broken magic
    bad = data.clone()
    bad[int(offs[1])] ^= 0xFF
    codec.decompress(bad, offs, sizes, 0, 1, check=False)
    assert N.nlc_sync_status(codec.ctx) == N.NLC_ERR_CORRUPT
    # truncated container
    offs2 = offs.clone()
    offs2[2] = offs2[2] - 40
    codec.decompress(data, offs2, sizes, 0, 1, check=False)
    assert N.nlc_sync_status(codec.ctx) == N.NLC_ERR_CORRUPT
    # wrong sizes for the container
    codec.decompress(data, offs, [(20, 31), (12, 12)], 0, 1, check=False)
    assert N.nlc_sync_status(codec.ctx) == N.NLC_ERR_CORRUPT
    # other weights
    other, _ = make_codec((2, 16, 1, 4), N.NLC_FP32, seed=11, scale=2.0)
    other.decompress(data, offs, sizes, 0, 1, check=False)
    assert N.nlc_sync_status(other.ctx) == N.NLC_ERR_WEIGHTS
    # output too small
    out = torch.zeros(64, dtype=torch.uint8, device=DEV)
    o = torch.zeros(3, dtype=torch.int64, device=DEV)
    N.nlc_compress(codec.ctx, dimgs, 0, 1, out, o)
    assert N.nlc_sync_status(codec.ctx) == N.NLC_ERR_CAPACITY
    # wavefront on one stream per unit is an argument error
    with pytest.raises(N.NLCError):
        codec.decompress(data, offs, sizes, 0, 0, N.NLC_SCHED_WAVEFRONT)
    # a negative image count is an argument error of every batch entry point
    L, ctx = N.load(), codec.ctx
    p = ctypes.c_void_p(dimgs[0].data_ptr())
    assert L.nlc_compress(ctx, p, -1, 0, 1, p, 16, p, None) == N.NLC_ERR_ARG
    assert L.nlc_compress_noalloc(ctx, p, -1, 0, 1, p, 16, p, None) == N.NLC_ERR_ARG
    assert L.nlc_decompress(ctx, p, p, p, -1, 0, 1, 1, None) == N.NLC_ERR_ARG
    assert L.nlc_forward(ctx, p, -1, 0, p, None, None) == N.NLC_ERR_ARG
    assert N.nlc_sync_status(codec.ctx) == N.NLC_OK


def test_oracle_decodes_same_partition_same_pixels():
    # the oracle's own raster codec and the GPU codec agree on the decoded image
    cfg = (3, 32, 2, 10)
    codec, w = make_codec(cfg, N.NLC_FP32, seed=0)
    img = images(0, [(32, 32)])[0]
    words, lens, bm, bq = O.encode_image(cfg, w, img, 0, 0)
    dec, ok = O.decode_image(cfg, w, words, lens, 32, 32, 0, 0)
    assert ok and (dec == img).all()
    data, offs = codec.compress([to_dev(img)], 0, 0)
    outs = codec.decompress(data, offs, [(32, 32)], 0, 0, N.NLC_SCHED_SEQUENTIAL)
    assert np.array_equal(outs[0].cpu().numpy(), dec)
    # one stream each: the payloads differ only through FP32 vs FP64 tables
    assert abs((int(offs[1]) - 32 - _len_width(32, 32, 0, 0)) - len(words)) <= 16
    assert 8 * len(words) <= bq + 32 + 1


@pytest.mark.parametrize("prec", [N.NLC_FP32, N.NLC_BF16])
def test_streams_equal_oracle_rans_on_gpu_tables(prec):
    # the container's per-row streams are byte-identical to the oracle's rANS
    # encoder fed the GPU's own tables (nlc_tables over nlc_forward's outputs)
    cfg = (2, 32, 1, 10)
    codec, _ = make_codec(cfg, prec, seed=12)
    img = images(17, [(20, 36)])[0]
    H, W = img.shape[:2]
    d = to_dev(img)
    data, offs = codec.compress([d], 0, 1)
    P, _ = codec.forward([d], 0)
    cum = codec.tables(P, d.reshape(-1, 3)).cpu().numpy().astype(np.int64)
    _check_increasing(cum)
    v = img.reshape(-1, 3).astype(np.int64)
    px, ch = np.arange(len(v))[:, None], np.arange(3)[None, :]
    start = cum[px, ch, v]
    freq = cum[px, ch, v + 1] - start
    buf = data.cpu().numpy()[int(offs[0]):int(offs[1])]
    assert _len_width(H, W, 0, 1) == 2
    lens = buf[32:32 + 2 * H].copy().view("<u2")
    pos = 32 + 2 * H
    for r in range(H):
        rows = slice(r * W, (r + 1) * W)
        ref = O.rans_encode(start[rows].reshape(-1), freq[rows].reshape(-1))
        assert np.array_equal(buf[pos:pos + int(lens[r])], ref), r
        pos += int(lens[r])


def _len_width(H, W, patch, layout):
    """Bytes per stream-length entry of a container (include/nlc.h): 2 when
    6 x (pixels of the image's largest stream) + 4 < 2^16, else 4."""
    P = patch if patch > 0 else max(H, W)
    px = min(W, P) if layout == 1 else min(H, P) * min(W, P)
    return 2 if 6 * px + 4 < 65536 else 4


def test_wide_rows_use_four_byte_lengths():
    # rows of 11000 pixels can exceed 2^16 bytes: 4-byte length entries
    codec, _ = make_codec((1, 16, 0, 2), N.NLC_BF16, seed=60)
    sizes = [(3, 11000), (5, 7)]
    imgs = images(61, sizes)
    d = [to_dev(i) for i in imgs]
    data, offs = codec.compress(d, 0, 1)
    assert _len_width(3, 11000, 0, 1) == 4 and _len_width(5, 7, 0, 1) == 2
    lens = data.cpu().numpy()[int(offs[0]) + 32:int(offs[0]) + 32 + 12].copy().view("<u4")
    assert int(offs[0]) + 32 + 12 + int(lens.sum()) <= int(offs[1])
    for sched in (N.NLC_SCHED_WAVEFRONT, N.NLC_SCHED_RASTER):
        outs = codec.decompress(data, offs, sizes, 0, 1, sched)
        for o, i in zip(outs, imgs):
            assert np.array_equal(o.cpu().numpy(), i)


def _check_increasing(cum):
    assert (cum[..., 0] == 0).all() and (cum[..., 256] == 65536).all()
    assert (np.diff(cum, axis=-1) >= 1).all()


def test_plan_graph_replay_and_tuner():
    # a decode plan issues device work only: it runs, tunes its pixels per CTA,
    # and its CUDA-graph capture decodes whatever containers are in the
    # captured buffers at replay time
    codec, _ = make_codec((3, 64, 2, 10), N.NLC_BF16, seed=1)
    sizes = [(96, 80), (64, 64), (33, 47)]
    imgs = images(21, sizes)
    data, offs = codec.compress([to_dev(i) for i in imgs], 32, 1)
    plan = codec.plan(sizes, 32, 1)
    outs = plan.run(data, offs)
    codec.check()
    for o, i in zip(outs, imgs):
        assert np.array_equal(o.cpu().numpy(), i)
    ppc, ms = plan.tune(data, offs, reps=1)
    assert ppc in (1, 2, 4, 8, 16, 32, 64, 128) and ms > 0
    codec.check()
    g = plan.graph(data, offs)
    for o in plan.outs:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    codec.check()
    for o, i in zip(plan.outs, imgs):
        assert np.array_equal(o.cpu().numpy(), i)
    imgs2 = images(22, sizes)
    data2, offs2 = codec.compress([to_dev(i) for i in imgs2], 32, 1)
    assert data2.numel() == data.numel()
    data.copy_(data2)
    offs.copy_(offs2)
    g.replay()
    torch.cuda.synchronize()
    codec.check()
    for o, i in zip(plan.outs, imgs2):
        assert np.array_equal(o.cpu().numpy(), i)
    plan.close()


def test_step_times_give_image_latencies():
    # the decoder's step end times are non-decreasing, and an image finishes at
    # its units' last wavefront step (W + (H-1)(h+1) steps, Algorithm 1)
    h = 2
    codec, _ = make_codec((h, 32, 1, 10), N.NLC_BF16, seed=2)
    sizes = [(64, 48), (16, 16), (40, 100)]
    imgs = images(23, sizes)
    data, offs = codec.compress([to_dev(i) for i in imgs], 0, 1)
    steps = [W + (H - 1) * (h + 1) for H, W in sizes]
    times = torch.full((max(steps) + 5,), -1, dtype=torch.int64, device=DEV)
    N.nlc_decode_step_times(codec.ctx, times)
    outs = codec.decompress(data, offs, sizes, 0, 1)
    N.nlc_decode_step_times(codec.ctx, None)
    for o, i in zip(outs, imgs):
        assert np.array_equal(o.cpu().numpy(), i)
    t = times.cpu().numpy()
    T = max(steps)
    assert t[0] > 0 and (np.diff(t[:T + 1]) >= 0).all() and (t[T + 1:] == 0).all()
    lat = [t[s] - t[0] for s in steps]
    assert lat[1] <= lat[2] <= lat[0] and lat[0] == t[T] - t[0]


@pytest.mark.parametrize("prec", [N.NLC_BF16, N.NLC_BF16_SHEARED])
def test_bounded_waits_report_timeouts_and_the_context_recovers(prec):
    # The decoder's waits are bounded: a grid-barrier wait or an MMA
    # completion wait that gives up records NLC_ERR_TIMEOUT and releases every
    # CTA; the launch ends and the context decodes again with normal limits.
    codec, _ = make_codec((3, 32, 1, 10), prec, seed=50)
    sizes = [(48, 48)] * 4
    imgs = images(51, sizes)
    d = [to_dev(i) for i in imgs]
    data, offs = codec.compress(d, 16, N.NLC_LAYOUT_ROW)
    N.nlc_set_tuning(codec.ctx, 1, 0)  # one pixel per CTA and step: many CTAs meet each step
    for grid_polls, mma_polls in ((1, 0), (0, 1)):
        N.nlc_set_wait_limits(codec.ctx, grid_polls, mma_polls)
        codec.decompress(data, offs, sizes, 16, N.NLC_LAYOUT_ROW, check=False)
        assert N.nlc_sync_status(codec.ctx) == N.NLC_ERR_TIMEOUT, (grid_polls, mma_polls)
        N.nlc_set_wait_limits(codec.ctx, 0, 0)
        outs = codec.decompress(data, offs, sizes, 16, N.NLC_LAYOUT_ROW)
        for o, i in zip(outs, imgs):
            assert np.array_equal(o.cpu().numpy(), i)
