"""Stage parity of the CUDA path against the FP64 oracle, through the C ABI.

Network outputs (Section 2.1 local PixelCNN): |delta| <= 1e-4 max(1, |ref|)
in FP32 and <= 2e-2 absolute in BF16.  Frequency tables: valid (every
frequency >= 1, sum 2^16) and within 2 counts of the oracle's, which
quantises the same FP32 network outputs in FP64.  rANS (Section 2, ANS):
byte-identical streams and symbols given the oracle's tables.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_05213_gb300 import nlc as N

from gpu_util import DEV, ensure_built, images, make_codec, to_dev

pytestmark = pytest.mark.gpu

SIZES = [(37, 29), (16, 70), (5, 3), (1, 1), (2, 9)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _oracle_params(cfg, w, imgs, patch):
    return np.concatenate([O.forward_image(cfg, w, im, patch).reshape(-1, 10 * cfg[3])
                           for im in imgs])


@pytest.mark.parametrize("cfg,patch", [((3, 32, 2, 10), 0), ((3, 32, 2, 10), 16),
                                       ((1, 16, 1, 4), 8), ((2, 48, 0, 3), 0)])
def test_forward_fp32_matches_oracle(cfg, patch):
    codec, w = make_codec(cfg, N.NLC_FP32, seed=1)
    imgs = images(3, SIZES)
    P, _ = codec.forward([to_dev(i) for i in imgs], patch)
    ref = _oracle_params(cfg, w, imgs, patch)
    got = P.cpu().numpy().astype(np.float64)
    assert got.shape == ref.shape
    err = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() <= 1e-4, err.max()


@pytest.mark.parametrize("cfg,patch", [((3, 64, 2, 10), 0), ((3, 64, 2, 10), 16),
                                       ((1, 32, 1, 4), 8), ((2, 16, 0, 3), 0)])
def test_forward_bf16_matches_oracle(cfg, patch):
    codec, w = make_codec(cfg, N.NLC_BF16, seed=2)
    imgs = images(4, SIZES)
    P, _ = codec.forward([to_dev(i) for i in imgs], patch)
    ref = _oracle_params(cfg, w, imgs, patch)
    got = P.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 2e-2, np.abs(got - ref).max()


def test_bf16_rows_independent_of_tile_position():
    # the same pixels computed in different tile rows give identical outputs
    cfg = (3, 64, 2, 10)
    codec, _ = make_codec(cfg, N.NLC_BF16, seed=3)
    img = images(5, [(20, 20)])[0]
    a, _ = codec.forward([to_dev(img)])
    pad = images(6, [(1, 37)])[0]
    b, _ = codec.forward([to_dev(pad), to_dev(img)])
    assert torch.equal(a, b[37:])


def _check_tables(cum):
    c = cum.astype(np.int64)
    assert (c[..., 0] == 0).all() and (c[..., 256] == 65536).all()
    assert (np.diff(c, axis=-1) >= 1).all()


@pytest.mark.parametrize("prec", [N.NLC_FP32, N.NLC_BF16])
def test_tables_match_oracle(prec):
    cfg = (3, 32, 2, 10)
    codec, w = make_codec(cfg, prec, seed=4, scale=2.5)
    imgs = images(7, [(24, 24)])
    ref_params = _oracle_params(cfg, w, imgs, 0).astype(np.float32)
    pix = imgs[0].reshape(-1, 3)
    cum = codec.tables(torch.from_numpy(ref_params).to(DEV), to_dev(pix)).cpu().numpy()
    _check_tables(cum)
    worst = 0
    for q in range(len(pix)):
        ref = O.pixel_tables(10, ref_params[q].astype(np.float64), pix[q, 0], pix[q, 1])
        worst = max(worst, int(np.abs(cum[q].astype(np.int64) - ref.astype(np.int64)).max()))
    assert worst <= 2, worst


def test_tables_extreme_parameters():
    # very sharp, very flat, saturated and far-off components stay valid
    cfg = (1, 16, 0, 3)
    codec, _ = make_codec(cfg, N.NLC_FP32)
    rng = np.random.default_rng(0)
    n = 64
    P = rng.normal(0, 30, (n, 30)).astype(np.float32)
    P[:, 12:21] = rng.choice([-20.0, -7.5, 0.0, 4.0, 12.0], (n, 9))
    pix = rng.integers(0, 256, (n, 3)).astype(np.uint8)
    cum = codec.tables(torch.from_numpy(P).to(DEV), torch.from_numpy(pix).to(DEV)).cpu().numpy()
    _check_tables(cum)


def test_tables_non_finite_parameters():
    # NaN and infinite network outputs (e.g. from corrupt weights) still give
    # valid tables: the locations are bounded before the CDF, the weights and
    # scales stay finite, so every term is a number and F stays monotone
    cfg = (1, 16, 0, 10)
    codec, _ = make_codec(cfg, N.NLC_FP32)
    rng = np.random.default_rng(1)
    n = 96
    P = rng.normal(0, 3, (n, 100)).astype(np.float32)
    bad = rng.random((n, 100)) < 0.2
    P[bad] = rng.choice(np.array([np.nan, np.inf, -np.inf], dtype=np.float32), bad.sum())
    P[:8] = np.nan  # whole rows
    P[8:16, 10:40] = np.inf
    pix = rng.integers(0, 256, (n, 3)).astype(np.uint8)
    cum = codec.tables(torch.from_numpy(P).to(DEV), torch.from_numpy(pix).to(DEV)).cpu().numpy()
    _check_tables(cum)


def _rand_tables(rng, n):
    tabs = []
    for _ in range(n):
        p = rng.dirichlet(np.full(256, rng.choice([0.05, 1.0, 10.0])))
        F = np.concatenate([[0], np.cumsum(p)])
        F[256] = 1
        tabs.append(O.quantise_cdf(F))
    return np.stack(tabs)


@pytest.mark.parametrize("nstreams", [1, 7, 40])
def test_rans_matches_oracle(nstreams):
    rng = np.random.default_rng(nstreams)
    lens_sym = rng.integers(0, 300, nstreams)
    lens_sym[0] = 0 if nstreams > 1 else lens_sym[0]
    off = np.concatenate([[0], np.cumsum(lens_sym)]).astype(np.int64)
    tot = int(off[-1])
    tabs = _rand_tables(rng, max(tot, 1))[:tot]
    sym = np.array([rng.choice(256, p=np.diff(t.astype(np.int64)) / 65536) for t in tabs],
                   dtype=np.int64)
    start = tabs[np.arange(tot), sym].astype(np.uint32)
    freq = (tabs[np.arange(tot), sym + 1] - start).astype(np.uint32)
    ref = [O.rans_encode(start[off[s]:off[s + 1]], freq[off[s]:off[s + 1]])
           for s in range(nstreams)]
    stride = int(2 * lens_sym.max() + 8) if tot else 8
    out = torch.zeros(nstreams * stride, dtype=torch.uint8, device=DEV)
    lens = torch.zeros(nstreams, dtype=torch.int32, device=DEV)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(DEV)
    N.nlc_rans_encode(t(start, np.int32) if tot else t(np.zeros(1), np.int32),
                      t(freq, np.int32) if tot else t(np.zeros(1), np.int32),
                      t(off, np.int64), out, stride, lens)
    got_lens = lens.cpu().numpy()
    buf = out.cpu().numpy().reshape(nstreams, stride)
    for s in range(nstreams):
        assert got_lens[s] == len(ref[s])
        np.testing.assert_array_equal(buf[s, stride - got_lens[s]:], ref[s])
    # decode the oracle's bytes with the oracle's tables on the GPU
    codec, _ = make_codec((1, 16, 0, 1), N.NLC_FP32)
    dbuf = np.zeros((nstreams, stride), np.uint8)
    for s in range(nstreams):
        dbuf[s, stride - len(ref[s]):] = ref[s]
    dsym = torch.zeros(max(tot, 1), dtype=torch.int32, device=DEV)
    cum = t(tabs if tot else np.zeros((1, 257)), np.int32)
    N.nlc_rans_decode(codec.ctx, t(dbuf.ravel(), np.uint8), stride,
                      t([len(r) for r in ref], np.int32), cum, t(off, np.int64), dsym)
    assert N.nlc_sync_status(codec.ctx) == N.NLC_OK
    np.testing.assert_array_equal(dsym.cpu().numpy()[:tot], sym)
    # a damaged stream is reported
    if tot > 10:
        bad = dbuf.copy()
        s = int(np.argmax(lens_sym))
        bad[s, stride - len(ref[s]) + 5] ^= 0x41
        N.nlc_rans_decode(codec.ctx, t(bad.ravel(), np.uint8), stride,
                          t([len(r) for r in ref], np.int32), cum, t(off, np.int64), dsym)
        assert N.nlc_sync_status(codec.ctx) == N.NLC_ERR_CORRUPT


def test_mufu_probe_rate_is_plausible():
    # the roofline denominator: MUFU ops/s of the search's ex2 + rcp pair;
    # between 1 and 64 operations per clock and SM at the device's clocks
    rate, ms = N.nlc_measure_mufu(4000)
    props = torch.cuda.get_device_properties(0)
    per_clk_sm = rate / (props.multi_processor_count * 2.07e9)
    assert ms > 0 and 1.0 <= per_clk_sm <= 64.0, per_clk_sm
