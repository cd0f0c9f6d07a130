"""Pins of the oracle's sampler (Section 5: the parallel schedules also serve
sampling from a local autoregressive model): the counter-based generator
against SplitMix64's known-answer values, the drawn symbols against their
quantised tables, and the empirical distribution of a pixel with an empty
context against its table (chi-square)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2201_05213_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return [int(l) for l in f if l.strip() and not l.startswith("#")]


def test_splitmix64_known_answers():
    ref = _golden("splitmix64_seed1234567.txt")
    assert [O.splitmix64(1234567, k) for k in range(5)] == ref


def test_sample_counter_layout():
    # channel c of pixel (y, x) of image n uses output ((n 2^21 + y) 2^21 + x) 3 + c
    for n, y, x, c in [(0, 0, 0, 0), (3, 17, 200, 2), (1, 2047, 5, 1)]:
        k = ((n * 2 ** 21 + y) * 2 ** 21 + x) * 3 + c
        assert O.sample_u16(99, n, y, x, c) == O.splitmix64(99, k) >> 48
    vals = {O.sample_u16(5, 0, 0, 0, c) for c in range(3)}
    assert len(vals) == 3


@pytest.mark.parametrize("patch", [0, 5])
def test_sampled_symbols_are_the_tables_inverse_cdf(patch):
    cfg = (2, 8, 1, 3)
    w = synth.xavier_weights(*cfg, seed=2) * 2
    H, W, seed, n = 9, 11, 77, 4
    img = O.sample_image(cfg, w, H, W, patch, seed, n)
    outs = O.forward_image(cfg, w, img, patch)
    for y in range(H):
        for x in range(W):
            r, g, b = (int(v) for v in img[y, x])
            cum = O.pixel_tables(cfg[3], outs[y, x], r, g)
            for c, v in enumerate((r, g, b)):
                u = O.sample_u16(seed, n, y, x, c)
                assert cum[c][v] <= u < cum[c][v + 1], (y, x, c)
    # another seed gives another image; the same seed the same one
    assert (O.sample_image(cfg, w, H, W, patch, seed + 1, n) != img).any()
    assert (O.sample_image(cfg, w, H, W, patch, seed, n) == img).all()


def test_empty_context_pixel_follows_its_table():
    # a 1x1 image has an empty context: its R value is drawn from one fixed
    # table; 3000 images (different counters) against it, chi-square with
    # bins merged to expected counts >= 5, at the 1e-4 level
    cfg = (1, 8, 0, 4)
    w = synth.xavier_weights(*cfg, seed=9) * 3
    n = 3000
    vals = np.array([O.sample_image(cfg, w, 1, 1, 0, 11, k)[0, 0, 0] for k in range(n)])
    out = O.forward_image(cfg, w, np.zeros((1, 1, 3), np.uint8))[0, 0]
    cum = O.pixel_tables(cfg[3], out, 0, 0)[0].astype(np.int64)
    p = np.diff(cum) / 65536.0
    obs = np.bincount(vals, minlength=256).astype(np.float64)
    exp = p * n
    # merge adjacent bins until each expected count is >= 5
    o_b, e_b, oa, ea = [], [], 0.0, 0.0
    for k in range(256):
        oa += obs[k]
        ea += exp[k]
        if ea >= 5:
            o_b.append(oa)
            e_b.append(ea)
            oa = ea = 0.0
    o_b[-1] += oa
    e_b[-1] += ea
    o_b, e_b = np.array(o_b), np.array(e_b)
    chi2 = float(((o_b - e_b) ** 2 / e_b).sum())
    from scipy import stats
    assert len(o_b) >= 5
    assert stats.chi2.sf(chi2, len(o_b) - 1) > 1e-4, chi2
