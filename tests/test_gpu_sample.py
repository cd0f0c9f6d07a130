"""The wavefront sampler (nlc_sample) through the C ABI: every schedule draws
the same images, each symbol is the inverse CDF of the GPU's own table at the
counter-based generator's uniform (computed here by the oracle's
independent SplitMix64), and a pixel with an empty context follows the
oracle's table (chi-square)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_05213_gb300 import nlc as N

from gpu_util import DEV, ensure_built, make_codec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("prec,patch", [(N.NLC_BF16, 0), (N.NLC_BF16, 16), (N.NLC_FP32, 0)])
def test_sampler_schedules_agree_and_follow_the_tables(prec, patch):
    cfg = (3, 32, 1, 10)
    codec, _ = make_codec(cfg, prec, seed=31)
    sizes = [(20, 37), (33, 16), (1, 5), (16, 16)]
    seed = 12345
    outs = {s: [o.cpu().numpy() for o in codec.sample(sizes, patch, seed, s)]
            for s in (N.NLC_SCHED_WAVEFRONT, N.NLC_SCHED_RASTER, N.NLC_SCHED_SEQUENTIAL)}
    for s in (N.NLC_SCHED_RASTER, N.NLC_SCHED_SEQUENTIAL):
        for a, b in zip(outs[N.NLC_SCHED_WAVEFRONT], outs[s]):
            assert np.array_equal(a, b), s
    imgs = outs[N.NLC_SCHED_WAVEFRONT]
    dimgs = [torch.from_numpy(i).to(DEV) for i in imgs]
    P, _ = codec.forward(dimgs, patch)
    pix = torch.cat([d.reshape(-1, 3) for d in dimgs])
    cum = codec.tables(P, pix).cpu().numpy().astype(np.int64)
    q = 0
    for n, img in enumerate(imgs):
        H, W = img.shape[:2]
        for y in range(H):
            for x in range(W):
                for c in range(3):
                    v = int(img[y, x, c])
                    u = O.sample_u16(seed, n, y, x, c)
                    assert cum[q, c, v] <= u < cum[q, c, v + 1], (n, y, x, c)
                q += 1
    # a different seed gives different images
    other = codec.sample(sizes, patch, seed + 1)
    assert any(not np.array_equal(o.cpu().numpy(), i) for o, i in zip(other, imgs))


def test_sampler_empty_context_matches_oracle_table():
    cfg = (1, 16, 0, 4)
    codec, w = make_codec(cfg, N.NLC_BF16, seed=9, scale=3.0)
    n = 6000  # units of one call: the decoder keeps a prefix per unit in shared memory
    outs = codec.sample([(1, 1)] * n, 0, 11)
    vals = np.array([int(o[0, 0, 0]) for o in torch.stack(outs).cpu()])
    out = O.forward_image(cfg, w.astype(np.float64), np.zeros((1, 1, 3), np.uint8))[0, 0]
    p = np.diff(O.pixel_tables(cfg[3], out, 0, 0)[0].astype(np.int64)) / 65536.0
    obs = np.bincount(vals, minlength=256).astype(np.float64)
    exp = p * n
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


def test_sampler_rejects_bad_arguments():
    codec, _ = make_codec((1, 16, 0, 2), N.NLC_FP32, seed=1)
    with pytest.raises(N.NLCError) as e:
        codec.sample([(4, 4)], 0, 1, schedule=7)
    assert e.value.code == N.NLC_ERR_ARG
