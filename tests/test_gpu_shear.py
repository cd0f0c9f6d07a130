"""The sheared model (ShearLoC, Section 3.1) through the C ABI: the first
layer evaluated as Fig. 5's sheared kernels.  Round trips under every
schedule (the wavefront decoder keeps decoded pixels in sheared rings and
reads each front's context as one window tile; raster and sequential decode
gather per pixel, so a round trip across them also shows that both
arrangements give the same bits), network outputs and code length against
the oracle at the BF16 tolerances, and containers that are the sheared
model's own."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_05213_gb300 import codec as CD
from paper_2201_05213_gb300 import nlc as N
from paper_2201_05213_gb300 import synth

from gpu_util import DEV, ensure_built, images, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _codec(cfg, seed, prec=N.NLC_BF16_SHEARED, scale=1.0):
    w = synth.xavier_weights(*cfg, seed=seed) * np.float32(scale)
    return CD.Codec(*cfg, prec, w), w


@pytest.mark.parametrize("cfg,patch", [((3, 64, 2, 10), 0), ((3, 64, 2, 10), 16),
                                       ((1, 32, 1, 4), 0), ((2, 48, 0, 6), 8)])
def test_sheared_round_trip_every_schedule(cfg, patch):
    codec, _ = _codec(cfg, 40, scale=1.5)
    sizes = [(37, 53), (16, 16), (1, 9), (9, 1), (5, 3), (64, 20)]
    imgs = images(41, sizes)
    d = [to_dev(i) for i in imgs]
    data, offs = codec.compress(d, patch, N.NLC_LAYOUT_ROW)
    for sched in (N.NLC_SCHED_WAVEFRONT, N.NLC_SCHED_RASTER, N.NLC_SCHED_SEQUENTIAL):
        outs = codec.decompress(data, offs, sizes, patch, N.NLC_LAYOUT_ROW, sched)
        for o, i in zip(outs, imgs):
            assert np.array_equal(o.cpu().numpy(), i), sched


def test_sheared_many_pieces_per_tile_and_decode_plan():
    # many narrow units: a CTA's share of a front spans many unit pieces, each
    # with its h halo rows, so tiles end early and shares span several tiles
    cfg = (3, 64, 2, 10)
    codec, _ = _codec(cfg, 42)
    sizes = [(96, 7)] * 12 + [(3, 40)] * 5
    imgs = images(43, sizes)
    d = [to_dev(i) for i in imgs]
    data, offs = codec.compress(d, 0, N.NLC_LAYOUT_ROW)
    for ppc in (1, 8, 128):
        N.nlc_set_tuning(codec.ctx, ppc, 0)
        outs = codec.decompress(data, offs, sizes, 0, N.NLC_LAYOUT_ROW)
        for o, i in zip(outs, imgs):
            assert np.array_equal(o.cpu().numpy(), i), ppc
    N.nlc_set_tuning(codec.ctx, 8, 0)
    plan = codec.plan(sizes, 0, N.NLC_LAYOUT_ROW)
    plan.tune(data, offs, reps=1)
    g = plan.graph(data, offs)
    g.replay()
    codec.check()
    for o, i in zip(plan.outs, imgs):
        assert np.array_equal(o.cpu().numpy(), i)
    plan.close()


def test_sheared_network_and_code_length_match_oracle():
    cfg = (3, 64, 2, 10)
    codec, w = _codec(cfg, 44)
    imgs = images(45, [(24, 40), (17, 9)])
    d = [to_dev(i) for i in imgs]
    P, bits = codec.forward(d, 0, params=True, bits=True)
    ref = np.concatenate([O.forward_image(cfg, w, im).reshape(-1, 100) for im in imgs])
    assert float(np.abs(P.cpu().numpy() - ref).max()) <= 2e-2
    ref_bits = sum(float(O.image_bits(cfg, w, im).sum()) for im in imgs)
    npx = sum(i.shape[0] * i.shape[1] for i in imgs)
    assert abs(float(bits.double().sum()) - ref_bits) / (3 * npx) <= 0.03


def test_sheared_containers_are_their_own():
    cfg = (2, 32, 1, 10)
    sh, w = _codec(cfg, 46)
    plain = CD.Codec(*cfg, N.NLC_BF16, w)
    imgs = images(47, [(20, 20)])
    d = [to_dev(i) for i in imgs]
    data, offs = sh.compress(d, 0, N.NLC_LAYOUT_ROW)
    plain.decompress(data, offs, [(20, 20)], 0, N.NLC_LAYOUT_ROW, check=False)
    assert N.nlc_sync_status(plain.ctx) == N.NLC_ERR_WEIGHTS
    assert sh.weight_hash() != plain.weight_hash()


def test_sheared_sampler_schedules_agree():
    cfg = (3, 32, 1, 10)
    codec, _ = _codec(cfg, 48)
    sizes = [(21, 33), (8, 8)]
    a = codec.sample(sizes, 0, 5, N.NLC_SCHED_WAVEFRONT)
    b = codec.sample(sizes, 0, 5, N.NLC_SCHED_RASTER)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_sheared_training_uses_the_same_weights():
    # a sheared context trains the canonical weights exactly as a BF16 one
    cfg = (3, 64, 2, 10)
    sh, w = _codec(cfg, 49)
    plain = CD.Codec(*cfg, N.NLC_BF16, w)
    batch = torch.from_numpy(synth.random_crops(3, 4, size=16, source=64)).to(DEV)
    l1, g1 = sh.loss_grad(batch)
    l2, g2 = plain.loss_grad(batch)
    assert torch.equal(g1, g2) and torch.equal(l1, l2)
