"""Parity at the sizes of the five benchmark configurations, through the C ABI.

Each configuration runs at its own size and launch configuration: round trips
are bit-exact for every pixel, and network outputs and model code lengths of
sampled pixels are compared one by one with the oracle (on the same unit
partition).  Tolerances: network outputs |d| <= 1e-4 (1 + |ref|) in FP32 and
<= 2e-2 in BF16; model code length |d bpd| <= 0.01 (FP32) / 0.03 (BF16).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_05213_gb300 import nlc as N
from paper_2201_05213_gb300 import synth

from gpu_util import DEV, ensure_built, make_codec, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _train(codec, steps, seed, batch, lr=2e-3):
    """In-run maximum-likelihood training on seeded 32x32 crops (Eq. 2)."""
    pool = torch.from_numpy(synth.random_crops(seed, 4096, size=32, source=256)).to(DEV)
    g = torch.Generator().manual_seed(seed)
    for s in range(steps):
        idx = torch.randint(0, pool.shape[0], (batch,), generator=g).to(DEV)
        codec.train_step(pool[idx].contiguous(), lr if s < steps * 3 // 4 else lr / 4,
                         want_loss=False)


def _sampled_parity(codec, cfg, imgs, dimgs, patch, n, seed, tol, bpd_tol):
    """Network outputs and code lengths of n random pixels against the oracle."""
    w = codec.get_weights().astype(np.float64)
    P, bits = codec.forward(dimgs, patch, params=True, bits=True)
    base = np.cumsum([0] + [i.shape[0] * i.shape[1] for i in imgs])
    rng = np.random.default_rng(seed)
    k_img = rng.integers(0, len(imgs), n)
    worst, gpu_bits, ref_bits = 0.0, 0.0, 0.0
    for k in np.unique(k_img):
        H, W = imgs[k].shape[:2]
        m = int((k_img == k).sum())
        ys, xs = rng.integers(0, H, m), rng.integers(0, W, m)
        ref = O.forward_pixels(cfg, w, imgs[k], ys, xs, patch)
        q = torch.from_numpy(base[k] + ys * W + xs).to(DEV)
        got = P[q].double().cpu().numpy()
        worst = max(worst, float((np.abs(got - ref) / (1.0 + np.abs(ref))).max()))
        gpu_bits += float(bits[q].double().sum())
        for j in range(m):
            r, g, b = imgs[k][ys[j], xs[j]]
            ref_bits += O.pixel_bits(cfg[3], ref[j], r, g, b)
    assert worst <= tol, worst
    assert abs(gpu_bits - ref_bits) / (3 * n) <= bpd_tol, (gpu_bits / (3 * n), ref_bits / (3 * n))


def _unit_bpd_parity(codec, cfg, imgs, dimgs, patch, units, bpd_tol):
    """Model code length of whole coding units (every pixel of each) against
    the oracle's, which runs one spawned process per host core."""
    w = codec.get_weights().astype(np.float64)
    _, bits = codec.forward(dimgs, patch, params=False, bits=True)
    base = np.cumsum([0] + [i.shape[0] * i.shape[1] for i in imgs])
    b = bits.double().cpu().numpy()
    gpu, npx = 0.0, 0
    for k, y0, x0, hu, wu in units:
        W = imgs[k].shape[1]
        rows = base[k] + (y0 + np.arange(hu))[:, None] * W + x0 + np.arange(wu)[None, :]
        gpu += float(b[rows].sum())
        npx += hu * wu
    ref, n_ref = O.batch_bits_parallel(cfg, w, imgs, patch, units=units)
    assert n_ref == npx
    d = abs(gpu - ref) / (3 * npx)
    assert d <= bpd_tol, (gpu / (3 * npx), ref / (3 * npx))
    return gpu / (3 * npx), ref / (3 * npx)


def _round_trip(codec, imgs, dimgs, patch, layout, schedules):
    data, offs = codec.compress(dimgs, patch, layout)
    sizes = [i.shape[:2] for i in imgs]
    for sched in schedules:
        outs = codec.decompress(data, offs, sizes, patch, layout, sched)
        for o, i in zip(outs, imgs):
            assert np.array_equal(o.cpu().numpy(), i), sched
    return data, offs


def test_cfg0_tiny_sequential_single_stream():
    # one 32x32 image (seed 0), h=3 C=32 R=2 K=10, FP32 Xavier weights (seed 0),
    # one raster stream; the GPU decodes the oracle's pixels and the oracle's
    # own raster codec round-trips
    cfg = (3, 32, 2, 10)
    codec, w = make_codec(cfg, N.NLC_FP32, seed=0)
    img = synth.make_batch(0, [(32, 32)])[0]
    d = [to_dev(img)]
    _round_trip(codec, [img], d, 0, N.NLC_LAYOUT_UNIT,
                [N.NLC_SCHED_SEQUENTIAL, N.NLC_SCHED_RASTER])
    words, lens, _, _ = O.encode_image(cfg, w, img, 0, 0)
    dec, ok = O.decode_image(cfg, w, words, lens, 32, 32, 0, 0)
    assert ok and np.array_equal(dec, img)
    _sampled_parity(codec, cfg, [img], d, 0, 128, 0, 1e-4, 0.01)


def test_cfg1_wavefront_fp32_trained():
    # 64 images of 64x64 (seed 1), h=3 C=64 R=2 K=10, FP32, trained 2000 steps
    # of batch 64 on 32x32 crops; wavefront and sequential decode of the same
    # per-row containers give the input
    cfg = (3, 64, 2, 10)
    codec, _ = make_codec(cfg, N.NLC_FP32, seed=0)
    _train(codec, 2000, seed=1, batch=64)
    imgs = synth.make_batch(1, [(64, 64)] * 64)
    d = [to_dev(i) for i in imgs]
    _round_trip(codec, imgs, d, 0, N.NLC_LAYOUT_ROW,
                [N.NLC_SCHED_WAVEFRONT, N.NLC_SCHED_SEQUENTIAL])
    _sampled_parity(codec, cfg, imgs, d, 0, 256, 1, 1e-4, 0.01)


@pytest.mark.parametrize("h", [1, 2, 3])
def test_cfg2_training_batch(h):
    # batch 128 of 32x32 crops (seed 2), C=64 K=10, BF16 forward and adjoint
    # on the tensor cores with FP32 accumulation: the loss of the whole batch
    # within the BF16 code-length tolerance (0.03 bpd) of the oracle's, the
    # gradient of the whole batch within the BF16 tolerance of
    # test_gpu_train.py (relative L2 error <= 3e-2, every element within 5e-2
    # of the largest); the FP32 context's adjoint on the same batch matches
    # the oracle to 1e-4 of the largest element
    cfg = (h, 64, 2, 10)
    codec, w = make_codec(cfg, N.NLC_BF16, seed=0)
    w64 = w.astype(np.float64)
    batch = synth.random_crops(2, 128, size=32, source=256)
    loss, grad = codec.loss_grad(to_dev(batch))
    ref_loss, ref_grad = O.nll_grad(cfg, w64, batch)
    assert abs(float(loss[0]) - ref_loss) <= 0.03, (float(loss[0]), ref_loss)
    g = grad.double().cpu().numpy()
    rel = np.linalg.norm(g - ref_grad) / np.linalg.norm(ref_grad)
    worst = np.abs(g - ref_grad).max() / np.abs(ref_grad).max()
    assert rel <= 3e-2 and worst <= 5e-2, (rel, worst)
    f32, _ = make_codec(cfg, N.NLC_FP32, seed=0)
    loss32, grad32 = f32.loss_grad(to_dev(batch))
    assert abs(float(loss32[0]) - ref_loss) <= 1e-5 * ref_loss
    g32 = grad32.double().cpu().numpy()
    assert np.abs(g32 - ref_grad).max() <= 1e-4 * np.abs(ref_grad).max()


def test_cfg3_uneven_batch_bf16():
    # 256 images, sides uniform in {32, 48, ..., 512} (seed 3), h=3 C=64 BF16,
    # whole images as units, one stream per row, one persistent launch
    cfg = (3, 64, 2, 10)
    codec, _ = make_codec(cfg, N.NLC_BF16, seed=0)
    sizes = synth.uneven_sizes(3, 256)
    imgs = synth.make_batch(3, sizes)
    d = [to_dev(i) for i in imgs]
    _round_trip(codec, imgs, d, 0, N.NLC_LAYOUT_ROW, [N.NLC_SCHED_WAVEFRONT])
    _sampled_parity(codec, cfg, imgs, d, 0, 256, 3, 2e-2, 0.03)
    # every pixel of 32 whole images (every 8th of the batch)
    units = [(k, 0, 0, sizes[k][0], sizes[k][1]) for k in range(0, 256, 8)]
    _unit_bpd_parity(codec, cfg, imgs, d, 0, units, 0.03)


@pytest.mark.parametrize("h", [1, 2, 3])
def test_cfg4_large_images_patches_bf16(h):
    # 1x2048^2 + 8x1024^2 (seed 4, 64 polygons), 256^2 patches decoded in
    # parallel with a wavefront inside each, C=64 BF16
    cfg = (h, 64, 2, 10)
    codec, _ = make_codec(cfg, N.NLC_BF16, seed=0)
    imgs = synth.make_batch(4, [(2048, 2048)] + [(1024, 1024)] * 8, n_poly=64)
    d = [to_dev(i) for i in imgs]
    _round_trip(codec, imgs, d, 256, N.NLC_LAYOUT_ROW, [N.NLC_SCHED_WAVEFRONT])
    _sampled_parity(codec, cfg, imgs, d, 256, 192, 4, 2e-2, 0.03)
    # model code length over whole 256^2 patches: every patch of every image
    # at h = 3 (12.6 M pixels), one patch per image (a different one each) else
    if h == 3:
        units = None
    else:
        units = [(k, 256 * ((k + h) % (im.shape[0] // 256)), 256 * ((3 * k) % (im.shape[1] // 256)),
                  256, 256) for k, im in enumerate(imgs)]
    if units is None:
        units = [(k, y, x, 256, 256) for k, im in enumerate(imgs)
                 for y in range(0, im.shape[0], 256) for x in range(0, im.shape[1], 256)]
    _unit_bpd_parity(codec, cfg, imgs, d, 256, units, 0.03)
