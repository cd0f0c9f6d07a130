"""Pins of the FP64 oracle's model, mixture, quantiser, coder and gradient.

Each check ties the oracle to something other than itself: a library routine
(a masked torch conv2d for the local first layer of Section 2.1), closed
forms evaluated in 50-digit arithmetic, normalisation and chain-rule
identities, brute force on tiny inputs, the round-trip identity of the stream
coder (Section 2) and central finite differences of the objective (Eq. 2).
"""
import mpmath
import numpy as np
import pytest
import torch

import oracle as O
from oracle import schedule as S
from paper_2201_05213_gb300 import synth

mpmath.mp.dps = 50


def _split(w, h, C, R, K):
    out, o = {}, 0
    for name, shp in synth.weight_shapes(h, C, R, K):
        n = int(np.prod(shp))
        out[name] = torch.tensor(np.asarray(w[o:o + n], dtype=np.float64).reshape(shp))
        o += n
    assert o == len(w)
    return out


def _torch_forward(w, img, h, C, R, K):
    """The local PixelCNN as a (2h+1)^2 type-A masked conv + 1x1 layers, in torch FP64."""
    t = _split(w, h, C, R, K)
    k = 2 * h + 1
    W0 = t["W0"].reshape(C, 2 * h * (h + 1), 3)  # [C][p][ch], p = unmasked tap in raster order
    conv = torch.zeros(C, 3, k * k, dtype=torch.float64)
    conv[:, :, : 2 * h * (h + 1)] = W0.permute(0, 2, 1)
    conv = conv.reshape(C, 3, k, k)
    mask = torch.zeros(k, k, dtype=torch.float64)
    mask[:h, :] = 1
    mask[h, :h] = 1
    assert (conv * (1 - mask)).abs().sum() == 0
    x = torch.tensor(img, dtype=torch.float64).permute(2, 0, 1)[None]
    x = (2 * x - 255) / 255
    a = torch.nn.functional.conv2d(x, conv * mask, t["b0"], padding=h)[0]  # C,H,W
    a = a.permute(1, 2, 0)
    elu = torch.nn.functional.elu
    for r in range(R):
        hid = elu(a) @ t[f"W1_{r}"].T + t[f"b1_{r}"]
        a = a + elu(hid) @ t[f"W2_{r}"].T + t[f"b2_{r}"]
    return (elu(a) @ t["WH"].T + t["bH"]).numpy()


@pytest.mark.parametrize("h,C,R,K", [(1, 8, 1, 2), (2, 6, 0, 3), (3, 8, 2, 10)])
def test_forward_matches_masked_conv(h, C, R, K):
    w = synth.xavier_weights(h, C, R, K, seed=h) * 2.0
    w[:] += np.random.default_rng(h).normal(0, 0.1, len(w)).astype(np.float32)  # nonzero biases
    img = synth.make_image(5, 11, 13)
    got = O.forward_image((h, C, R, K), w, img)
    ref = _torch_forward(w, img, h, C, R, K)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_forward_is_local_and_patch_bounded():
    h, C, R, K = 2, 6, 1, 2
    w = synth.xavier_weights(h, C, R, K, seed=4) * 2
    img = synth.make_image(6, 12, 12)
    base = O.forward_image((h, C, R, K), w, img)
    i, j = 6, 6
    ctx = {(i + dy, j + dx) for dy, dx in S.context_offsets(h)}
    for y in range(12):
        for x in range(12):
            im2 = img.copy()
            im2[y, x] = 255 - im2[y, x]
            out = O.forward_pixels((h, C, R, K), w, im2, [i], [j])[0]
            changed = np.abs(out - base[i, j]).max() > 0
            assert changed == ((y, x) in ctx), (y, x)
    # a patch partition equals running each patch as its own image
    P = 5
    full = O.forward_image((h, C, R, K), w, img, patch=P)
    for y0, x0, Hu, Wu in S.patch_units(12, 12, P):
        sub = O.forward_image((h, C, R, K), w, np.ascontiguousarray(img[y0:y0 + Hu, x0:x0 + Wu]))
        np.testing.assert_array_equal(full[y0:y0 + Hu, x0:x0 + Wu], sub)


def _mp_logistic_mass(m, ls, v):
    """Bin mass of a logistic in 50-digit arithmetic; the upper tail is taken as a
    difference of survival functions so that tiny masses keep their digits."""
    s = mpmath.e ** mpmath.mpf(ls)
    m = mpmath.mpf(m)
    cdf = lambda e: 1 / (1 + mpmath.e ** (-(e - m) / s))
    sf = lambda e: 1 / (1 + mpmath.e ** ((e - m) / s))
    lo = None if v == 0 else mpmath.mpf(2 * v - 256) / 255
    hi = None if v == 255 else mpmath.mpf(2 * v - 254) / 255
    centre = mpmath.mpf(2 * v - 255) / 255
    if centre <= m:
        return (1 if hi is None else cdf(hi)) - (0 if lo is None else cdf(lo))
    return (1 if lo is None else sf(lo)) - (0 if hi is None else sf(hi))


@pytest.mark.parametrize("m,ls", [(0.0, 0.0), (0.3, -3.0), (-0.9, -7.0), (0.99, -5.5),
                                  (-1.5, -2.0), (2.0, 1.0), (0.5, -6.9)])
def test_log_bin_mass_against_50_digit_closed_form(m, ls):
    tot = 0.0
    for v in range(256):
        got = O.log_bin_mass(m, ls, v)
        ref = _mp_logistic_mass(m, ls, v)
        tot += np.exp(got)
        if ref > mpmath.mpf(10) ** -300:
            assert abs(got - float(mpmath.log(ref))) <= 1e-9 * max(1.0, abs(float(mpmath.log(ref))))
    assert abs(tot - 1.0) < 1e-12


def _rand_params(K, rng, scale=1.0):
    p = rng.normal(0, scale, 10 * K)
    p[4 * K:7 * K] = rng.uniform(-6, 0, 3 * K)
    p[K:4 * K] = rng.uniform(-1, 1, 3 * K)
    return p


def test_single_component_uncoupled_is_logistic():
    K = 1
    p = np.zeros(10)
    p[1:4] = [0.2, -0.4, 0.7]  # mu_R, mu_G, mu_B
    p[4:7] = [-3.0, -2.5, -4.0]  # log-scales
    for ch in range(3):
        for v in (0, 3, 100, 127, 200, 255):
            got = O.channel_prob(K, p, ch, 17, 230, v)
            ref = float(_mp_logistic_mass(p[1 + ch], p[4 + ch], v))
            assert abs(got - ref) <= 1e-12 + 1e-10 * ref


@pytest.mark.parametrize("seed", range(4))
def test_chain_rule_equals_joint_mixture(seed):
    K = 10
    rng = np.random.default_rng(seed)
    p = _rand_params(K, rng)
    for r, g, b in [(0, 0, 0), (255, 255, 255), (17, 200, 91), tuple(rng.integers(0, 256, 3))]:
        pr = O.channel_prob(K, p, 0, r, g, r)
        pg = O.channel_prob(K, p, 1, r, g, g)
        pb = O.channel_prob(K, p, 2, r, g, b)
        bits = -np.log2(pr * pg * pb)
        assert abs(bits - O.pixel_bits(K, p, r, g, b)) < 1e-9
    # each coding distribution is normalised
    r, g = 40, 60
    for ch in range(3):
        assert abs(sum(O.channel_prob(K, p, ch, r, g, v) for v in range(256)) - 1) < 1e-12


def test_joint_mixture_normalised_brute_force():
    # sum over all 256^3 pixel values of the joint, for a 2-component pixel
    K = 2
    rng = np.random.default_rng(9)
    p = _rand_params(K, rng)
    tot = 0.0
    for r in range(256):
        pr = O.channel_prob(K, p, 0, r, 0, r)
        if pr < 1e-30:
            continue
        for g in range(256):
            pg = O.channel_prob(K, p, 1, r, g, g)
            if pr * pg < 1e-30:
                continue
            tot += pr * pg  # sum_b p(b|r,g) = 1 (checked above)
    assert abs(tot - 1) < 1e-10


def _check_table(cum):
    cum = np.asarray(cum, dtype=np.int64)
    assert cum[0] == 0 and cum[256] == 65536
    freq = np.diff(cum)
    assert (freq >= 1).all()
    assert freq.sum() == 65536


def test_quantiser_closed_forms():
    b = np.arange(257)
    cum = O.quantise_cdf(b / 256.0)
    np.testing.assert_array_equal(np.diff(cum.astype(np.int64)), np.full(256, 256))
    for v in (0, 1, 128, 254, 255):
        F = (b > v).astype(np.float64)
        freq = np.diff(O.quantise_cdf(F).astype(np.int64))
        assert freq[v] == 65281 and (np.delete(freq, v) == 1).all()
    # round half to even: 65280 * F = 0.5 and 1.5 at b = 1, 2
    F = np.zeros(257)
    F[1], F[2], F[3:] = 0.5 / 65280, 1.5 / 65280, 1.0
    F[256] = 1
    cum = O.quantise_cdf(F)
    assert cum[1] == 0 + 1 and cum[2] == 2 + 2


@pytest.mark.parametrize("seed", range(6))
def test_quantiser_invariants_adversarial(seed):
    rng = np.random.default_rng(seed)
    F = np.sort(rng.uniform(0, 1, 257))
    F[0], F[256] = 0, 1
    _check_table(O.quantise_cdf(F))
    G = F + rng.normal(0, 0.01, 257)  # non-monotone, outside [0, 1]
    G[0], G[256] = 0, 1
    _check_table(O.quantise_cdf(G))
    _check_table(O.quantise_cdf(np.zeros(257)))
    _check_table(O.quantise_cdf(np.ones(257)))


@pytest.mark.parametrize("seed", range(3))
def test_pixel_tables_follow_the_model(seed):
    K = 10
    rng = np.random.default_rng(100 + seed)
    p = _rand_params(K, rng)
    r, g = (int(v) for v in rng.integers(0, 256, 2))
    cum = O.pixel_tables(K, p, r, g)
    for ch in range(3):
        _check_table(cum[ch])
        freq = np.diff(cum[ch].astype(np.int64))
        P = np.array([O.channel_prob(K, p, ch, r, g, v) for v in range(256)])
        # q_b within 1/2 of 65280 F(b) before the running max; F is monotone, so
        # |freq_v - 65280 P(v) - 1| <= 1
        assert np.abs(freq - 65280 * P - 1).max() <= 1.0 + 1e-6


def _rand_table(rng, conc):
    p = rng.dirichlet(np.full(256, conc))
    F = np.concatenate([[0], np.cumsum(p)])
    F[256] = 1
    return O.quantise_cdf(F)


@pytest.mark.parametrize("n,conc", [(0, 1.0), (1, 1.0), (7, 0.05), (3000, 0.05), (3000, 5.0)])
def test_rans_round_trip_and_length(n, conc):
    rng = np.random.default_rng(n)
    tabs = np.stack([_rand_table(rng, conc) for _ in range(max(n, 1))])[:n].reshape(n, 257)
    sym = np.array([rng.choice(256, p=np.diff(t.astype(np.int64)) / 65536) for t in tabs], dtype=np.int64)
    start = tabs[np.arange(n), sym] if n else np.zeros(0, np.uint32)
    freq = (tabs[np.arange(n), sym + 1] - start) if n else np.zeros(0, np.uint32)
    stream = O.rans_encode(start, freq)
    dec, ok = O.rans_decode(stream, tabs)
    assert ok
    np.testing.assert_array_equal(dec, sym)
    ideal = float(np.sum(-np.log2(freq / 65536.0)))
    assert 8 * len(stream) <= ideal + 32 + 1.0
    # a truncated or extended stream is detected
    if n:
        _, ok2 = O.rans_decode(stream[:-1], tabs)
        _, ok3 = O.rans_decode(np.concatenate([stream, [7]]).astype(np.uint8), tabs)
        assert not ok2 and not ok3


def test_rans_brute_force_tiny_alphabet():
    # all symbol sequences of length 4 over a 3-symbol distribution
    F = np.ones(257)
    F[0] = 0
    F[1], F[2] = 0.2, 0.7
    tab = O.quantise_cdf(F)
    import itertools
    for seq in itertools.product(range(3), repeat=4):
        seq = np.array(seq)
        start = tab[seq]
        freq = tab[seq + 1] - start
        stream = O.rans_encode(start, freq)
        dec, ok = O.rans_decode(stream, np.tile(tab, (4, 1)))
        assert ok and (dec == seq).all()


@pytest.mark.parametrize("patch,layout", [(0, 0), (0, 1), (8, 1), (12, 0)])
def test_raster_codec_round_trip(patch, layout):
    cfg = (3, 8, 1, 4)
    w = synth.xavier_weights(*cfg, seed=0)
    img = synth.make_image(0, 20, 18)
    words, lens, bm, bq = O.encode_image(cfg, w, img, patch, layout)
    dec, ok = O.decode_image(cfg, w, words, lens, 20, 18, patch, layout)
    assert ok and (dec == img).all()
    assert len(lens) == O.num_streams(20, 18, patch, layout)
    # bytes within 32 bits per stream of the quantised-ideal code length
    assert 8 * len(words) <= bq + 32 * len(lens) + 1
    # corrupting one byte is detected or changes the image
    bad = words.copy()
    bad[len(bad) // 2] ^= 0x5A
    dec2, ok2 = O.decode_image(cfg, w, bad, lens, 20, 18, patch, layout)
    assert (not ok2) or (dec2 != img).any()


@pytest.mark.parametrize("cfg", [(1, 4, 1, 2), (2, 5, 1, 3), (3, 4, 2, 2)])
def test_gradient_central_differences(cfg):
    w = synth.xavier_weights(*cfg, seed=1).astype(np.float64) * 3
    w += np.random.default_rng(2).normal(0, 0.05, len(w))
    imgs = synth.random_crops(2, 2, size=6, source=32)
    v, g = O.nll_grad(cfg, w, imgs)
    assert abs(v - O.nll_grad(cfg, w, imgs, grad=False)) == 0
    # the objective equals the mean model code length of the pixels
    tot = 0.0
    for n in range(imgs.shape[0]):
        outs = O.forward_image(cfg, w, imgs[n])
        for i in range(6):
            for j in range(6):
                tot += O.pixel_bits(cfg[3], outs[i, j], *imgs[n, i, j])
    assert abs(v - tot / (3 * imgs.shape[0] * 36)) < 1e-12
    rng = np.random.default_rng(0)
    idx = rng.choice(len(w), 16, replace=False)
    for k in idx:
        # O(e^2) truncation; the objective has large third derivatives where a
        # component is very sharp, hence the small step
        e = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[k] += e
        wm[k] -= e
        fd = (O.nll_grad(cfg, wp, imgs, False) - O.nll_grad(cfg, wm, imgs, False)) / (2 * e)
        assert abs(fd - g[k]) <= 1e-5 * max(1.0, abs(fd)) + 1e-7, (k, fd, g[k])


def test_tiny_workload_oracle_round_trip():
    # one 32x32 image, h=3, C=32, 2 residual blocks, K=10, Xavier weights from
    # seed 0, one raster-order stream
    cfg = (3, 32, 2, 10)
    w = synth.xavier_weights(*cfg, seed=0)
    img = synth.make_image(0, 32, 32, 4)
    words, lens, bm, bq = O.encode_image(cfg, w, img, 0, 0)
    assert len(lens) == 1
    dec, ok = O.decode_image(cfg, w, words, lens, 32, 32, 0, 0)
    assert ok and (dec == img).all()
    assert 8 * len(words) <= bq + 32 + 1


def _mp_scaled(v):
    return mpmath.mpf(2 * v - 255) / 255


@pytest.mark.parametrize("raw", [(0.8, -1.3, 0.45), (-2.0, 0.6, -0.9), (3.0, 3.0, -3.0)])
def test_single_component_coupled_means_closed_form(raw):
    # K = 1, nonzero coupling: the G location is mu_G + tanh(a) x_R and the B
    # location mu_B + tanh(b) x_R + tanh(c) x_G, x = (2v - 255)/255; each
    # channel's coding distribution is then the plain logistic bin mass there.
    K = 1
    p = np.zeros(10)
    p[1:4] = [0.15, -0.35, 0.6]
    p[4:7] = [-3.2, -2.7, -3.9]
    p[7:10] = raw
    a, b, c = (mpmath.tanh(mpmath.mpf(x)) for x in raw)
    for r, g in [(17, 230), (255, 0), (128, 64), (0, 255)]:
        xr, xg = _mp_scaled(r), _mp_scaled(g)
        loc = [mpmath.mpf(p[1]), p[2] + a * xr, p[3] + b * xr + c * xg]
        for ch in range(3):
            for v in (0, 5, 60, 127, 128, 190, 255):
                got = O.channel_prob(K, p, ch, r, g, v)
                ref = float(_mp_logistic_mass(loc[ch], p[4 + ch], v))
                assert abs(got - ref) <= 1e-13 + 1e-10 * ref, (r, g, ch, v, got, ref)


def _mp_joint(p, K, r, g, b):
    """p(r, g, b) of the joint mixture written out in 50-digit arithmetic:
    sum_k softmax(logits)_k * L(r; mu_R) * L(g; mu_G + tanh(a_k) x_r)
    * L(b; mu_B + tanh(b_k) x_r + tanh(c_k) x_g), L the logistic bin mass with
    log-scale max(ls, -7)."""
    logits = [mpmath.mpf(p[k]) for k in range(K)]
    z = sum(mpmath.e ** l for l in logits)
    xr, xg = _mp_scaled(r), _mp_scaled(g)
    tot = mpmath.mpf(0)
    for k in range(K):
        mu = [mpmath.mpf(p[K + c * K + k]) for c in range(3)]
        ls = [max(float(p[4 * K + c * K + k]), -7.0) for c in range(3)]
        t = [mpmath.tanh(mpmath.mpf(p[7 * K + c * K + k])) for c in range(3)]
        pr = _mp_logistic_mass(mu[0], ls[0], r)
        pg = _mp_logistic_mass(mu[1] + t[0] * xr, ls[1], g)
        pb = _mp_logistic_mass(mu[2] + t[1] * xr + t[2] * xg, ls[2], b)
        tot += mpmath.e ** logits[k] / z * pr * pg * pb
    return tot


@pytest.mark.parametrize("seed", range(3))
def test_three_component_coupled_mixture_against_50_digit_joint(seed):
    K = 3
    rng = np.random.default_rng(200 + seed)
    p = _rand_params(K, rng)
    p[4 * K:7 * K] = rng.uniform(-4, -1, 3 * K)
    p[7 * K:] = rng.uniform(-2, 2, 3 * K)  # strong coupling of every component
    p[4 * K] = -7.5  # one log-scale below the clamp
    for r, g, b in [(40, 200, 90), (255, 0, 128), (0, 0, 0), tuple(int(v) for v in rng.integers(0, 256, 3))]:
        ref = _mp_joint(p, K, r, g, b)
        if ref < mpmath.mpf(10) ** -250:
            continue
        ref_bits = float(-mpmath.log(ref, 2))
        assert abs(O.pixel_bits(K, p, r, g, b) - ref_bits) <= 1e-9 * max(1.0, ref_bits)
        # chain rule: the channel coding distributions multiply to the joint
        pr = _mp_joint_marg(p, K, r)
        pg = _mp_joint_marg(p, K, r, g) / pr
        assert abs(O.channel_prob(K, p, 0, r, g, r) - float(pr)) <= 1e-12 + 1e-9 * float(pr)
        assert abs(O.channel_prob(K, p, 1, r, g, g) - float(pg)) <= 1e-12 + 1e-9 * float(pg)
        pb = ref / (pr * pg)
        assert abs(O.channel_prob(K, p, 2, r, g, b) - float(pb)) <= 1e-12 + 1e-9 * float(pb)


def _mp_joint_marg(p, K, r, g=None):
    """Marginal p(r), or p(r, g), of the joint mixture (the later channels'
    bin masses sum to one), in 50-digit arithmetic."""
    logits = [mpmath.mpf(p[k]) for k in range(K)]
    z = sum(mpmath.e ** l for l in logits)
    xr = _mp_scaled(r)
    tot = mpmath.mpf(0)
    for k in range(K):
        term = mpmath.e ** logits[k] / z
        term *= _mp_logistic_mass(mpmath.mpf(p[K + k]), max(float(p[4 * K + k]), -7.0), r)
        if g is not None:
            m_g = mpmath.mpf(p[2 * K + k]) + mpmath.tanh(mpmath.mpf(p[7 * K + k])) * xr
            term *= _mp_logistic_mass(m_g, max(float(p[5 * K + k]), -7.0), g)
        tot += term
    return tot


def test_image_bits_is_forward_then_pixel_bits():
    cfg = (2, 8, 1, 3)
    w = synth.xavier_weights(*cfg, seed=7) * 2
    img = synth.make_image(8, 13, 11)
    for patch in (0, 5):
        outs = O.forward_image(cfg, w, img, patch=patch)
        ref = np.array([[O.pixel_bits(cfg[3], outs[i, j], *img[i, j]) for j in range(11)]
                        for i in range(13)])
        np.testing.assert_array_equal(O.image_bits(cfg, w, img, patch), ref)
    # the unit-parallel total over spawned processes equals the serial sum
    tot, n = O.batch_bits_parallel(cfg, w, [img, img[:7]], 5, n_proc=2)
    assert n == 13 * 11 + 7 * 11
    ser = O.image_bits(cfg, w, img, 5).sum() + O.image_bits(cfg, w, img[:7], 5).sum()
    assert abs(tot - ser) <= 1e-9 * ser
