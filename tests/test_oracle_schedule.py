"""Pins of the schedule and shear definitions to the paper's worked examples.

Section 3 (Fig. 3, the step-count law), Section 3.1 (Fig. 4, Fig. 5) and a
brute-force dependency check of Eq. 3 on small units.
"""
import os

import numpy as np
import pytest

from oracle import schedule as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_matrix(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def _read_blocks(name):
    blocks, cur = {}, None
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("=="):
            cur = line[2:].strip()
            blocks[cur] = []
        else:
            blocks[cur].append(line.split())
    return blocks


def test_fig3_schedule_matrix():
    gold = np.array(_read_matrix("fig3_schedule_5x5_h1.txt"), dtype=int)
    assert (S.schedule_matrix(5, 5, 1) + 1 == gold).all()


def test_fig3_step_counts():
    # 5x5, h=1: T = 13 wavefront steps versus 25 sequential ones.
    assert S.num_steps(5, 5, 1) == 13
    assert 5 * 5 == 25
    # parallel units floor((D+h)/(h+1)) = 3 for this example
    assert S.max_parallel(5, 1) == 3


@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_step_count_law_square(h):
    for D in range(1, 14):
        steps = S.schedule_matrix(D, D, h)
        T = int(steps.max()) + 1
        assert T == D + (D - 1) * (h + 1) == S.num_steps(D, D, h)
        fronts = [len(S.front(t, D, D, h)) for t in range(T)]
        assert sum(fronts) == D * D
        # a unit narrower than h+1 has idle steps between its rows
        assert (min(fronts) >= 1) == (D >= h + 1 or D == 1)
        assert max(fronts) == S.max_parallel(D, h) == -(-D // (h + 1))


@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_step_count_rectangular(h):
    for H in range(1, 10):
        for W in range(1, 10):
            T = int(S.schedule_matrix(H, W, h).max()) + 1
            assert T == W + (H - 1) * (h + 1)
            fronts = [len(S.front(t, H, W, h)) for t in range(T)]
            assert max(fronts) == min(H, -(-W // (h + 1)))


@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_wavefront_respects_dependencies(h):
    for H in range(1, 13, 3):
        for W in range(1, 13, 2):
            assert S.check_schedule(H, W, h, S.schedule_matrix(H, W, h)) == 0
            raster = [[S.raster_step(i, j, W) for j in range(W)] for i in range(H)]
            assert S.check_schedule(H, W, h, raster) == 0


@pytest.mark.parametrize("h", [1, 2, 3])
def test_offset_h_plus_1_is_minimal(h):
    # t = j + o*i is a valid order only for o >= h+1 (Section 3.1: o = h+1).
    H = W = 12
    for o in range(0, h + 1):
        steps = [[j + o * i for j in range(W)] for i in range(H)]
        assert S.check_schedule(H, W, h, steps) > 0
    steps = [[j + (h + 1) * i for j in range(W)] for i in range(H)]
    assert S.check_schedule(H, W, h, steps) == 0


def test_patch_units_partition_image():
    for H, W, P in [(9, 7, 4), (16, 16, 8), (5, 13, 5), (3, 3, 8)]:
        cover = np.zeros((H, W), dtype=int)
        for y0, x0, Hu, Wu in S.patch_units(H, W, P):
            assert 1 <= Hu <= P and 1 <= Wu <= P
            cover[y0:y0 + Hu, x0:x0 + Wu] += 1
        assert (cover == 1).all()


@pytest.mark.parametrize("h,P", [(1, 4), (2, 5), (3, 8)])
def test_patch_schedule_dependencies(h, P):
    # Inside every unit the wavefront is valid and uses T_u = Wu + (Hu-1)(h+1) steps.
    for y0, x0, Hu, Wu in S.patch_units(11, 13, P):
        m = S.schedule_matrix(Hu, Wu, h)
        assert S.check_schedule(Hu, Wu, h, m) == 0
        assert int(m.max()) + 1 == S.num_steps(Hu, Wu, h)


def test_fig4_sheared_image():
    gold = _read_matrix("fig4_sheared_5x5_o2.txt")
    labels = np.array([[10 * (i + 1) + (j + 1) for j in range(5)] for i in range(5)])
    sheared = S.shear(labels, 2)
    assert sheared.shape == (5, 13)
    assert (sheared == np.array(gold, dtype=int)).all()
    assert (S.unshear(sheared, 2, 5) == labels).all()
    # the front at 0-indexed step t is sheared column t
    for t in range(13):
        col = {(i, j) for i in range(5) for j in range(5) if sheared[i, t] == labels[i, j] and sheared[i, t]}
        assert col == set(S.front(t, 5, 5, 1))


def test_fig5_sheared_kernels():
    b = _read_blocks("fig5_sheared_kernels.txt")
    for h in (1, 2):
        nel = b[f"nelloc_h{h}"]
        rows = [[v for v in r if v != "0"] for r in nel]
        rows = [r for r in rows if r]
        sk = S.sheared_kernel(rows, h)
        got = [[str(v) for v in r] for r in sk]
        assert got == b[f"shearloc_h{h}"]


@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_sheared_window_covers_context(h):
    # every context pixel of (i, j) lies in the h(h+2) sheared columns before t
    o = h + 1
    for dy, dx in S.context_offsets(h):
        dt = dx + o * dy
        assert -h * (h + 2) <= dt <= -1
    assert min(dx + o * dy for dy, dx in S.context_offsets(h)) == -h * (h + 2)


@pytest.mark.parametrize("h", [1, 2, 3])
def test_sheared_first_layer_equals_masked_layer(h):
    # Section 3.1: on the sheared image (row i moved right by (h+1) i), the
    # first layer is a plain correlation of Fig. 5's sheared kernels with the
    # h+1 rows of the h(h+2) sheared columns before the pixel's own; in FP64
    # it equals the masked layer on the context of Eq. 3 (zero padding).
    rng = np.random.default_rng(h)
    C, H, W = 3, 7, 9
    ntap = 2 * h * (h + 1)
    W0 = rng.normal(0, 1, (C, 3 * ntap))
    img = rng.integers(0, 256, (H, W, 3))
    x = (2.0 * img - 255.0) / 255.0
    o = h + 1
    Sx = S.shear(x, o)
    Ws = h * (h + 2)
    offs = S.context_offsets(h)
    for oc in range(C):
        # per input channel: the unmasked kernel rows, top first
        kern = []
        for c in range(3):
            rows, p = [], 0
            for dy in range(-h, 1):
                n = 2 * h + 1 if dy < 0 else h
                rows.append([W0[oc, 3 * (p + k) + c] for k in range(n)])
                p += n
            kern.append(np.array(S.sheared_kernel(rows, h), dtype=np.float64))
        for i in range(H):
            for j in range(W):
                ref = 0.0
                for p, (dy, dx) in enumerate(offs):
                    ii, jj = i + dy, j + dx
                    if 0 <= ii < H and 0 <= jj < W:
                        ref += float(np.dot(W0[oc, 3 * p:3 * p + 3], x[ii, jj]))
                t = j + o * i
                got = 0.0
                for dd in range(h + 1):
                    r = i - h + dd
                    if r < 0:
                        continue
                    for q in range(Ws):
                        col = t - Ws + q
                        if col < 0:
                            continue
                        for c in range(3):
                            got += kern[c][dd][q] * Sx[r, col, c]
                assert abs(got - ref) < 1e-12, (oc, i, j)
