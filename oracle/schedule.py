"""Decode schedules and the sheared layout, written out plainly (test infrastructure).

Section 3 / Fig. 3: with horizon h, pixel (i, j) (0-indexed here, 1-indexed in
the paper) can be decoded at step t = j + (h+1) i, so a H x W unit takes
T = W + (H-1)(h+1) steps; for a D x D image that is D + (D-1)(h+1) (P. 219's
step-count law) on floor((D+h)/(h+1)) parallel units.

Section 3.1 / Fig. 4: shearing row i right by o = h+1 puts the whole step-t
front in sheared column t (width L = W + (H-1) o).  Fig. 5: only the first
kernel changes; its window is the h(h+2) sheared columns before column t.
"""
from __future__ import annotations

import numpy as np


def context_offsets(h):
    """(dy, dx) of the causal context of Eq. 3, in the order of the feature vector."""
    offs = [(dy, dx) for dy in range(-h, 0) for dx in range(-h, h + 1)]
    offs += [(0, dx) for dx in range(-h, 0)]
    return offs


def step_index(i, j, h):
    """Wavefront step of pixel (i, j), 0-indexed (Fig. 3 shows this + 1)."""
    return j + (h + 1) * i


def raster_step(i, j, W):
    """Sequential (raster) step of pixel (i, j)."""
    return i * W + j


def num_steps(H, W, h):
    """T = W + (H-1)(h+1)."""
    return W + (H - 1) * (h + 1)


def max_parallel(D, h):
    """Parallel units needed for a D x D image: floor((D+h)/(h+1))."""
    return (D + h) // (h + 1)


def front(t, H, W, h):
    """Pixels decoded at step t, by direct enumeration of the unit."""
    return [(i, j) for i in range(H) for j in range(W) if step_index(i, j, h) == t]


def schedule_matrix(H, W, h):
    return np.array([[step_index(i, j, h) for j in range(W)] for i in range(H)], dtype=np.int64)


def check_schedule(H, W, h, steps):
    """Brute-force validity of a schedule steps[i][j] for the local model of Eq. 3.

    Every in-unit context pixel of every pixel must carry a strictly smaller step.
    Returns the number of violations.
    """
    bad = 0
    for i in range(H):
        for j in range(W):
            for dy, dx in context_offsets(h):
                ii, jj = i + dy, j + dx
                if 0 <= ii < H and 0 <= jj < W and not steps[ii][jj] < steps[i][j]:
                    bad += 1
    return bad


def patch_units(H, W, P):
    """(y0, x0, Hu, Wu) of the P x P coding units in raster order (ragged edges)."""
    if P <= 0:
        return [(0, 0, H, W)]
    return [(y, x, min(P, H - y), min(P, W - x)) for y in range(0, H, P) for x in range(0, W, P)]


def shear(img, o):
    """Sheared copy: row i moved right by o*i, zeros elsewhere (Fig. 4b)."""
    img = np.asarray(img)
    H, W = img.shape[:2]
    L = W + (H - 1) * o
    out = np.zeros((H, L) + img.shape[2:], dtype=img.dtype)
    for i in range(H):
        out[i, o * i:o * i + W] = img[i]
    return out


def unshear(simg, o, W):
    simg = np.asarray(simg)
    H = simg.shape[0]
    return np.stack([simg[i, o * i:o * i + W] for i in range(H)])


def sheared_kernel_positions(h):
    """Window position (column within the h(h+2) columns before the current one)
    of every context offset, for each kernel row d = h..0 (farthest row first)."""
    o = h + 1
    Wk = h * (h + 2)
    rows = []
    for d in range(h, -1, -1):
        dxs = range(-h, h + 1) if d > 0 else range(-h, 0)
        rows.append([Wk + (-d * o + dx) for dx in dxs])
    return rows


def sheared_kernel(kernel_rows, h):
    """Shear the first-layer kernel of Fig. 5.

    kernel_rows[r] lists the unmasked weights of kernel row r (top row first):
    2h+1 entries for rows above the pixel, h for the pixel's own row.  Returns
    the (h+1) x h(h+2) sheared kernel as a list of lists (0 = structural zero).
    """
    Wk = h * (h + 2)
    out = []
    for vals, pos in zip(kernel_rows, sheared_kernel_positions(h)):
        row = [0] * Wk
        for v, p in zip(vals, pos):
            row[p] = v
        out.append(row)
    return out
