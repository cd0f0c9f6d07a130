"""Helpers shared by the GPU tests (input marshalling only)."""
import numpy as np
import torch

from paper_2201_05213_gb300 import build as B
from paper_2201_05213_gb300 import codec as CD
from paper_2201_05213_gb300 import synth

DEV = torch.device("cuda")


def ensure_built():
    B.build()


def to_dev(img):
    return torch.from_numpy(np.ascontiguousarray(img)).to(DEV)


def make_codec(cfg, prec, seed=0, scale=1.0):
    h, C, R, K = cfg
    w = synth.xavier_weights(h, C, R, K, seed=seed) * np.float32(scale)
    return CD.Codec(h, C, R, K, prec, w), w


def images(seed, sizes, n_poly=4):
    return synth.make_batch(seed, sizes, n_poly)
