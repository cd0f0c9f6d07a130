"""The hand-written adjoint (mixture NLL, 1x1 residual blocks, masked first
layer) against the oracle's FP64 analytic gradient and against central
finite differences of the oracle's FP64 objective (Eq. 2), plus a short
training run that must reduce the code length."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_05213_gb300 import codec as CD
from paper_2201_05213_gb300 import nlc as N
from paper_2201_05213_gb300 import synth

from gpu_util import DEV, ensure_built, make_codec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("cfg", [(1, 16, 1, 4), (2, 32, 1, 10), (3, 64, 2, 10)])
def test_gradient_matches_oracle(cfg):
    codec, w = make_codec(cfg, N.NLC_FP32, seed=3, scale=1.5)
    batch = synth.random_crops(2, 3, size=12, source=64)
    loss, grad = codec.loss_grad(torch.from_numpy(batch).to(DEV))
    ref_loss, ref_grad = O.nll_grad(cfg, w.astype(np.float64), batch)
    assert abs(float(loss) - ref_loss) <= 1e-5 * ref_loss
    g = grad.cpu().numpy().astype(np.float64)
    scale = np.abs(ref_grad).max()
    assert np.abs(g - ref_grad).max() <= 1e-4 * scale, np.abs(g - ref_grad).max() / scale


def test_gradient_central_differences():
    # 64 random weights, step 1e-3, FP64 objective of the oracle
    cfg = (3, 64, 2, 10)
    codec, w = make_codec(cfg, N.NLC_FP32, seed=4)
    batch = synth.random_crops(5, 2, size=10, source=64)
    _, grad = codec.loss_grad(torch.from_numpy(batch).to(DEV))
    g = grad.cpu().numpy().astype(np.float64)
    w64 = w.astype(np.float64)
    rng = np.random.default_rng(0)
    idx = rng.choice(len(w), 64, replace=False)
    fd = []
    for k in idx:
        wp, wm = w64.copy(), w64.copy()
        wp[k] += 1e-3
        wm[k] -= 1e-3
        fd.append((O.nll_grad(cfg, wp, batch, False) - O.nll_grad(cfg, wm, batch, False)) / 2e-3)
    fd = np.array(fd)
    scale = np.abs(g).max()
    assert np.abs(fd - g[idx]).max() <= 2e-3 * scale + 1e-6, np.abs(fd - g[idx]).max() / scale


def test_autograd_function_uses_the_adjoint():
    cfg = (1, 16, 1, 4)
    codec, w = make_codec(cfg, N.NLC_FP32, seed=5)
    batch = torch.from_numpy(synth.random_crops(6, 2, size=8, source=32)).to(DEV)
    wt = torch.tensor(w, requires_grad=True)
    loss = CD.LocalModelNLL.apply(wt, codec, batch)
    loss.backward()
    _, grad = codec.loss_grad(batch)
    assert torch.allclose(wt.grad, grad.cpu())


def test_training_reduces_code_length():
    cfg = (3, 32, 1, 10)
    codec, _ = make_codec(cfg, N.NLC_FP32, seed=6)
    crops = torch.from_numpy(synth.random_crops(7, 256, size=16, source=128)).to(DEV)
    first = None
    for step in range(60):
        b = crops[(step * 32) % 256:(step * 32) % 256 + 32]
        loss = codec.train_step(b, 3e-3)
        first = loss if first is None else first
    final, _ = codec.loss_grad(crops[:64])
    assert float(final) < first - 1.0, (first, float(final))
