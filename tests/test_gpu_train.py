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
    wt = torch.tensor(w, device=DEV, requires_grad=True)
    loss = CD.LocalModelNLL.apply(wt, codec, batch)
    loss.backward()
    _, grad = codec.loss_grad(batch)
    assert torch.equal(wt.grad, grad)


# BF16 tensor-core adjoint: every weight, activation and output gradient is
# rounded to BF16 (relative error 2^-9 each) and products accumulate in FP32,
# so the gradient is compared in norm: relative L2 error <= 3e-2 and every
# element within 5e-2 of the largest; the loss (bits per dimension) within the
# BF16 code-length tolerance 0.03 of the FP64 oracle's.  The network's own
# adjoint agrees with an FP64 emulation of the same BF16 roundings to ~1e-4;
# what remains is the likelihood gradient's sensitivity to the BF16 outputs,
# about 0.5 % at Xavier-scale weights (and ~10 % at weights scaled by 1.5,
# where the untrained mixtures are very sharp), so the weights here are the
# Xavier ones.
def _bf16_close(g, ref):
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    worst = np.abs(g - ref).max() / np.abs(ref).max()
    assert rel <= 3e-2 and worst <= 5e-2, (rel, worst)
    return rel, worst


@pytest.mark.parametrize("cfg", [(1, 16, 1, 4), (2, 32, 0, 10), (3, 64, 2, 10), (3, 64, 3, 10)])
def test_bf16_tensor_core_gradient_matches_oracle(cfg):
    codec, w = make_codec(cfg, N.NLC_BF16, seed=3)
    batch = synth.random_crops(2, 3, size=12, source=64)
    loss, grad = codec.loss_grad(torch.from_numpy(batch).to(DEV))
    ref_loss, ref_grad = O.nll_grad(cfg, w.astype(np.float64), batch)
    assert abs(float(loss) - ref_loss) <= 0.03, (float(loss), ref_loss)
    _bf16_close(grad.cpu().numpy().astype(np.float64), ref_grad)
    # deterministic: the same call gives the same bits
    loss2, grad2 = codec.loss_grad(torch.from_numpy(batch).to(DEV))
    assert torch.equal(grad, grad2) and torch.equal(loss, loss2)


def test_bf16_tensor_core_gradient_ragged_tile():
    # 3 x 23 x 29 = 2001 pixels: fifteen full 128-pixel tiles and a ragged
    # one of 81 pixels, tiles spanning image boundaries
    cfg = (3, 64, 2, 10)
    codec, w = make_codec(cfg, N.NLC_BF16, seed=8)
    batch = np.stack([synth.make_image(40 + k, 23, 29) for k in range(3)])
    _, grad = codec.loss_grad(torch.from_numpy(batch).to(DEV))
    _, ref_grad = O.nll_grad(cfg, w.astype(np.float64), batch)
    _bf16_close(grad.cpu().numpy().astype(np.float64), ref_grad)


def _oracle_outputs_dot(cfg, w, batch, R):
    """sum over pixels and outputs of R * network outputs (FP64 oracle)."""
    tot = 0.0
    K10 = 10 * cfg[3]
    n = batch.shape[1] * batch.shape[2]
    for k in range(batch.shape[0]):
        out = O.forward_image(cfg, w, batch[k]).reshape(-1, K10)
        tot += float((out * R[k * n:(k + 1) * n]).sum())
    return tot


@pytest.mark.parametrize("prec", [N.NLC_FP32, N.NLC_BF16])
def test_backward_of_outputs_against_central_differences(prec):
    # nlc_backward maps an upstream gradient of the network outputs to the
    # weights: against central differences (step 1e-3) of the FP64 oracle's
    # sum(R * outputs) on 32 random weights
    cfg = (2, 32, 1, 4)
    codec, w = make_codec(cfg, prec, seed=12, scale=1.5)
    batch = synth.random_crops(9, 2, size=9, source=32)
    rng = np.random.default_rng(1)
    R = rng.normal(0, 1, (2 * 81, 10 * cfg[3]))
    dw = codec.backward(torch.from_numpy(batch).to(DEV),
                        torch.from_numpy(R.astype(np.float32)).to(DEV)).cpu().numpy()
    w64 = w.astype(np.float64)
    idx = rng.choice(len(w), 32, replace=False)
    fd = []
    for k in idx:
        wp, wm = w64.copy(), w64.copy()
        wp[k] += 1e-3
        wm[k] -= 1e-3
        fd.append((_oracle_outputs_dot(cfg, wp, batch, R) - _oracle_outputs_dot(cfg, wm, batch, R)) / 2e-3)
    fd = np.array(fd)
    scale = np.abs(fd).max()
    tol = 1e-3 if prec == N.NLC_FP32 else 5e-2
    assert np.abs(dw[idx] - fd).max() <= tol * scale, np.abs(dw[idx] - fd).max() / scale


def test_local_model_autograd_composes_with_any_loss():
    cfg = (3, 64, 2, 10)
    codec, w = make_codec(cfg, N.NLC_BF16, seed=13)
    batch = torch.from_numpy(synth.random_crops(10, 2, size=16, source=32)).to(DEV)
    wt = torch.tensor(w, device=DEV, requires_grad=True)
    P = CD.LocalModel.apply(wt, codec, batch)
    assert P.shape == (2 * 256, 100)
    R = torch.randn_like(P)
    (P * R).sum().backward()
    ref = codec.backward(batch, R)
    assert torch.equal(wt.grad, ref)
    # the forward equals nlc_forward on the same weights
    P2, _ = codec.forward([batch[0], batch[1]], 0)
    assert torch.equal(P, P2)


def test_bf16_training_reduces_code_length():
    cfg = (3, 64, 2, 10)
    codec, _ = make_codec(cfg, N.NLC_BF16, seed=6)
    crops = torch.from_numpy(synth.random_crops(7, 512, size=32, source=128)).to(DEV)
    first = None
    for step in range(80):
        b = crops[(step * 64) % 512:(step * 64) % 512 + 64]
        loss = codec.train_step(b, 3e-3)
        first = loss if first is None else first
    final, _ = codec.loss_grad(crops[:64])
    assert float(final) < first - 1.0, (first, float(final))


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
