"""Convenience layer over the nlc binding: buffer allocation with torch and
status checking.  All compute runs in libnlc.so kernels."""
from __future__ import annotations

import numpy as np
import torch

from . import nlc as N


def _raise_status(ctx, stream=None):
    code = N.nlc_sync_status(ctx, stream)
    if code != N.NLC_OK:
        raise N.NLCError(code, N.load().nlc_last_error().decode())


class Codec:
    """A local autoregressive compressor (one nlc context) on the current GPU."""

    def __init__(self, h, C, n_res, K, precision, weights):
        self.cfg = (h, C, n_res, K, precision)
        self.n_weights = N.nlc_num_weights(h, C, n_res, K, precision)
        self.ctx = N.nlc_create(h, C, n_res, K, precision, weights)

    def close(self):
        if self.ctx is not None:
            N.nlc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- weights -------------------------------------------------------------
    def get_weights(self):
        return N.nlc_get_weights(self.ctx, self.n_weights)

    def set_weights(self, w):
        N.nlc_set_weights(self.ctx, w)

    def weight_hash(self):
        return N.nlc_weight_hash(self.ctx)

    def check(self, stream=None):
        _raise_status(self.ctx, stream)

    # -- codec ---------------------------------------------------------------
    def compress(self, imgs, patch=0, layout=1, stream=None, check=True):
        sizes = [(int(t.shape[0]), int(t.shape[1])) for t in imgs]
        cap = N.nlc_compress_bound(sizes, patch, layout)
        dev = imgs[0].device if imgs else torch.device("cuda")
        out = torch.empty(max(cap, 16), dtype=torch.uint8, device=dev)
        offs = torch.empty(len(imgs) + 1, dtype=torch.int64, device=dev)
        N.nlc_compress(self.ctx, imgs, patch, layout, out, offs, stream)
        if check:
            self.check(stream)
        return out, offs

    def decompress(self, data, offs, sizes, patch=0, layout=1, schedule=N.NLC_SCHED_WAVEFRONT,
                   stream=None, outs=None, check=True):
        if outs is None:
            outs = [torch.empty((H, W, 3), dtype=torch.uint8, device=data.device) for H, W in sizes]
        N.nlc_decompress(self.ctx, data, offs, outs, patch, layout, schedule, stream)
        if check:
            self.check(stream)
        return outs

    def sample(self, sizes, patch=0, seed=0, schedule=N.NLC_SCHED_WAVEFRONT, stream=None,
               outs=None):
        """Images of the given sizes drawn from the model (nlc_sample)."""
        if outs is None:
            outs = [torch.empty((H, W, 3), dtype=torch.uint8, device="cuda") for H, W in sizes]
        N.nlc_sample(self.ctx, outs, patch, seed, schedule, stream)
        self.check(stream)
        return outs

    def plan(self, sizes, patch=0, layout=1, schedule=N.NLC_SCHED_WAVEFRONT, outs=None):
        """A DecodePlan for a fixed batch of image sizes."""
        return DecodePlan(self, sizes, patch, layout, schedule, outs)

    def forward(self, imgs, patch=0, params=True, bits=False, stream=None):
        npx = sum(int(t.shape[0]) * int(t.shape[1]) for t in imgs)
        dev = imgs[0].device
        P = torch.empty((npx, 10 * self.cfg[3]), dtype=torch.float32, device=dev) if params else None
        B = torch.empty(npx, dtype=torch.float32, device=dev) if bits else None
        N.nlc_forward(self.ctx, imgs, patch, P, B, stream)
        self.check(stream)
        return P, B

    def tables(self, params, pixels, stream=None):
        n = int(pixels.shape[0])
        cum = torch.empty((n, 3, 257), dtype=torch.int32, device=pixels.device)
        N.nlc_tables(self.ctx, params, pixels, cum, stream)
        self.check(stream)
        return cum

    # -- training ------------------------------------------------------------
    def train_step(self, batch, lr, want_loss=True, stream=None):
        return N.nlc_train_step(self.ctx, batch, lr, stream, want_loss)

    def backward(self, batch, dparams, stream=None):
        """Weight gradient of sum(dparams * network outputs) over the batch."""
        dw = torch.empty(self.n_weights, dtype=torch.float32, device=batch.device)
        N.nlc_backward(self.ctx, batch, dparams, dw, stream)
        self.check(stream)
        return dw

    def loss_grad(self, batch, stream=None):
        loss = torch.empty(1, dtype=torch.float32, device=batch.device)
        grad = torch.empty(self.n_weights, dtype=torch.float32, device=batch.device)
        N.nlc_loss_grad(self.ctx, batch, loss, grad, stream)
        self.check(stream)
        return loss, grad


class DecodePlan:
    """nlc_plan_* for one batch shape: run() issues device work only, so it can
    be captured with graph(); tune() picks the decoder's pixels per CTA."""

    def __init__(self, codec, sizes, patch, layout, schedule, outs=None):
        self.codec = codec
        self.outs = outs if outs is not None else [
            torch.empty((H, W, 3), dtype=torch.uint8, device="cuda") for H, W in sizes]
        self.handle = N.nlc_plan_decode(codec.ctx, self.outs, patch, layout, schedule)

    def run(self, data, offs, stream=None):
        N.nlc_plan_run(self.handle, data, offs, stream)
        return self.outs

    def tune(self, data, offs, reps=2, stream=None):
        return N.nlc_plan_tune(self.handle, data, offs, reps, stream)

    def graph(self, data, offs):
        """A torch.cuda.CUDAGraph whose replay decodes the containers at data."""
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(data, offs, s)  # first run outside the capture
        torch.cuda.current_stream().wait_stream(s)
        with torch.cuda.graph(g):
            self.run(data, offs, torch.cuda.current_stream())
        return g

    def close(self):
        if getattr(self, "handle", None) is not None:
            N.nlc_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _batch_images(batch):
    return [batch[n] for n in range(batch.shape[0])]


class LocalModel(torch.autograd.Function):
    """Network outputs (N H W x 10K, the layout of nlc_forward) of a uint8
    batch (N x H x W x 3, each image one unit) as a function of the FP32
    weights (a CUDA tensor); backward maps the outputs' gradient to the
    weights' with the library's adjoint (nlc_backward)."""

    @staticmethod
    def forward(ctx, weights, codec, batch):
        N.nlc_load_weights(codec.ctx, weights.detach().contiguous())
        P, _ = codec.forward(_batch_images(batch), 0)
        ctx.codec, ctx.batch = codec, batch
        return P

    @staticmethod
    def backward(ctx, gP):
        codec = ctx.codec
        dw = torch.empty(codec.n_weights, dtype=torch.float32, device=gP.device)
        N.nlc_backward(codec.ctx, ctx.batch, gP.contiguous().float(), dw)
        codec.check()
        return dw, None, None


class LocalModelNLL(torch.autograd.Function):
    """Mean code length (bits per dimension) of a uint8 batch as a function of
    the FP32 weights (a CUDA tensor); backward is the library's hand-written
    adjoint of the mixture likelihood and the network."""

    @staticmethod
    def forward(ctx, weights, codec, batch):
        N.nlc_load_weights(codec.ctx, weights.detach().contiguous())
        loss, grad = codec.loss_grad(batch)
        ctx.save_for_backward(grad)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None


def ideal_bits_from_tables(cum, pixels):
    """sum over symbols of -log2(freq / 2^16) for tables cum[n][3][257]."""
    c = cum.to(torch.int64)
    v = pixels.to(torch.int64)
    lo = torch.gather(c, 2, v.unsqueeze(-1)).squeeze(-1)
    hi = torch.gather(c, 2, (v + 1).unsqueeze(-1)).squeeze(-1)
    return float(torch.sum(-torch.log2((hi - lo).to(torch.float64) / 65536.0)))
