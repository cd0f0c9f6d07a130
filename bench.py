"""Benchmark: decoded pixels/s of the batched wavefront + adjacent-patch decoder.

Workload (one step = one decode of the whole batch through the hot path):
one 2048x2048 and eight 1024x1024 RGB images from the seeded generator
(seed 4, 64 polygons each), coded in independent 256x256 patches with one
rANS stream per patch row, h=3, C=64, 2 residual blocks, K=10, BF16 network
on tcgen05 tensor cores with FP32 mixture/CDF and integer rANS.  The model is
first trained in-run on seeded 32x32 crops (no pretrained weights exist).

Reported next to the decoder: the same containers decoded sequentially on the
same GPU (one pixel per image per step, the paper's sequential decoder), the
encoder's throughput, code lengths (actual bytes and model-ideal), the FP64
oracle's code length on sampled pixels, a roofline line for the decode
kernel, an end-to-end number through the C ABI with host buffers, and the
oracle decoder timed on bounded samples on one host core and on all of them
(one process per core over independent patches).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import glob
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "decoded pixels/s and bpd vs same-GPU sequential decode, 32^2-2048^2 RGB"
UNIT = "decoded px/s"
CFG = (3, 64, 2, 10)
PATCH = 256
WORKLOADS = {
    # the headline configuration (one 2048^2 and eight 1024^2 images)
    "full": [(2048, 2048)] + [(1024, 1024)] * 8,
    # one 1024^2 image: the small case for profiler captures
    "small": [(1024, 1024)],
}
SIZES = WORKLOADS["full"]
SEED = 4
N_POLY = 64
L2_BYTES = 129 * 2 ** 20


def workload_name():
    imgs = {}
    for s in SIZES:
        imgs[s] = imgs.get(s, 0) + 1
    desc = " + ".join(f"{n}x{h}^2" if h == w else f"{n}x{h}x{w}" for (h, w), n in imgs.items())
    return f"{desc} RGB, 256^2 patches, h=3 C=64 R=2 K=10, BF16 net"


# DRAM traffic of decode_kernel per decoded pixel from one ncu capture of the
# small case at 16 CTAs (1x1024^2: 5.82 MB read + 0.29 MB written for
# 1,048,576 px), scaled to a launch by its pixels.  It holds only for the
# kernel sources it was taken on: TRAFFIC_SRC_SHA is the sha256 of
# DECODER_SOURCES, and any other sources report null.
TRAFFIC_B_PER_PX = 5.82
TRAFFIC_SRC_SHA = "e10c941e99c22be48bf826ed2ee2ac989cf61d75567d02f7f1d9470621dcf631"


# the sources decode_kernel is compiled from
DECODER_SOURCES = ["nlc_decode.cu", "nlc_decode_kernel.cuh", "nlc_tile.cuh", "nlc_tc.cuh",
                   "nlc_model.cuh", "nlc_common.cuh", "nlc_kernels.cuh"]


def _csrc_sha():
    import hashlib
    h = hashlib.sha256()
    for name in DECODER_SOURCES:
        f = os.path.join(ROOT, "paper_2201_05213_gb300", "csrc", name)
        h.update(name.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(rank=0):
    from paper_2201_05213_gb300 import synth
    return synth.make_batch(SEED + 1000 * rank, SIZES, N_POLY)


def train_model(codec, steps, batch=64, lr=2e-3, seed=1):
    """In-run maximum-likelihood training on seeded 32x32 crops (Eq. 2)."""
    import torch
    from paper_2201_05213_gb300 import synth
    pool = torch.from_numpy(synth.random_crops(seed, 4096, size=32, source=256)).cuda()
    g = torch.Generator(device="cpu").manual_seed(seed)
    last = None
    for s in range(steps):
        idx = torch.randint(0, pool.shape[0], (batch,), generator=g).cuda()
        last = codec.train_step(pool[idx].contiguous(), lr if s < steps * 3 // 4 else lr / 4,
                                want_loss=(s == steps - 1))
    return last


def oracle_sample_bpd(w, imgs, n=256, seed=0, patch=PATCH):
    """FP64 oracle model code length (bits/dim) of n sampled pixels, patch units."""
    import oracle as O
    rng = np.random.default_rng(seed)
    tot = 0.0
    per = []
    for k in range(n):
        i = int(rng.integers(0, len(imgs)))
        H, W = imgs[i].shape[:2]
        y, x = int(rng.integers(0, H)), int(rng.integers(0, W))
        P = O.forward_pixels(CFG, w, imgs[i], [y], [x], patch=patch)[0]
        b = O.pixel_bits(CFG[3], P, *imgs[i][y, x])
        per.append((i, y, x, b))
        tot += b
    return tot / (3 * n), per


def uneven_batch_report(codec, w, stream, reps=5):
    """256 generator images with sides uniform in {32, 48, ..., 512} (seed 3),
    whole images as units, one stream per row: one tuned decode plan replayed
    from a CUDA graph; per-image decode latency from the decoder's step end
    times (image i ends at step W_i + (H_i - 1)(h + 1), Algorithm 1)."""
    import torch
    from paper_2201_05213_gb300 import nlc as N
    from paper_2201_05213_gb300 import synth
    sizes = synth.uneven_sizes(3, 256)
    imgs = synth.make_batch(3, sizes)
    d = [torch.from_numpy(i).cuda() for i in imgs]
    n_px = sum(H * W for H, W in sizes)
    data, offs = codec.compress(d, 0, N.NLC_LAYOUT_ROW)
    plan = codec.plan(sizes, 0, N.NLC_LAYOUT_ROW)
    ppc, _ = plan.tune(data, offs, reps=1, stream=stream)
    graph = plan.graph(data, offs)
    for _ in range(2):
        graph.replay()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        graph.replay()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    codec.check()
    for o, i in zip(plan.outs, imgs):
        assert np.array_equal(o.cpu().numpy(), i), "uneven batch round trip differs"
    h = CFG[0]
    steps = np.array([W + (H - 1) * (h + 1) for H, W in sizes])
    times = torch.zeros(int(steps.max()) + 1, dtype=torch.int64, device="cuda")
    N.nlc_decode_step_times(codec.ctx, times)
    plan.run(data, offs, stream)
    torch.cuda.synchronize()
    N.nlc_decode_step_times(codec.ctx, None)
    t = times.cpu().numpy()
    lat = (t[steps] - t[0]) / 1e6
    _, bits = codec.forward(d, 0, params=False, bits=True)
    ob, per = oracle_sample_bpd(w, imgs, n=128, seed=1, patch=0)
    base = np.cumsum([0] + [H * W for H, W in sizes])
    bits_np = bits.cpu().numpy()
    gb = sum(float(bits_np[base[i] + y * sizes[i][1] + x]) for i, y, x, _ in per) / (3 * len(per))
    plan.close()
    return {"workload": "256 images, sides uniform in {32,48,...,512} (seed 3), whole images, "
                        "row streams, h=3 C=64 R=2 K=10 BF16",
            "pixels": n_px, "value": n_px / (ms / 1e3), "unit": UNIT, "ms": ms,
            "px_per_cta": ppc, "steps": int(steps.max()),
            "image_latency_ms": {"p50": float(np.percentile(lat, 50)),
                                 "p99": float(np.percentile(lat, 99)), "max": float(lat.max())},
            "bpd": {"actual": 8.0 * int(offs[-1]) / (3 * n_px),
                    "gpu_model": float(bits.double().sum()) / (3 * n_px),
                    "oracle_model_sample": ob, "gpu_model_sample": gb,
                    "sample": "128 random pixels"}}


def heldout_bpd(codec, n=256, seed=5):
    """Model code length of n held-out 32x32 generator images (bits/dim)."""
    import torch
    from paper_2201_05213_gb300 import synth
    d = [torch.from_numpy(i).cuda() for i in synth.make_batch(seed, [(32, 32)] * n)]
    _, bits = codec.forward(d, 0, params=False, bits=True)
    return float(bits.double().sum()) / (3 * 32 * 32 * n)


def timed_decode(fn, stream, flush, reps=1):
    """Mean CUDA-event time (ms) of fn() over reps runs, L2 flushed before each."""
    import torch
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.mean(ts))


def mufu_peak(local):
    """Measured MUFU rate (ops/s) of the search's ex2 + rcp pair at full
    occupancy, best of three, with the SM clock sampled while it runs."""
    from paper_2201_05213_gb300 import nlc as N
    N.nlc_measure_mufu(2000)
    runs = []
    with ClockSampler(local) as clk:
        for _ in range(3):
            runs.append(N.nlc_measure_mufu(40000))
    c = clk.summary()
    rate, ms = max(runs)
    import torch
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = c["sm_mhz"] or 2070.0
    return {"ops_per_s": rate, "kernel_ms": ms, "sms": sms, "sm_mhz": c["sm_mhz"],
            "ops_per_clk_per_sm": rate / (sms * mhz * 1e6), "clocks": c,
            "how": "nlc_measure_mufu: 8 independent rcp.approx(1 + ex2.approx(x)) chains per "
                   "thread, 512-thread CTAs at full occupancy on every SM, CUDA events"}


def decode_decomposition(codec, imgs, dimgs, data, offs, stream, flush, wave_ms):
    """The speed-up split into its two sources (Table 2b separates the
    sequential and wavefront decoders; the patches are this workload's own):
    raster order inside every patch (one pixel per patch and step), the
    wavefront on whole images (no patches), and both (the timed decoder)."""
    import torch
    from paper_2201_05213_gb300 import nlc as N
    n_px = sum(i.shape[0] * i.shape[1] for i in imgs)
    outs = [torch.empty_like(t) for t in dimgs]
    res = {}
    # raster inside each patch, same containers
    plan = codec.plan(SIZES, PATCH, N.NLC_LAYOUT_ROW, N.NLC_SCHED_RASTER, outs=outs)
    ppc, _ = plan.tune(data, offs, reps=1, stream=stream)
    ms = timed_decode(lambda: plan.run(data, offs, stream), stream, flush, reps=1)
    codec.check()
    for a, b in zip(outs, imgs):
        assert np.array_equal(a.cpu().numpy(), b), "raster round trip differs"
    plan.close()
    res["patch_raster"] = {"value": n_px / (ms / 1e3), "ms": ms, "steps": PATCH * PATCH,
                           "px_per_cta": ppc, "how": "NLC_SCHED_RASTER on the same patch "
                           "containers: one pixel per patch per step"}
    # wavefront on whole images (each image one unit, one stream per row)
    wdata, woffs = codec.compress(dimgs, 0, N.NLC_LAYOUT_ROW)
    plan = codec.plan(SIZES, 0, N.NLC_LAYOUT_ROW, N.NLC_SCHED_WAVEFRONT, outs=outs)
    ppc, _ = plan.tune(wdata, woffs, reps=1, stream=stream)
    ms = timed_decode(lambda: plan.run(wdata, woffs, stream), stream, flush, reps=2)
    codec.check()
    for a, b in zip(outs, imgs):
        assert np.array_equal(a.cpu().numpy(), b), "whole-image wavefront round trip differs"
    plan.close()
    H, W = max(SIZES)
    res["image_wavefront"] = {"value": n_px / (ms / 1e3), "ms": ms,
                              "steps": W + (H - 1) * (CFG[0] + 1), "px_per_cta": ppc,
                              "bytes": int(woffs[-1]),
                              "how": "NLC_SCHED_WAVEFRONT on whole-image containers"}
    res["patch_wavefront"] = {"value": n_px / (wave_ms / 1e3), "ms": wave_ms,
                              "steps": PATCH + (PATCH - 1) * (CFG[0] + 1),
                              "how": "the timed decoder (both schemes)"}
    return res


def cfg1_wavefront_fp32(w, stream, flush):
    """64 generator images of 64x64 (seed 1), h=3 C=64 R=2 K=10, FP32 network,
    the in-run trained weights, one stream per row: wavefront decode against
    the sequential decode of the same containers on the same GPU."""
    import torch
    from paper_2201_05213_gb300 import codec as CD
    from paper_2201_05213_gb300 import nlc as N
    from paper_2201_05213_gb300 import synth
    sizes = [(64, 64)] * 64
    imgs = synth.make_batch(1, sizes)
    d = [torch.from_numpy(i).cuda() for i in imgs]
    codec = CD.Codec(*CFG, N.NLC_FP32, w)
    data, offs = codec.compress(d, 0, N.NLC_LAYOUT_ROW)
    n_px = 64 * 64 * 64
    res = {"workload": "64 x 64^2 RGB (seed 1), whole images, row streams, h=3 C=64 R=2 K=10, "
                       "FP32 network"}
    for name, sched in (("wavefront", N.NLC_SCHED_WAVEFRONT), ("sequential", N.NLC_SCHED_SEQUENTIAL)):
        plan = codec.plan(sizes, 0, N.NLC_LAYOUT_ROW, sched)
        ppc, _ = plan.tune(data, offs, reps=1, stream=stream)
        ms = timed_decode(lambda: plan.run(data, offs, stream), stream, flush, reps=3)
        codec.check()
        for a, b in zip(plan.outs, imgs):
            assert np.array_equal(a.cpu().numpy(), b), f"cfg1 {name} round trip differs"
        plan.close()
        res[name] = {"value": n_px / (ms / 1e3), "unit": UNIT, "ms": ms, "px_per_cta": ppc,
                     "steps": 316 if name == "wavefront" else 4096}
    res["speedup"] = res["sequential"]["ms"] / res["wavefront"]["ms"]
    _, bits = codec.forward(d, 0, params=False, bits=True)
    res["bpd"] = {"actual": 8.0 * int(offs[-1]) / (3 * n_px),
                  "gpu_model": float(bits.double().sum()) / (3 * n_px)}
    codec.close()
    return res


def cfg2_training(steps):
    """Training throughput at batch 128 of 32x32 crops (seed 2) for h = 1, 2,
    3 (C=64, R=2, K=10, BF16 context), and the held-out code length on 256
    generator images after `steps` steps."""
    import torch
    from paper_2201_05213_gb300 import codec as CD
    from paper_2201_05213_gb300 import nlc as N
    from paper_2201_05213_gb300 import synth
    out = {}
    pool = torch.from_numpy(synth.random_crops(2, 8192, size=32, source=256)).cuda()
    for h in (1, 2, 3):
        cfg = (h, CFG[1], CFG[2], CFG[3])
        codec = CD.Codec(*cfg, N.NLC_BF16, synth.xavier_weights(*cfg, seed=0))
        g = torch.Generator(device="cpu").manual_seed(2)
        idx = [torch.randint(0, pool.shape[0], (128,), generator=g).cuda() for _ in range(steps)]
        for i in idx[:3]:
            codec.train_step(pool[i].contiguous(), 2e-3, want_loss=False)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        last = None
        for s_ in range(steps):
            b = pool[idx[s_]].contiguous()
            last = codec.train_step(b, 2e-3 if s_ < steps * 3 // 4 else 5e-4,
                                    want_loss=(s_ == steps - 1))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[f"h{h}"] = {"steps": steps, "batch": 128, "steps_per_s": steps / dt,
                        "px_per_s": steps * 128 * 1024 / dt, "final_loss_bpd": last,
                        "heldout_bpd": heldout_bpd(codec)}
        codec.close()
    out["heldout"] = "256 generator images of 32x32 (seed 5)"
    out["timed"] = "wall clock of the steps (data indexing on the GPU included), after 3 warm-ups"
    return out


def model_size_sweep(imgs, dimgs, stream, flush, train_steps):
    """Table 2a's axis on this workload: decode throughput and code length of
    the local model with 0, 1 and 3 residual blocks (h=3, C=64, K=10, BF16),
    each trained in-run like the headline model."""
    from paper_2201_05213_gb300 import codec as CD
    from paper_2201_05213_gb300 import nlc as N
    from paper_2201_05213_gb300 import synth
    import torch
    n_px = sum(i.shape[0] * i.shape[1] for i in imgs)
    res = {}
    for R in (0, 1, 3):
        cfg = (CFG[0], CFG[1], R, CFG[3])
        codec = CD.Codec(*cfg, N.NLC_BF16, synth.xavier_weights(*cfg, seed=0))
        train_model(codec, train_steps)
        data, offs = codec.compress(dimgs, PATCH, N.NLC_LAYOUT_ROW)
        plan = codec.plan(SIZES, PATCH, N.NLC_LAYOUT_ROW)
        ppc, _ = plan.tune(data, offs, reps=1, stream=stream)
        ms = timed_decode(lambda: plan.run(data, offs, stream), stream, flush, reps=3)
        codec.check()
        for a, b in zip(plan.outs, imgs):
            assert np.array_equal(a.cpu().numpy(), b), f"R={R} round trip differs"
        plan.close()
        _, bits = codec.forward(dimgs, PATCH, params=False, bits=True)
        res[f"R{R}"] = {"value": n_px / (ms / 1e3), "unit": UNIT, "ms": ms, "px_per_cta": ppc,
                        "weights": N.nlc_num_weights(*cfg),
                        "bpd": {"actual": 8.0 * int(offs[-1]) / (3 * n_px),
                                "gpu_model": float(bits.double().sum()) / (3 * n_px)}}
        codec.close()
    res["how"] = ("each model trained in-run on seeded 32x32 crops (batch 64, "
                  f"{train_steps} steps), then the headline decode (tuned plan)")
    return res


def shearloc_report(w, imgs, dimgs, stream, flush, decomposition):
    """Section 3.1 / Table 2's ShearLoC column on this workload: the same
    weights as a sheared model (first layer as Fig. 5's sheared kernels; the
    wavefront decoder keeps decoded pixels in sheared rings and reads each
    front's context as one window tile), on the 256^2 patches and on whole
    images, beside the plain wavefront decoder's times of the same run."""
    from paper_2201_05213_gb300 import codec as CD
    from paper_2201_05213_gb300 import nlc as N
    n_px = sum(i.shape[0] * i.shape[1] for i in imgs)
    codec = CD.Codec(*CFG, N.NLC_BF16_SHEARED, w)
    res = {}
    for name, patch, plain in (("patches", PATCH, decomposition.get("patch_wavefront")),
                               ("whole_images", 0, decomposition.get("image_wavefront"))):
        data, offs = codec.compress(dimgs, patch, N.NLC_LAYOUT_ROW)
        plan = codec.plan(SIZES, patch, N.NLC_LAYOUT_ROW)
        ppc, _ = plan.tune(data, offs, reps=1, stream=stream)
        graph = plan.graph(data, offs)
        ms = timed_decode(lambda: graph.replay(), stream, flush, reps=3)
        codec.check()
        for a, b in zip(plan.outs, imgs):
            assert np.array_equal(a.cpu().numpy(), b), f"ShearLoC {name} round trip differs"
        plan.close()
        _, bits = codec.forward(dimgs, patch, params=False, bits=True)
        res[name] = {"value": n_px / (ms / 1e3), "unit": UNIT, "ms": ms, "px_per_cta": ppc,
                     "bpd": {"actual": 8.0 * int(offs[-1]) / (3 * n_px),
                             "gpu_model": float(bits.double().sum()) / (3 * n_px)}}
        if plain and "ms" in plain:
            res[name]["plain_wavefront_ms"] = plain["ms"]
            res[name]["speedup_vs_plain_wavefront"] = plain["ms"] / ms
    codec.close()
    res["how"] = ("NLC_BF16_SHEARED context with the headline model's weights; tuned decode plan "
                  "replayed from a CUDA graph, L2 flushed before each of 3 timed runs")
    return res


def sampler_report(codec, stream, flush):
    """Sampling from the model with the same schedules (Section 5): the
    headline workload's image sizes and 256^2 patches, wavefront and raster
    order inside the patches; the samples' own code length under the model."""
    import torch
    from paper_2201_05213_gb300 import nlc as N
    outs = [torch.empty((H, W, 3), dtype=torch.uint8, device="cuda") for H, W in SIZES]
    n_px = sum(H * W for H, W in SIZES)
    res = {}
    for name, sched, reps in (("wavefront", N.NLC_SCHED_WAVEFRONT, 3),
                              ("patch_raster", N.NLC_SCHED_RASTER, 1)):
        codec.sample(SIZES, PATCH, 7, sched, stream, outs)  # warm-up and set-up
        ms = timed_decode(lambda: N.nlc_sample(codec.ctx, outs, PATCH, 7, sched, stream), stream,
                          flush, reps)
        codec.check()
        res[name] = {"value": n_px / (ms / 1e3), "unit": "sampled px/s", "ms": ms}
    _, bits = codec.forward(outs, PATCH, params=False, bits=True)
    res["sample_bpd"] = float(bits.double().sum()) / (3 * n_px)
    res["speedup"] = res["patch_raster"]["ms"] / res["wavefront"]["ms"]
    res["how"] = ("nlc_sample: the decoder's schedule, network and tables, each symbol the "
                  "inverse CDF of its table at a SplitMix64 counter-based uniform (seed 7)")
    return res


def cpu_baseline(w, img, budget_s=12.0):
    """The oracle's sequential decoder on a bounded sample (first rows of the
    first 256x256 patch, decoded as one unit) on one host core."""
    import oracle as O
    rows = 8
    sub = np.ascontiguousarray(img[:rows, :PATCH])
    words, lens, _, _ = O.encode_image(CFG, w, sub, 0, 1)
    t0 = time.perf_counter()
    dec, ok = O.decode_image(CFG, w, words, lens, rows, PATCH, 0, 1)
    dt = time.perf_counter() - t0
    assert ok and (dec == sub).all()
    # grow the sample to fill roughly the budget
    if dt < budget_s / 4:
        rows = int(min(PATCH, max(rows, rows * budget_s / max(dt, 1e-3) / 2)))
        sub = np.ascontiguousarray(img[:rows, :PATCH])
        words, lens, _, _ = O.encode_image(CFG, w, sub, 0, 1)
        t0 = time.perf_counter()
        dec, ok = O.decode_image(CFG, w, words, lens, rows, PATCH, 0, 1)
        dt = time.perf_counter() - t0
        assert ok and (dec == sub).all()
    px = rows * PATCH
    return {"value": px / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "rows": rows,
            "sample": f"{rows}x{PATCH} px of the first 256^2 patch of the 2048^2 image, "
                      f"sequential FP64 decode, {dt:.1f} s"}


_BARRIER = None


def _pool_init(barrier):
    global _BARRIER
    _BARRIER = barrier
    sys.path.insert(0, ROOT)


def _oracle_decode_task(task):
    """One worker: encode its own unit (untimed), wait for all workers, then
    time the oracle's sequential decode of it."""
    import oracle as O
    w, sub = task
    words, lens, _, _ = O.encode_image(CFG, w, sub, 0, 1)
    _BARRIER.wait()
    t0 = time.perf_counter()
    dec, ok = O.decode_image(CFG, w, words, lens, sub.shape[0], sub.shape[1], 0, 1)
    dt = time.perf_counter() - t0
    return sub.shape[0] * sub.shape[1], dt, bool(ok and (dec == sub).all())


def cpu_model():
    """The host CPU's model (lscpu's "Model name", else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


class ParallelOracle:
    """The oracle's sequential decoder over independent units, one process
    per online host core (spawned, so safe beside an initialised CUDA
    context): every worker decodes the first `rows` rows of its own 256x256
    patch of the 2048^2 image, all starting together; px/s = all workers'
    pixels / the longest worker's decode time."""

    def __init__(self):
        import multiprocessing as mp
        self.n = os.cpu_count() or 1
        ctx = mp.get_context("spawn")
        self.pool = ctx.Pool(self.n, initializer=_pool_init, initargs=(ctx.Barrier(self.n),))

    def run(self, w, img, rows):
        per = img.shape[1] // PATCH
        tasks = []
        for k in range(self.n):
            y, x = PATCH * ((k // per) % (img.shape[0] // PATCH)), PATCH * (k % per)
            tasks.append((w, np.ascontiguousarray(img[y:y + rows, x:x + PATCH])))
        res = self.pool.map(_oracle_decode_task, tasks, chunksize=1)
        assert all(r[2] for r in res), "parallel oracle round trip differs"
        px, dt = sum(r[0] for r in res), max(r[1] for r in res)
        return {"value": px / dt, "unit": UNIT, "cores": self.n, "kind": "oracle",
                "pixels": px, "seconds": dt,
                "cpu": cpu_model(),
                "sample": f"{self.n} processes, each {rows}x{PATCH} px of its own 256^2 patch "
                          f"of the 2048^2 image, sequential FP64 decode, {dt:.1f} s"}

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2201_05213_gb300 import synth
    w = synth.xavier_weights(*CFG, seed=0)
    img = synth.make_image(SEED, 2048, 2048, N_POLY, index=0)
    # one core sizes the sample (about 4 s); then every step decodes half as
    # many rows in each of one process per host core
    single = cpu_baseline(w, img, budget_s=4.0)
    rows = max(8, single.pop("rows") // 2)
    par = ParallelOracle()
    try:
        vals = [par.run(w, img, rows) for _ in range(args.warmup + args.steps)]
    finally:
        par.close()
    timed = vals[args.warmup:]
    # each step decodes the bounded sample; value = its pixels / its time
    v = float(np.sum([t["pixels"] for t in timed]) / np.sum([t["seconds"] for t in timed]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * float(np.mean([t["seconds"] for t in timed])),
            "pixels_per_step": int(timed[-1]["pixels"]),
            "full_workload_ms_extrapolated": 1000.0 * sum(h * w_ for h, w_ in SIZES) / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(), "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": timed[-1]["cores"],
                             "kind": "oracle", "cpu": timed[-1]["cpu"],
                             "sample": timed[-1]["sample"]},
            "cpu_baseline_one_core": single,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nlc", choices=["nlc", "reference"])
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--cfg2-steps", type=int, default=2000,
                    help="training steps per horizon of the batch-128 training report")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the decomposition, FP32, training and model-size reports")
    ap.add_argument("--no-seq", action="store_true", help="skip the sequential baseline")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--workload", default="full", choices=sorted(WORKLOADS))
    ap.add_argument("--no-uneven", action="store_true", help="skip the 256-image uneven batch")
    ap.add_argument("--max-ctas", type=int, default=0,
                    help="cap the decoder's CTAs (0 = all co-resident; profiling of small cases)")
    args = ap.parse_args()
    global SIZES
    SIZES = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    import __graft_entry__
    __graft_entry__.build()
    from paper_2201_05213_gb300 import codec as CD
    from paper_2201_05213_gb300 import nlc as N
    from paper_2201_05213_gb300 import shard
    from paper_2201_05213_gb300 import synth

    dev = torch.device("cuda", local)
    imgs = make_workload(rank)
    n_px = sum(h * w for h, w in SIZES)
    w0 = synth.xavier_weights(*CFG, seed=0)
    codec = CD.Codec(*CFG, N.NLC_BF16, w0)
    if args.max_ctas > 0:
        N.nlc_set_tuning(codec.ctx, 8, args.max_ctas)
    t0 = time.perf_counter()
    train_loss = train_model(codec, args.train_steps) if args.train_steps > 0 else None
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    w = codec.get_weights()

    dimgs = [torch.from_numpy(i).to(dev) for i in imgs]
    stream = torch.cuda.current_stream()
    # encoder
    data, offs = codec.compress(dimgs, PATCH, N.NLC_LAYOUT_ROW)
    torch.cuda.synchronize()
    te0 = torch.cuda.Event(enable_timing=True)
    te1 = torch.cuda.Event(enable_timing=True)
    te0.record(stream)
    data, offs = codec.compress(dimgs, PATCH, N.NLC_LAYOUT_ROW, check=False)
    te1.record(stream)
    codec.check()
    enc_ms = te0.elapsed_time(te1)
    total_bytes = int(offs[-1])
    outs = [torch.empty_like(t) for t in dimgs]
    sizes = SIZES
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)

    def decode_call():
        N.nlc_decompress(codec.ctx, data, offs, outs, PATCH, N.NLC_LAYOUT_ROW,
                         N.NLC_SCHED_WAVEFRONT, stream)

    # the timed decode: a decode plan (host work done once), its pixels per CTA
    # picked by the library's tuner, replayed from a CUDA graph
    plan = codec.plan(sizes, PATCH, N.NLC_LAYOUT_ROW, outs=outs)
    tuned_ppc, _ = plan.tune(data, offs, reps=1, stream=stream)
    graph = plan.graph(data, offs)

    def decode():
        graph.replay()

    for _ in range(args.warmup):
        decode()
    codec.check()
    for a, b in zip(outs, imgs):
        assert np.array_equal(a.cpu().numpy(), b), "round trip differs"
    times = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            decode()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    codec.check()
    ms = shard.max_over_ranks(float(np.mean(times)), dev)
    value = world * n_px / (ms / 1e3)

    # the same decode through nlc_decompress (host planning on every call)
    call_times = []
    for _ in range(max(2, args.steps // 2)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        decode_call()
        e1.record(stream)
        e1.synchronize()
        call_times.append(e0.elapsed_time(e1))
    codec.check()
    call_ms = float(np.mean(call_times))

    # per-step latency against the dependency-bound step count: a run of the
    # plan outside the graph (captured without profiling), which launches the
    # decoder's instrumented build, timed on its own
    N.nlc_decode_profile(codec.ctx, 1, read=False)
    flush.zero_()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    plan.run(data, offs, stream)
    p1.record(stream)
    p1.synchronize()
    prof_ms = p0.elapsed_time(p1)
    cnt = N.nlc_decode_profile(codec.ctx, 0).astype(np.float64)
    steps_T = max(int(cnt[7]), 1)
    ctas = max(int(cnt[6]), 1)
    mhz = 2070.0
    phase_us = {name: float(cnt[i]) / ctas / steps_T / mhz
                for i, name in enumerate(["front", "slots", "gather_network", "coding", "barrier"])}
    npx0 = max(float(cnt[12]), 1.0)
    coding_us = {name: float(cnt[8 + i]) / npx0 / mhz
                 for i, name in enumerate(["setup", "cdf_search", "rans", "posterior"])}
    net_us = {name: float(cnt[13 + i]) / ctas / steps_T / mhz
              for i, name in enumerate(["gather", "mma", "epilogue"])}
    phases = {"steps": steps_T, "ctas": ctas, "tiles_per_cta_step": float(cnt[5]) / ctas / steps_T,
              "network_us_per_step": net_us,
              "us_per_step_measured": 1000.0 * ms / steps_T,
              "instrumented_build_ms": prof_ms,
              "us_per_step_instrumented": 1000.0 * prof_ms / steps_T,
              "us_per_step_by_phase_at_2070MHz": phase_us,
              "coding_us_per_pixel_warp0": coding_us,
              "how": "phase cycles of thread 0 per CTA from the decoder's instrumented build "
                     "(nlc_decode_profile), which keeps its counters in registers and runs "
                     "slower than the timed build: the split of its step, us_per_step_instrumented"}

    # end to end through the C ABI with host buffers
    h_data = data[:total_bytes].cpu().pin_memory()
    h_offs = offs.cpu().pin_memory()
    h_outs = [torch.empty(t.shape, dtype=torch.uint8).pin_memory() for t in dimgs]
    d_in = torch.empty(total_bytes, dtype=torch.uint8, device=dev)
    d_offs = torch.empty_like(offs)
    e2e_times = []
    for it in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d_in.copy_(h_data, non_blocking=True)
        d_offs.copy_(h_offs, non_blocking=True)
        N.nlc_decompress(codec.ctx, d_in, d_offs, outs, PATCH, N.NLC_LAYOUT_ROW,
                         N.NLC_SCHED_WAVEFRONT, stream)
        for ho, do in zip(h_outs, outs):
            ho.copy_(do, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if it >= args.warmup:
            e2e_times.append(e0.elapsed_time(e1))
    codec.check()
    for a, b in zip(h_outs, imgs):
        assert np.array_equal(a.numpy(), b), "end-to-end round trip differs"
    e2e_ms = shard.max_over_ranks(float(np.mean(e2e_times)), dev)

    # code lengths
    _, bits = codec.forward(dimgs, PATCH, params=False, bits=True)
    dims = 3 * n_px
    gpu_model_bpd = float(bits.double().sum()) / dims
    actual_bpd = 8.0 * total_bytes / dims

    extra = {}
    if rank == 0:
        # sequential baseline: same containers, one pixel per image per step
        if not args.no_seq:
            torch.cuda.synchronize()
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            N.nlc_set_tuning(codec.ctx, 1, 0)  # one pixel (image) per CTA and step
            s0.record(stream)
            N.nlc_decompress(codec.ctx, data, offs, outs, PATCH, N.NLC_LAYOUT_ROW,
                             N.NLC_SCHED_SEQUENTIAL, stream)
            s1.record(stream)
            s1.synchronize()
            N.nlc_set_tuning(codec.ctx, 8, 0)
            codec.check()
            seq_ms = s0.elapsed_time(s1)
            for a, b in zip(outs, imgs):
                assert np.array_equal(a.cpu().numpy(), b), "sequential round trip differs"
            extra["sequential_baseline"] = {
                "value": n_px / (seq_ms / 1e3), "unit": UNIT, "ms": seq_ms,
                "steps": max(h * w_ for h, w_ in SIZES), "speedup": seq_ms / ms,
                "how": "same library and containers, NLC_SCHED_SEQUENTIAL (one pixel per image "
                       "per step, patches of an image one after another), one full run"}
        oracle_bpd, _ = oracle_sample_bpd(w.astype(np.float64), imgs, n=192)
        sample_idx = np.random.default_rng(0)
        # GPU model bits on the same sampled pixels
        rng = np.random.default_rng(0)
        bits_np = bits.cpu().numpy()
        base = np.cumsum([0] + [h * w_ for h, w_ in SIZES])
        gsum = 0.0
        for k in range(192):
            i = int(rng.integers(0, len(imgs)))
            H, W = imgs[i].shape[:2]
            y, x = int(rng.integers(0, H)), int(rng.integers(0, W))
            gsum += float(bits_np[base[i] + y * W + x])
        extra["bpd"] = {"actual": actual_bpd, "gpu_model": gpu_model_bpd,
                        "oracle_model_sample": oracle_bpd, "gpu_model_sample": gsum / (3 * 192),
                        "sample": "192 random pixels"}
        extra["encode"] = {"value": n_px / (enc_ms / 1e3), "unit": "encoded px/s", "ms": enc_ms}
        extra["train"] = {"steps": args.train_steps, "batch": 64, "crop": "32x32",
                          "seconds": train_s, "steps_per_s": args.train_steps / max(train_s, 1e-9),
                          "final_loss_bpd": train_loss,
                          "heldout_bpd": heldout_bpd(codec),
                          "heldout": "256 generator images of 32x32 (seed 5)"}
        if not args.no_uneven:
            extra["uneven_batch"] = uneven_batch_report(codec, w.astype(np.float64), stream)
        if not args.no_extra:
            def report(key, fn):  # a failing report is recorded, the line still prints
                try:
                    extra[key] = fn()
                except Exception as e:  # noqa: BLE001
                    extra[key] = {"error": f"{type(e).__name__}: {e}"[:400]}
                    print(f"bench: report {key} failed: {e}", file=sys.stderr)
            report("decode_decomposition",
                   lambda: decode_decomposition(codec, imgs, dimgs, data, offs, stream, flush, ms))
            if not args.no_seq and "error" not in extra["decode_decomposition"]:
                seq = extra["sequential_baseline"]["ms"]
                for k, v in extra["decode_decomposition"].items():
                    v["speedup_vs_sequential"] = seq / v["ms"]
            report("cfg1_wavefront_fp32", lambda: cfg1_wavefront_fp32(w, stream, flush))
            report("cfg2_training", lambda: cfg2_training(args.cfg2_steps))
            report("model_size_sweep",
                   lambda: model_size_sweep(imgs, dimgs, stream, flush, args.train_steps))
            report("sampler", lambda: sampler_report(codec, stream, flush))
            report("shearloc", lambda: shearloc_report(w, imgs, dimgs, stream, flush,
                                                       extra.get("decode_decomposition", {})))
        if not args.no_cpu:
            import oracle as O
            t0 = time.perf_counter()
            ob, npx_o = O.batch_bits_parallel(CFG, w.astype(np.float64), imgs, PATCH)
            extra["bpd"]["oracle_model_full"] = ob / (3 * npx_o)
            extra["bpd"]["oracle_model_full_seconds"] = time.perf_counter() - t0
            extra["bpd"]["gpu_minus_oracle_full"] = gpu_model_bpd - ob / (3 * npx_o)
            extra["bpd"]["actual_minus_oracle_full"] = actual_bpd - ob / (3 * npx_o)

    peaks, src = _measured_peaks()
    # roofline of the decode kernel: MUFU work of the symbol search, two
    # rounds of 15 boundaries x K logistic terms (ex2 + rcp) per channel
    evals_per_px = 3 * 2 * 15 * CFG[3]
    mufu_ops = 2.0 * evals_per_px * n_px
    clk = clk.summary()
    mufu = mufu_peak(local)
    achieved = mufu_ops / (ms / 1e3)
    flops = 54784.0 * n_px
    hbm_bytes = total_bytes + 3.0 * n_px  # containers read, pixels written
    roof = {"bound": "alu", "unit": "MUFU op/s", "achieved": achieved, "peak": mufu["ops_per_s"],
            "frac": achieved / mufu["ops_per_s"],
            "traffic": TRAFFIC_B_PER_PX * n_px if _csrc_sha() == TRAFFIC_SRC_SHA else None,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the 1x1024^2 "
                              "decode at 16 CTAs, scaled by pixels (bytes per launch)",
            "peak_source": "measured in this run (nlc_measure_mufu, best of 3)",
            "mufu_probe": mufu,
            "work": f"{2 * evals_per_px} MUFU ops/px (search terms only)",
            "tensor": {"achieved_tflops": flops / (ms / 1e3) / 1e12,
                       "peak_tflops": peaks.get("bf16_tflops_sustained"),
                       "frac": flops / (ms / 1e3) / 1e12 / peaks.get("bf16_tflops_sustained", 1700),
                       "peak_source": f"bf16_tflops_sustained, {src}"},
            "hbm": {"achieved_gbs": hbm_bytes / (ms / 1e3) / 1e9, "peak_gbs": peaks.get("hbm_gbs"),
                    "frac": hbm_bytes / (ms / 1e3) / 1e9 / peaks.get("hbm_gbs", 6800.0),
                    "bytes_per_launch": hbm_bytes,
                    "work": "algorithmic: containers read once + 3 B per decoded pixel written",
                    "peak_source": src}}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic (seeded generator; model "
            "trained in-run on seeded crops)",
            "config": {"workload": workload_name(), "images": len(SIZES), "pixels": n_px,
                       "patch": PATCH, "units": sum(((h + PATCH - 1) // PATCH) * ((w + PATCH - 1) // PATCH)
                                                    for h, w in SIZES), "h": CFG[0], "C": CFG[1], "R": CFG[2],
                       "K": CFG[3], "schedule": "wavefront", "layout": "row streams",
                       "decode_path": "nlc_plan_run replayed from a CUDA graph, px_per_cta "
                                      f"{tuned_ppc} picked by nlc_plan_tune",
                       "nlc_decompress_ms": call_ms,
                       "l2": "flushed before every timed step (256 MiB write)"},
            "roofline": roof,
            "e2e": {"value": world * n_px / (e2e_ms / 1e3), "unit": UNIT, "ms": e2e_ms,
                    "h2d_bytes_per_step": total_bytes + 8 * (len(SIZES) + 1),
                    "d2h_bytes_per_step": 3 * n_px},
            "gpu_launches": 5 * args.steps,
            "clocks": clk,
            "decode_phases": phases,
            **extra,
        }
        if not args.no_cpu:
            w64 = w.astype(np.float64)
            line["cpu_baseline"] = cpu_baseline(w64, imgs[0])
            rows = max(8, line["cpu_baseline"].pop("rows") // 2)
            par = ParallelOracle()
            try:
                line["cpu_baseline_all_cores"] = par.run(w64, imgs[0], rows)
            finally:
                par.close()
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
