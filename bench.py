#!/usr/bin/env python
"""Benchmark of the NTC hot path on one GB300 (replicas on N GPUs).

One step = one pass of the whole hot path over synthetic inputs shaped like
the paper's workloads:
  * random-access decode of a 4096^2 x 16-channel material (13 mips,
    G0 1024^2 x 12, G1 512^2 x 12 at 4 bits, MLP 48-64-64-16) at 2^24
    queries with (u, v) uniform in [0,1)^2 and an integer LOD uniform over
    0..12 -> the headline `value`, decoded texels/s;
  * one optimisation step (sampler, noise, forward, L2 loss, backward,
    Adam) of a 2048^2 x 12-channel material (G0 512^2 x 16, G1 256^2 x 16,
    MLP 48-64-64-12) on 2^18 training texels -> `train_samples_per_s`.
The decode pass streams 0.74 GB (> L2) between training steps, so every
training step starts with a cold L2.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ntc_inputs as gen  # noqa: E402

METRIC = "decoded texels/s & train samples/s (fwd+bwd), % tensor peak, vs FP32 path"
DEC_SIDE, DEC_C, DEC_C0, DEC_K = 4096, 16, 12, 48
TRN_SIDE, TRN_C, TRN_C0, TRN_K = 2048, 12, 16, 48
CROP_STEPS = 20
MAX_SM_MHZ = 2070.0
# DRAM bytes (read + write) of one FP16 decode_ws_kernel launch of the 2^24
# query workload, from a single-launch ncu capture at that size (summarised
# with the other ncu captures); valid only for the kernel sources it was
# taken on (their hash), null otherwise.
DECODE_SOURCES = ("tc_decode_ws.cuh", "tc_decode_common.cuh", "tc_decode_ws.cu", "tc_ptx.cuh",
                  "ntc_device.cuh")
DECODE_TRAFFIC = ("6af1ee09e7d63671", 213.02e6 + 483.10e6)  # (sources sha256[:16], bytes per launch)


def decode_sources_sha():
    h = hashlib.sha256()
    for f in DECODE_SOURCES:
        with open(os.path.join(ROOT, "paper_2305_17105_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "f32", "f16", "f8"])
    ap.add_argument("--train-precision", default="auto", choices=["auto", "f32", "f16"])
    ap.add_argument("--queries", type=int, default=1 << 24)
    ap.add_argument("--batch", type=int, default=1 << 18)
    ap.add_argument("--cpu-seconds", type=float, default=8.0,
                    help="target CPU time of each oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--no-render", action="store_true",
                    help="skip the camera-frame decode of the trained model")
    ap.add_argument("--no-multi", action="store_true",
                    help="skip the 64-material batched decode and training graph")
    ap.add_argument("--decode-train-steps", type=int, default=1000,
                    help="training steps that compress the 4096^2 x 16 decode material "
                         "(0: random grids and weights, for profiling runs)")
    ap.add_argument("--render-steps", type=int, default=0,
                    help="(unused: the camera frame decodes the trained decode material)")
    ap.add_argument("--decode-shape", type=int, default=0, choices=[0, 2, 3, 4, 5],
                    help="tensor-core decode launch shape; 0: chosen by the autotuner "
                         "(profiling runs fix it: the autotuner's timing is not "
                         "meaningful under a profiler)")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed step: skip the crop-sampler, paper-form, 64-material, "
                         "render, FP32, e2e and CPU sections (profiling runs)")
    ap.add_argument("--multi-only", action="store_true",
                    help="the timed step and the 64-material section only (profiling runs)")
    a = ap.parse_args()
    if a.multi_only:
        a.no_cpu_baseline = a.no_e2e = a.no_fp32_compare = a.no_render = True
    if a.no_extras:
        a.no_cpu_baseline = a.no_e2e = a.no_fp32_compare = a.no_render = a.no_multi = True
    return a


# ----------------------------------------------------------------------------
# distributed plumbing (replicas: no data-path collective)
# ----------------------------------------------------------------------------
def dist_init(args=None):
    """One process per GPU (torchrun environment): NCCL with GPUs, gloo on a
    CPU-only host.  Replicas only: the process group carries the barrier and
    the max-over-ranks timing, never data-path traffic."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index, self.samples, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 6:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return None
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
def decode_shapes():
    import paper_2305_17105_gb300 as ntc
    return ntc.pyramid(DEC_SIDE, DEC_SIDE)


def make_random_decode_material(precision, device="cuda"):
    """4096^2 x 16 material: random 4-bit grids (packed on the device by the
    library's quantiser) and random MLP weights of the requested precision.
    Returns (Material, host float grid values, host weights)."""
    import torch
    import paper_2305_17105_gb300 as ntc
    rng = np.random.default_rng(1001)
    n, q = 16, 1.0 / 16
    lo, hi = -(n - 1) / 2 * q, n / 2 * q
    g0h, g1h, g0, g1 = [], [], [], []
    for (w0, h0), (w1, h1) in decode_shapes():
        a = gen.uniform_grid_values((h0, w0, DEC_C0), lo, hi, rng)
        b = gen.uniform_grid_values((h1, w1, DEC_C0), lo, hi, rng)
        g0h.append(a)
        g1h.append(b)
        for src, dst in ((a, g0), (b, g1)):
            t = torch.from_numpy(src).to(device)
            p = ntc.ntc_quantize_pack(t, DEC_C0, 4, q)
            dst.append(p.view(src.shape[0], src.shape[1], -1))
    w = gen.random_mlp(DEC_K, 64, DEC_C, seed=2001, n_used=2 * DEC_C0 + 13)
    dev_w = [torch.from_numpy(w[l]).to(device).to(
        torch.float32 if precision == "f32" else torch.float16) for l in (0, 2, 4)]
    dev_b = [torch.from_numpy(w[l]).to(device) for l in (1, 3, 5)]
    mat = ntc.Material(DEC_SIDE, DEC_SIDE, DEC_C, DEC_C0, DEC_C0, 4, 4, q, q, g0, g1, dev_w, dev_b,
                       DEC_K, ntc.PREC_F32 if precision == "f32" else ntc.PREC_F16)
    if precision == "f8":
        calib = torch.from_numpy(gen.random_queries(1 << 16, 13, seed=4999)).to(device)
        mat = ntc.f8_material(mat, [w[0], w[2], w[4]], calib)
    return mat, (g0h, g1h), w


def make_decode_material(precision, train_steps, batch, device="cuda"):
    """The 4096^2 x 16 decode material compressed by the library's own trainer:
    a synthetic 16-channel texture set (seed 1001), grids G0 1024^2 x 12 and
    G1 512^2 x 12 (4-bit range) and an MLP 48-64-64-16 trained for
    `train_steps` FP16 tensor-core steps of `batch` texels (seed 1004), then
    exported with 4-bit packed grids.  Returns the material in the requested
    precision (FP8: per-layer scales from ntc_f8_quantize_weights and
    ntc_f8_activation_scales), the host grid values, the FP32 master
    weights (layer order, with biases), the 8-bit mip chain and a summary."""
    import torch
    import paper_2305_17105_gb300 as ntc
    if train_steps <= 0:
        mat, gh, w = make_random_decode_material(precision, device)
        return mat, gh, w, None, {"trained": False}, None
    t0 = time.perf_counter()
    tex = gen.synthetic_texture(DEC_SIDE, DEC_SIDE, DEC_C, seed=1001)
    chain = gen.box_mip_chain_u8(tex)
    del tex
    t_gen = time.perf_counter() - t0
    rng = np.random.default_rng(1001)
    n, q = 16, 1.0 / 16
    lo, hi = -(n - 1) / 2 * q, n / 2 * q
    g0, g1 = [], []
    for (w0, h0), (w1, h1) in decode_shapes():
        g0.append(gen.uniform_grid_values((h0, w0, DEC_C0), lo, hi, rng))
        g1.append(gen.uniform_grid_values((h1, w1, DEC_C0), lo, hi, rng))
    w = gen.random_mlp(DEC_K, 64, DEC_C, seed=2001, n_used=2 * DEC_C0 + 13)
    tr = ntc.Trainer(DEC_SIDE, DEC_SIDE, DEC_C, DEC_C0, DEC_C0, 4, 4, q, q, g0, g1,
                     [w[0], w[2], w[4]], [w[1], w[3], w[5]], DEC_K, ntc.PREC_F16,
                     total_steps=train_steps, device=device)
    target = ntc.Target(chain, device=device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(train_steps):
        ntc.ntc_train_step(tr, target, batch, 1004)
    loss = float(tr.loss.item())
    t_train = time.perf_counter() - t0
    m16 = tr.export(ntc.PREC_F16)
    w32 = [x.detach().cpu().numpy().astype(np.float32) for x in tr.w_master]
    b32 = [x.detach().cpu().numpy().astype(np.float32) for x in tr.b]
    w_host = [w32[0], b32[0], w32[1], b32[1], w32[2], b32[2]]
    grids_host = ([g.cpu().numpy() for g in tr.material.grids0],
                  [g.cpu().numpy() for g in tr.material.grids1])
    calib = torch.from_numpy(gen.random_queries(1 << 16, 13, seed=4999)).to(device)
    forms = {"f16": m16, "f32": tr.export(ntc.PREC_F32), "f8": ntc.f8_material(m16, w32, calib)}
    mat = forms[precision]
    # texture quality of the export: every texel of mip 0 against the reference
    ys, xs = np.meshgrid(np.arange(DEC_SIDE), np.arange(DEC_SIDE), indexing="ij")
    t0q = np.stack([(xs + 0.5) / DEC_SIDE, (ys + 0.5) / DEC_SIDE, np.zeros_like(xs, float)],
                   -1).reshape(-1, 3).astype(np.float32)
    dec = ntc.ntc_decode(m16, torch.from_numpy(t0q).to(device))
    refm = torch.from_numpy(chain[0].reshape(-1, DEC_C)).to(device).float() / 255.0
    mse = float(((dec - refm) ** 2).mean())
    info = {"trained": True, "steps": train_steps, "batch": batch, "final_loss": loss,
            "train_s": t_train, "texture_gen_s": t_gen,
            "texture_psnr_mip0_db_f16": 10 * math.log10(1.0 / mse) if mse > 0 else None}
    del tr, target, dec, refm
    torch.cuda.empty_cache()
    return mat, grids_host, w_host, chain, info, forms


def make_trainer(precision, total_steps, device="cuda", k_in=TRN_K):
    import paper_2305_17105_gb300 as ntc
    tex = gen.synthetic_texture(TRN_SIDE, TRN_SIDE, TRN_C, seed=1002)
    chain = gen.box_mip_chain_u8(tex)
    rng = np.random.default_rng(1003)
    n, q = 16, 1.0 / 16
    lo, hi = -(n - 1) / 2 * q, n / 2 * q
    g0, g1 = [], []
    for (w0, h0), (w1, h1) in ntc.pyramid(TRN_SIDE, TRN_SIDE):
        g0.append(gen.uniform_grid_values((h0, w0, TRN_C0), lo, hi, rng))
        g1.append(gen.uniform_grid_values((h1, w1, TRN_C0), lo, hi, rng))
    w = gen.random_mlp(k_in, 64, TRN_C, seed=2002, n_used=2 * TRN_C0 + 13)
    prec = {"f32": ntc.PREC_F32, "f16": ntc.PREC_F16, "f8": ntc.PREC_F8}[precision]
    tr = ntc.Trainer(TRN_SIDE, TRN_SIDE, TRN_C, TRN_C0, TRN_C0, 4, 4, q, q, g0, g1,
                     [w[0], w[2], w[4]], [w[1], w[3], w[5]], k_in, prec,
                     total_steps=total_steps, device=device,
                     f8_act_scales=[1.0 / 256, 1.0 / 64, 1.0 / 64] if precision == "f8" else None)
    return tr, ntc.Target(chain, device=device), chain, (g0, g1), w


# ----------------------------------------------------------------------------
# Render-like decode of a trained model (camera frame, trilinear filtering)
# ----------------------------------------------------------------------------
def render_eval(ntc, forms, grids_host, w_host, stream, stride=127):
    """The camera workload on the trained 4096^2 x 16 decode material: a
    3840x2160 frame with trilinear filtering (8 decodes per pixel) in FP16,
    FP8-E4M3 and FP32.  Reports frame times and, for each precision, the
    PSNR against the FP64 oracle with the FP32 master weights (every
    `stride`-th pixel), plus stochastic filtering (one decode per pixel)."""
    import torch
    import oracle
    mips = ntc.mips_of(DEC_SIDE, DEC_SIDE)
    q = gen.camera_queries(3840, 2160, DEC_SIDE, mips)
    uvl = torch.from_numpy(q).cuda()
    res = {"workload": f"3840x2160 camera frame over the trained {DEC_SIDE}^2x{DEC_C} material "
                       "(plane pitched 60 deg, 90 deg FoV), trilinear: 8 decodes per pixel",
           "pixels": int(q.shape[0])}
    frames = {}
    for name in ("f16", "f8", "f32"):
        m = forms[name]
        o = torch.empty((q.shape[0], DEC_C), dtype=torch.float32, device="cuda")
        ntc.ntc_decode(m, uvl, out=o, filter=ntc.FILTER_TRILINEAR)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            ntc.ntc_decode(m, uvl, out=o, filter=ntc.FILTER_TRILINEAR)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 3
        res[f"frame_ms_{name}"] = ms
        res[f"decodes_per_s_{name}"] = 8 * q.shape[0] / (ms / 1e3)
        frames[name] = o

    def psnr(x, y):
        mse = float(np.mean((np.asarray(x, np.float64) - np.asarray(y, np.float64)) ** 2))
        return float("inf") if mse == 0 else 10 * math.log10(1.0 / mse)

    # the FP64 oracle of the same model (4-bit grids, FP32 master weights) on
    # a pixel subset: the total precision loss of each form
    md = oracle_decoder(grids_host, [np.asarray(x, np.float64) for x in w_host])
    idx = np.arange(0, q.shape[0], stride)
    t0 = time.perf_counter()
    ref = md.decode_trilinear(q[idx])
    res["oracle_pixels"] = int(idx.size)
    res["oracle_s"] = time.perf_counter() - t0
    sel = torch.from_numpy(idx).cuda()
    res["psnr_vs_fp64_oracle_db"] = {k: psnr(frames[k][sel].cpu().numpy(), ref)
                                     for k in ("f32", "f16", "f8")}
    res["max_abs_vs_fp64_oracle"] = {
        k: float(np.abs(frames[k][sel].cpu().numpy() - ref).max()) for k in ("f32", "f16", "f8")}
    # stochastic filtering (Sec. 5.3): one jittered nearest decode per pixel
    o = torch.empty((q.shape[0], DEC_C), dtype=torch.float32, device="cuda")

    def stoch(frame=[0]):
        frame[0] += 1
        ntc.ntc_decode(forms["f16"], uvl, out=o, filter=ntc.FILTER_STOCHASTIC, noise_seed=9,
                       noise_step=frame[0])
    stoch()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(5):
        stoch()
    b.record(stream)
    torch.cuda.synchronize()
    res["frame_ms_stochastic_f16"] = a.elapsed_time(b) / 5
    res["psnr_stochastic_frame_vs_trilinear_db"] = psnr(o.cpu().numpy(),
                                                        frames["f16"].cpu().numpy())
    return res


def equal_psnr_eval(ntc, chain, batch, seed, stream, steps=1500):
    """Training precision at equal steps: the training material compressed
    twice from the same initialisation and samples, once with the FP16
    tensor-core step and once with the FP32 CUDA-core step, `steps` steps
    each; both exports (4-bit grids) decoded in the FP32 form at every texel
    of mip 0 and compared with the 8-bit reference (PSNR), with the time of
    each training run."""
    import torch
    ys, xs = np.meshgrid(np.arange(TRN_SIDE), np.arange(TRN_SIDE), indexing="ij")
    t0 = torch.from_numpy(np.stack([(xs + 0.5) / TRN_SIDE, (ys + 0.5) / TRN_SIDE,
                                    np.zeros_like(xs, float)], -1).reshape(-1, 3)
                          .astype(np.float32)).cuda()
    refm = torch.from_numpy(chain[0].reshape(-1, TRN_C).astype(np.float32) / 255.0).cuda()
    res = {"workload": f"{TRN_SIDE}^2x{TRN_C} material, {steps} steps of {batch} texels from the "
                       "same initialisation and samples; PSNR of mip 0 of the 4-bit export "
                       "(decoded in FP32) against the 8-bit reference", "steps": steps}
    # f16 / f32: K = 48; f8 needs K in steps of 32, so it runs against its own
    # FP16 twin at K = 64 (zero columns; the same initialisation for both)
    for prec, arm, k in (("f16", "f16", TRN_K), ("f32", "f32", TRN_K), ("f16", "f16_k64", 64),
                         ("f8", "f8", 64)):
        tr, target, _, _, _ = make_trainer(prec, steps, k_in=k)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            ntc.ntc_train_step(tr, target, batch, seed)
        b.record(stream)
        torch.cuda.synchronize()
        dec = ntc.ntc_decode(tr.export(ntc.PREC_F32), t0)
        mse = float(((dec - refm) ** 2).mean())
        res[f"train_s_{arm}"] = a.elapsed_time(b) / 1e3
        res[f"psnr_db_{arm}_trained"] = 10 * math.log10(1.0 / mse)
        res[f"status_{arm}"] = ntc.ntc_device_status()
        del tr, target
    res["delta_db"] = res["psnr_db_f16_trained"] - res["psnr_db_f32_trained"]
    res["speedup_f16_over_f32"] = res["train_s_f32"] / res["train_s_f16"]
    res["delta_db_f8_minus_f16_k64"] = res["psnr_db_f8_trained"] - res["psnr_db_f16_k64_trained"]
    res["speedup_f8_over_f16_k64"] = res["train_s_f16_k64"] / res["train_s_f8"]
    res["f8_samples_per_s"] = steps * batch / res["train_s_f8"]
    res["f16_k64_samples_per_s"] = steps * batch / res["train_s_f16_k64"]
    return res


# ----------------------------------------------------------------------------
# The paper's decoder form: learned interpolation of G0, hardGELU, identity
# ----------------------------------------------------------------------------
def paper_form_eval(ntc, q_dev, batch, stream, hidden_layers=2):
    """Decode of the 2^24 queries with the paper's own decoder input (Sec.
    4.3.1, 4.4: the four G0 taps concatenated, 4 c0 + c1 + 13 inputs,
    hardGELU, no output activation) on a 4096^2 x 16 material with the NTC
    2.25 profile's grids (G0 1024^2 x 16 at 4 bits, G1 512^2 x 12 at 4 bits),
    random weights, FP16 tensor cores, `hidden_layers` hidden layers of 64;
    then the training step of the same decoder form (paper_form_train)."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(7007)
    c0, c1, k = 16, 12, 96
    cb0, cb1 = ntc.cell_bytes(c0, 4), ntc.cell_bytes(c1, 4)
    levels = ntc.ntc_pyramid(DEC_SIDE, DEC_SIDE)
    g0 = [torch.randint(0, 256, (h0, w0, cb0), dtype=torch.uint8, device="cuda", generator=g)
          for (w0, h0), _ in levels]
    g1 = [torch.randint(0, 256, (h1, w1, cb1), dtype=torch.uint8, device="cuda", generator=g)
          for _, (w1, h1) in levels]
    w = gen.random_mlp(k, 64, DEC_C, seed=7008, n_used=4 * c0 + c1 + 13,
                       hidden_layers=hidden_layers)
    mat = ntc.Material(DEC_SIDE, DEC_SIDE, DEC_C, c0, c1, 4, 4, 1 / 16, 1 / 16, g0, g1,
                       [torch.from_numpy(x).cuda().half() for x in w[0::2]],
                       [torch.from_numpy(x).cuda() for x in w[1::2]], k, ntc.PREC_F16,
                       act=ntc.ACT_HARDGELU, out_act=ntc.OUT_IDENTITY, interp0=1)
    out = torch.empty((q_dev.shape[0], DEC_C), dtype=torch.float16, device="cuda")
    ntc.ntc_decode(mat, q_dev, out=out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(5):
        ntc.ntc_decode(mat, q_dev, out=out)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 5
    flop = 2 * (k * 64 + (hidden_layers - 1) * 64 * 64 + 64 * DEC_C)
    mlp = "-".join(["96"] + ["64"] * hidden_layers + ["16"])
    res = {"workload": "4096^2x16, G0 1024^2x16 (learned interpolation: 4 taps concatenated) + "
                       f"G1 512^2x12 at 4 bits, MLP {mlp} hardGELU/identity, 2^24 random queries",
           "decode_ms": ms, "texels_per_s": q_dev.shape[0] / (ms / 1e3),
           "tflops": flop * q_dev.shape[0] / (ms / 1e3) / 1e12, "status": ntc.ntc_device_status()}
    res["train"] = paper_form_train(ntc, batch, stream, hidden_layers=hidden_layers)
    if hidden_layers == 2:
        res["three_hidden_layers"] = paper_form_eval(ntc, q_dev, batch, stream, hidden_layers=3)
    return res


def paper_form_train(ntc, batch, stream, steps=20, hidden_layers=2):
    """Training step of the paper-form decoder (learned G0 interpolation,
    hardGELU, identity output) on a 2048^2 x 12 material with the NTC 2.25
    profile's grids (G0 512^2 x 16, G1 256^2 x 12, FP32 values in the 4-bit
    range), MLP 96-64-64(-64)-12, FP16 tensor-core step with noise, `batch`
    sampled texels per step."""
    import torch
    side, c, c0, c1, k = TRN_SIDE, TRN_C, 16, 12, 96
    tex = gen.synthetic_texture(side, side, c, seed=1102)
    chain = gen.box_mip_chain_u8(tex)
    rng = np.random.default_rng(1103)
    n, q = 16, 1.0 / 16
    lo, hi = -(n - 1) / 2 * q, n / 2 * q
    g0, g1 = [], []
    for (w0, h0), (w1, h1) in ntc.pyramid(side, side):
        g0.append(gen.uniform_grid_values((h0, w0, c0), lo, hi, rng))
        g1.append(gen.uniform_grid_values((h1, w1, c1), lo, hi, rng))
    w = gen.random_mlp(k, 64, c, seed=1104, n_used=4 * c0 + c1 + 13, hidden_layers=hidden_layers)
    tr = ntc.Trainer(side, side, c, c0, c1, 4, 4, q, q, g0, g1, w[0::2], w[1::2], k,
                     ntc.PREC_F16, act=ntc.ACT_HARDGELU, out_act=ntc.OUT_IDENTITY,
                     total_steps=steps + 3, interp0=ntc.INTERP_LEARNED)
    target = ntc.Target(chain)
    for _ in range(3):
        ntc.ntc_train_step(tr, target, batch, 5)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        ntc.ntc_train_step(tr, target, batch, 5)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    mlp = "-".join(["96"] + ["64"] * hidden_layers + ["12"])
    return {"workload": f"2048^2x12, G0 512^2x16 (learned interpolation) + G1 256^2x12, "
                        f"MLP {mlp} hardGELU/identity, {batch} texels per step",
            "train_ms": ms, "samples_per_s": batch / (ms / 1e3), "loss": float(tr.loss.item()),
            "status": ntc.ntc_device_status()}


def u8_output_eval(ntc, mat, q_dev, q_host, stream, reps=5):
    """The same decode with 8-bit UNORM outputs: on the device (inputs
    resident) and end to end through ntc_decode_host (pinned host buffers,
    chunks of 2^20 queries)."""
    import torch
    n = q_dev.shape[0]
    out = torch.empty((n, DEC_C), dtype=torch.uint8, device="cuda")
    out_host = torch.empty((n, DEC_C), dtype=torch.uint8).pin_memory()
    chunk = min(1 << 20, n)
    ws = torch.empty(ntc.lib().ntc_decode_host_workspace_bytes(DEC_C, ntc.DTYPE_U8, chunk),
                     dtype=torch.uint8, device="cuda")
    res = {}
    for name, fn in (("device", lambda: ntc.ntc_decode(mat, q_dev, out=out)),
                     ("e2e", lambda: ntc.ntc_decode_host(mat, q_host, out_host=out_host,
                                                         workspace=ws))):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        res[name + "_ms"] = ms
        res[name + "_texels_per_s"] = n / (ms / 1e3)
    res["bytes_per_query"] = 12 + DEC_C
    res["h2d_bytes_per_step"], res["d2h_bytes_per_step"] = n * 12, n * DEC_C
    res["status"] = ntc.ntc_device_status()
    return res


def vq_eval(ntc, q_dev, stream):
    """Decode of the 2^24 queries with a vector-quantised G0 (the paper's
    VQ-8: two 256-entry codebooks of 8 values, two 8-bit indices per cell,
    features = the sum of the two entries) on the 4096^2 x 16 material, G0
    1024^2 (16 bits per cell) + G1 512^2 x 12 at 4 bits, MLP 48-64-64-16,
    FP16 tensor cores, random indices, codebooks and weights."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(7107)
    books, c0, c1, k = 2, 8, 12, 48
    levels = ntc.ntc_pyramid(DEC_SIDE, DEC_SIDE)
    g0 = [torch.randint(0, 256, (h0, w0, books), dtype=torch.uint8, device="cuda", generator=g)
          for (w0, h0), _ in levels]
    g1 = [torch.randint(0, 256, (h1, w1, ntc.cell_bytes(c1, 4)), dtype=torch.uint8, device="cuda",
                        generator=g) for _, (w1, h1) in levels]
    cb = (torch.rand((books, 256, c0), device="cuda", generator=g) - 0.5) * 0.5
    w = gen.random_mlp(k, 64, DEC_C, seed=7108, n_used=c0 + c1 + 13)
    mat = ntc.Material(DEC_SIDE, DEC_SIDE, DEC_C, c0, c1, 8, 4, 1 / 16, 1 / 16, g0, g1,
                       [torch.from_numpy(x).cuda().half() for x in w[0::2]],
                       [torch.from_numpy(x).cuda() for x in w[1::2]], k, ntc.PREC_F16,
                       codebook0=cb.contiguous())
    out = torch.empty((q_dev.shape[0], DEC_C), dtype=torch.float16, device="cuda")
    ntc.ntc_decode(mat, q_dev, out=out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(5):
        ntc.ntc_decode(mat, q_dev, out=out)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 5
    return {"workload": "4096^2x16, G0 1024^2 VQ-8 (2 codebooks x 256 x 8, 16 bits per cell) + "
                        "G1 512^2x12 at 4 bits, MLP 48-64-64-16, 2^24 random queries",
            "decode_ms": ms, "texels_per_s": q_dev.shape[0] / (ms / 1e3),
            "status": ntc.ntc_device_status()}


def sq_vq_train_eval(ntc, chain, batch, seed, stream, steps=1000):
    """The appendix comparison of scalar and vector quantisation on the
    synthetic training material (2048^2 x 12): G0 at 16 bits per cell as
    SQ-8 (8 channels x 2 bits) or VQ-8 (two 256-entry codebooks of 8 values,
    VQ-VAE terms, commitment 0.25), G1 256^2 x 12 at 4 bits, MLP with 48
    inputs, FP16 step, `steps` steps of `batch` texels from the
    same initialisation; PSNR of mip 0 of the export (decoded in FP16)
    against the 8-bit reference, and the training time."""
    import torch
    side, c, c0, c1, k = TRN_SIDE, TRN_C, 8, 12, 48
    rng = np.random.default_rng(1203)
    levels = ntc.pyramid(side, side)
    ys, xs = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    t0 = torch.from_numpy(np.stack([(xs + 0.5) / side, (ys + 0.5) / side, np.zeros_like(xs, float)],
                                   -1).reshape(-1, 3).astype(np.float32)).cuda()
    refm = torch.from_numpy(chain[0].reshape(-1, c).astype(np.float32) / 255.0).cuda()
    g1 = [gen.uniform_grid_values((h1, w1, c1), -7 / 16, 8 / 16, rng) for _, (w1, h1) in levels]
    w = gen.random_mlp(k, 64, c, seed=1204, n_used=c0 + c1 + 13)
    cb = rng.uniform(-0.5, 0.5, (2, 256, c0)).astype(np.float32)
    cb[1] *= 0.25
    res = {"workload": f"{side}^2x{c}, G0 at 16 bits per cell (SQ-8: 8 x 2 bits; VQ-8: 2 x 256 x 8 "
                       f"codebooks) + G1 at 4 bits, MLP 48-64-64-{c}, {steps} steps of {batch} "
                       "texels, FP16 step", "steps": steps}
    target = ntc.Target(chain)
    for name in ("sq", "vq"):
        if name == "sq":  # 2-bit levels k Q, Q = 1/2: clamp range [-3/4, 1]
            g0 = [gen.uniform_grid_values((h0, w0, c0), -0.75, 1.0, rng) for (w0, h0), _ in levels]
            tr = ntc.Trainer(side, side, c, c0, c1, 2, 4, 0.5, 1 / 16, g0, g1, w[0::2], w[1::2], k,
                             ntc.PREC_F16, total_steps=steps)
        else:
            g0 = [gen.uniform_grid_values((h0, w0, c0), -0.5, 0.5, rng) for (w0, h0), _ in levels]
            tr = ntc.Trainer(side, side, c, c0, c1, 8, 4, 1 / 16, 1 / 16, g0, g1, w[0::2], w[1::2],
                             k, ntc.PREC_F16, total_steps=steps, codebook0=cb, vq_beta=0.25)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            ntc.ntc_train_step(tr, target, batch, seed)
        b.record(stream)
        torch.cuda.synchronize()
        dec = ntc.ntc_decode(tr.export(ntc.PREC_F16), t0)
        mse = float(((dec - refm) ** 2).mean())
        res[f"train_s_{name}"] = a.elapsed_time(b) / 1e3
        res[f"psnr_db_{name}"] = 10 * math.log10(1.0 / mse)
        res[f"status_{name}"] = ntc.ntc_device_status()
        del tr
    res["psnr_delta_db_vq_minus_sq"] = res["psnr_db_vq"] - res["psnr_db_sq"]
    res["train_time_ratio_vq_over_sq"] = res["train_s_vq"] / res["train_s_sq"]
    return res


# ----------------------------------------------------------------------------
# Many materials: batched decode launch, graph-captured training of all of them
# ----------------------------------------------------------------------------
def multi_material_eval(ntc, n_mat, q_per, train_batch, stream):
    """The multi-material workload: n_mat square materials (side 2^k, k
    uniform over 8..12; C uniform over {8, 12, 16}; G0 = side/4 and G1 =
    side/8 with 12 channels each at 4 bits; random grids and MLPs), q_per
    random queries each.  Decode: one persistent batched launch against one
    launch per material.  Training: one step of train_batch texels for every
    material (FP32 state, FP16 tensor-core step), captured once as a CUDA
    graph and replayed."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(5005)
    shapes = gen.material_set_shapes(n_mat, seed=5000)
    q = 1.0 / 16
    cb = ntc.cell_bytes(12, 4)
    mats, uvls = [], []
    for i, (side, c) in enumerate(shapes):
        levels = ntc.ntc_pyramid(side, side)
        g0 = [torch.randint(0, 256, (h0, w0, cb), dtype=torch.uint8, device="cuda", generator=g)
              for (w0, h0), _ in levels]
        g1 = [torch.randint(0, 256, (h1, w1, cb), dtype=torch.uint8, device="cuda", generator=g)
              for _, (w1, h1) in levels]
        w = gen.random_mlp(48, 64, c, seed=6000 + i, n_used=2 * 12 + 13)
        wd = [torch.from_numpy(w[l]).cuda().half() for l in (0, 2, 4)]
        bd = [torch.from_numpy(w[l]).cuda() for l in (1, 3, 5)]
        mats.append(ntc.Material(side, side, c, 12, 12, 4, 4, q, q, g0, g1, wd, bd, 48, ntc.PREC_F16))
        mips = ntc.mips_of(side, side)
        uv = torch.rand((q_per, 2), generator=g, device="cuda")
        lod = torch.randint(0, mips, (q_per, 1), generator=g, device="cuda").float()
        uvls.append(torch.cat([uv, lod], 1).contiguous())
    uvl = torch.cat(uvls)
    res = {"workload": f"{n_mat} materials (sides 256-4096, C in {{8,12,16}}, G0 side/4 and G1 side/8 "
                       f"x 12 ch at 4 bits), {q_per} random queries each; one training step of "
                       f"{train_batch} texels per material",
           "sides": [s for s, _ in shapes], "channels": [c for _, c in shapes]}

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    batch = ntc.Batch(mats, [q_per] * n_mat)
    out = torch.empty(int(batch.desc.total_outputs), dtype=torch.float16, device="cuda")
    ms_b = timed(lambda: ntc.ntc_decode_batched(batch, uvl, out=out))
    outs = [torch.empty((q_per, m.channels), dtype=torch.float16, device="cuda") for m in mats]

    def separate():
        for m, u, o in zip(mats, uvls, outs):
            ntc.ntc_decode(m, u, out=o)
    ms_s = timed(separate)
    res["decode_batched_ms"] = ms_b
    res["decode_batched_texels_per_s"] = n_mat * q_per / (ms_b / 1e3)
    res["decode_per_material_launches_ms"] = ms_s
    res["decode_per_material_texels_per_s"] = n_mat * q_per / (ms_s / 1e3)
    del out, outs, uvl, uvls, batch

    trainers, targets = [], []
    lo, hi = -(16 - 1) / 2 * q, 16 / 2 * q
    for i, (side, c) in enumerate(shapes):
        levels = ntc.ntc_pyramid(side, side)
        z0 = [np.zeros((h0, w0, 12), np.float32) for (w0, h0), _ in levels]
        z1 = [np.zeros((h1, w1, 12), np.float32) for _, (w1, h1) in levels]
        w = gen.random_mlp(48, 64, c, seed=6000 + i, n_used=2 * 12 + 13)
        tr = ntc.Trainer(side, side, c, 12, 12, 4, 4, q, q, z0, z1, [w[0], w[2], w[4]],
                         [w[1], w[3], w[5]], 48, ntc.PREC_F16, total_steps=1000)
        for t in tr.material.grids0 + tr.material.grids1:
            t.uniform_(lo, hi, generator=g)
        tg = ntc.Target.__new__(ntc.Target)
        offs, n = [], 0
        for m in range(ntc.mips_of(side, side)):
            offs.append(n)
            n += (max(1, side >> m) ** 2 * c + 15) // 16 * 16
        tg.texels = torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda", generator=g)
        tg.offsets = offs
        trainers.append(tr)
        targets.append(tg)

    def capture(fn):
        fn()  # warm-up outside the capture
        torch.cuda.synchronize()
        side_stream = torch.cuda.Stream()
        side_stream.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side_stream):
            with torch.cuda.graph(graph, stream=side_stream):
                fn(side_stream)
        torch.cuda.current_stream().wait_stream(side_stream)
        return graph

    # every material's step in one batched call: noise pass, one persistent
    # fused fwd+bwd launch, one Adam launch (its last block advances the step
    # counters), captured as a CUDA graph
    tb = ntc.TrainBatch(trainers, targets, [train_batch] * n_mat, 55)
    g_b = capture(lambda st=None: ntc.ntc_train_step_batched(tb, stream=st))
    ms_t = timed(g_b.replay, reps=5)
    n_params = sum(tr.params.numel() for tr in trainers)
    algo = n_mat * train_batch * 1036 + n_params * 32
    res["train_batched_graph_step_ms"] = ms_t
    res["train_samples_per_s"] = n_mat * train_batch / (ms_t / 1e3)
    # the whole compression schedule of the workload: 1,000 steps of every
    # material, one graph replay each
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(1000):
        g_b.replay()
    b.record(stream)
    torch.cuda.synchronize()
    res["train_1000_steps_s"] = a.elapsed_time(b) / 1e3
    res["train_1000_steps_samples_per_s"] = 1000 * n_mat * train_batch / res["train_1000_steps_s"]
    res["train_final_loss_mean"] = float(tb.loss.mean().item())
    res["train_kernels_per_step"] = 3
    res["train_params"] = n_params
    res["train_algorithmic_bytes_per_step"] = algo
    res["train_hbm_gbs_algorithmic"] = algo / (ms_t / 1e3) / 1e9
    # for comparison: one ntc_train_step per material (5 kernels each), the
    # same steps captured in one graph
    g_s = capture(lambda st=None: [ntc.ntc_train_step(tr, tg, train_batch, 55, stream=st)
                                   for tr, tg in zip(trainers, targets)])
    ms_s = timed(g_s.replay, reps=5)
    res["train_per_material_graph_step_ms"] = ms_s
    res["train_per_material_kernels_per_step"] = 5 * n_mat
    res["status"] = ntc.ntc_device_status()
    return res


# ----------------------------------------------------------------------------
# Measured peaks of the reduced and widened precision forms
# ----------------------------------------------------------------------------
def fp8_gemm_tflops(n=8192, reps=10):
    """Dense FP8-E4M3 GEMM throughput (TFLOP/s, best of `reps`): the library
    GEMM behind torch._scaled_mm on n^3 operands, scales 1, BF16 output."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    a = (torch.randn(n, n, device="cuda", generator=g) * 0.5).to(torch.float8_e4m3fn)
    b = (torch.randn(n, n, device="cuda", generator=g) * 0.5).to(torch.float8_e4m3fn)
    one = torch.ones((), device="cuda", dtype=torch.float32)

    def f():
        return torch._scaled_mm(a, b.t(), scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
    for _ in range(3):
        f()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        f()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 2.0 * n ** 3 / (best / 1e3) / 1e12


def measured_peaks(ntc):
    out = {}
    try:
        out["fp32_fma_tflops"] = ntc.ntc_probe_fma_tflops()
        out["fp32_fma_source"] = "ntc_probe_fma_tflops: 16 independent FMA chains per thread, best of 5"
    except Exception as e:  # reported, never fatal
        out["fp32_fma_error"] = f"{type(e).__name__}: {e}"[:200]
    try:
        out["fp8_tflops"] = fp8_gemm_tflops()
        out["fp8_source"] = "torch._scaled_mm E4M3 8192^3, BF16 out, best of 10 (burst)"
    except Exception as e:  # reported, never fatal
        out["fp8_error"] = f"{type(e).__name__}: {e}"[:200]
    return out


# ----------------------------------------------------------------------------
# CPU oracle baseline (bounded samples)
# ----------------------------------------------------------------------------
def oracle_decoder(grids_host, weights):
    """The FP64 oracle's model of the decode material (4-bit grids)."""
    import oracle
    q = 1.0 / 16
    g0 = [oracle.dequantize(oracle.quantize(a.astype(np.float64), 16, q), 16, q)
          for a in grids_host[0]]
    g1 = [oracle.dequantize(oracle.quantize(a.astype(np.float64), 16, q), 16, q)
          for a in grids_host[1]]
    return oracle.Model(DEC_SIDE, DEC_SIDE, DEC_C, DEC_C0, DEC_C0, 16, 16, q, q, g0, g1, weights,
                        DEC_K)


def oracle_decode_rate(grids_host, weights, queries, seconds):
    """Decoded texels/s of the FP64 oracle on the host cores, on a prefix of
    the decode workload sized to about `seconds` of work."""
    import oracle
    md = oracle_decoder(grids_host, weights)
    threads = oracle.default_threads()
    n = 4096
    t0 = time.perf_counter()
    md.decode(queries[:n], threads=threads)
    dt = time.perf_counter() - t0
    n = int(min(len(queries), max(n, n * seconds / max(dt, 1e-6))))
    t0 = time.perf_counter()
    md.decode(queries[:n], threads=threads)
    dt = time.perf_counter() - t0
    return n / dt, n, threads, dt


def oracle_train_rate(chain, grids_host, weights, batch, seconds):
    import oracle
    q = 1.0 / 16
    md = oracle.Model(TRN_SIDE, TRN_SIDE, TRN_C, TRN_C0, TRN_C0, 16, 16, q, q,
                      [g.astype(np.float64) for g in grids_host[0]],
                      [g.astype(np.float64) for g in grids_host[1]], weights, TRN_K)
    threads = min(oracle.default_threads(), 8)  # one private FP64 gradient copy per thread
    n = 2048
    xym = oracle.sample_batch(7, 0, batch, TRN_SIDE, TRN_SIDE, md.mips)
    t = oracle.targets_of_xym(chain, xym)
    t0 = time.perf_counter()
    md.loss_grad_xym(xym[:n], t[:n], noise=(7, 0), threads=threads)
    dt = time.perf_counter() - t0
    n = int(min(batch, max(n, n * seconds / max(dt, 1e-6))))
    t0 = time.perf_counter()
    md.loss_grad_xym(xym[:n], t[:n], noise=(7, 0), threads=threads)
    dt = time.perf_counter() - t0
    return n / dt, n, threads, dt


# ----------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # the oracle needs the material only; build it on the host
    rng = np.random.default_rng(1001)
    n, q = 16, 1.0 / 16
    lo, hi = -(n - 1) / 2 * q, n / 2 * q
    import oracle
    g0, g1 = [], []
    for (w0, h0), (w1, h1) in oracle.pyramid(DEC_SIDE, DEC_SIDE):
        g0.append(gen.uniform_grid_values((h0, w0, DEC_C0), lo, hi, rng))
        g1.append(gen.uniform_grid_values((h1, w1, DEC_C0), lo, hi, rng))
    w = gen.random_mlp(DEC_K, 64, DEC_C, seed=2001, n_used=2 * DEC_C0 + 13)
    queries = gen.random_queries(args.queries, 13, seed=4001)
    md = oracle_decoder((g0, g1), w)
    threads = oracle.default_threads()
    # one step = a bounded slice of the workload, sized so that the whole run
    # takes about `budget` seconds of host time
    budget = max(10.0, min(120.0, 15.0 * args.cpu_seconds))
    t0 = time.perf_counter()
    md.decode(queries[:4096], threads=threads)
    rate0 = 4096 / max(time.perf_counter() - t0, 1e-6)
    ns = int(min(len(queries), max(1024, rate0 * budget / (args.warmup + args.steps))))
    times, rates = [], []
    for i in range(args.warmup + args.steps):
        off = (i * ns) % max(1, len(queries) - ns + 1)
        t0 = time.perf_counter()
        md.decode(queries[off:off + ns], threads=threads)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            rates.append(ns / dt)
            times.append(dt)
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "texels/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "decode 4096^2x16 material, 2^24 random (u,v,lod) queries "
                                   "(bounded prefix per step)", "queries_per_step": ns},
            "cpu_baseline": {"value": value, "unit": "texels/s", "cores": threads, "kind": "oracle",
                             "sample": f"{ns} of the 2^24 decode queries per step (consecutive "
                                       f"slices; whole run sized to ~{budget:.0f} s of host time)"},
            "e2e": {"value": value, "unit": "texels/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import paper_2305_17105_gb300 as ntc
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    rank, world = dist_init(args)
    ntc.lib()
    precision = args.precision
    if precision == "auto":
        precision = os.environ.get("NTC_BENCH_PRECISION", "f16")
    train_prec = args.train_precision
    if train_prec == "auto":
        train_prec = "f32" if precision == "f32" else "f16"
    dev = "cuda"
    stream = torch.cuda.current_stream()

    # ---- inputs resident in HBM -------------------------------------------
    mat, grids_host, w_host, dec_chain, dec_info, forms = make_decode_material(
        precision, args.decode_train_steps, args.batch)
    queries = gen.random_queries(args.queries, 13, seed=4001 + rank)
    q_host = torch.from_numpy(queries).pin_memory()
    q_dev = q_host.to(dev)
    out = torch.empty((args.queries, DEC_C), dtype=torch.float16, device=dev)
    total = args.warmup + args.steps + 40 + CROP_STEPS + args.render_steps  # + e2e, crops, render
    tr, target, chain, tgrids, tw = make_trainer(train_prec, total)
    seed = 77 + rank

    def decode():
        ntc.ntc_decode(mat, q_dev, out=out)

    def train():
        ntc.ntc_train_step(tr, target, args.batch, seed)

    tuning = None
    if precision != "f32" and args.decode_shape:
        ntc.ntc_set_decode_warpgroups(args.decode_shape)
        tuning = {"decode_warpgroups": args.decode_shape, "ms_per_shape": None}
    elif precision != "f32":
        best, ms = ntc.ntc_autotune_decode(mat, q_dev, out)
        tuning = {"decode_warpgroups": best, "ms_per_shape": ms}
    for _ in range(args.warmup):
        decode()
        train()
    torch.cuda.synchronize()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t_wall = time.perf_counter()
        for s in range(args.steps):
            ev[s][0].record(stream)
            decode()
            ev[s][1].record(stream)
            train()
            ev[s][2].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        t_wall = time.perf_counter() - t_wall
    dec_ms = [a.elapsed_time(b) for a, b, _ in ev]
    trn_ms = [b.elapsed_time(c) for _, b, c in ev]
    step_ms = [a.elapsed_time(c) for a, _, c in ev]
    total_ms = max_over_ranks(sum(step_ms), world)
    dec_total = max_over_ranks(sum(dec_ms), world)
    trn_total = max_over_ranks(sum(trn_ms), world)
    value = world * args.queries * args.steps / (dec_total / 1e3)
    train_rate = world * args.batch * args.steps / (trn_total / 1e3)
    loss = float(tr.loss.item())

    # ---- roofline of the decode kernel (one launch per decode call) -------
    flop_per_q = 2 * (DEC_K * 64 + 64 * 64 + 64 * DEC_C)
    dec_avg_s = statistics.mean(dec_ms) / 1e3
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    mpeaks = measured_peaks(ntc)
    if precision == "f32":
        peak = mpeaks.get("fp32_fma_tflops") or 152 * 128 * 2 * MAX_SM_MHZ * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flop_per_q * args.queries / dec_avg_s / 1e12,
                "peak": peak, "unit": "TFLOP/s",
                "peak_source": ("measured FP32 FMA probe" if "fp32_fma_tflops" in mpeaks
                                else "fallback: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz")}
    elif precision == "f8":
        peak = mpeaks.get("fp8_tflops") or 2.0 * peaks.get("bf16_tflops", 1900.0)
        roof = {"bound": "tensor", "achieved": flop_per_q * args.queries / dec_avg_s / 1e12,
                "peak": peak, "unit": "TFLOP/s",
                "peak_source": ("measured FP8-E4M3 GEMM burst" if "fp8_tflops" in mpeaks
                                else "fallback: measured bf16 burst x 2 (nominal ratio)")}
    else:
        peak = peaks.get("bf16_tflops", 1900.0)
        roof = {"bound": "tensor", "achieved": flop_per_q * args.queries / dec_avg_s / 1e12,
                "peak": peak, "unit": "TFLOP/s", "peak_source": "measured bf16 burst"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # DRAM bytes per launch from the committed full-size ncu capture, when it
    # was taken on these kernel sources, this precision, shape and size
    sha = decode_sources_sha()
    ok = (DECODE_TRAFFIC is not None and DECODE_TRAFFIC[0] == sha and precision == "f16"
          and args.queries == 1 << 24 and tuning and tuning["decode_warpgroups"] == 5)
    roof["traffic"] = DECODE_TRAFFIC[1] if ok else None
    roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch "
                              "at 2^24 queries" if ok else f"no capture for sources {sha}")
    roof["traffic_unit"] = "bytes"
    dec_bytes = args.queries * (12 + DEC_C * 2)
    hbm = peaks.get("hbm_gbs", 6773.2)
    roof["hbm_gbs_algorithmic"] = dec_bytes / dec_avg_s / 1e9
    roof["hbm_frac"] = roof["hbm_gbs_algorithmic"] / hbm
    roof["kernel"] = "decode"

    # ---- roofline of the training step (HBM primary, tensor secondary) -----
    # per sample: 8 taps x 16 channels x 4 B gathered (512 B), the same
    # scatter-added (512 B), 12 B of 8-bit target; per step the dense Adam
    # pass: 32 B per parameter (p, m, v, g read; p, m, v written; g cleared)
    trn_avg_s = statistics.mean(trn_ms) / 1e3
    n_params = int(tr.params.numel())
    tbytes = args.batch * (2 * 8 * TRN_C0 * 4 + TRN_C) + n_params * 32
    tflop = args.batch * 3 * 2 * (TRN_K * 64 + 64 * 64 + 64 * TRN_C)
    hbm_peak = peaks.get("hbm_gbs", 6773.2)
    bf16_peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
    train_roof = {"bound": "hbm", "achieved": tbytes / trn_avg_s / 1e9, "peak": hbm_peak,
                  "unit": "GB/s", "frac": tbytes / trn_avg_s / 1e9 / hbm_peak,
                  "algorithmic_bytes_per_step": tbytes,
                  "tensor_tflops": tflop / trn_avg_s / 1e12,
                  "tensor_frac": tflop / trn_avg_s / 1e12 / bf16_peak,
                  "tensor_peak_source": "measured bf16 sustained",
                  "note": "the grids and their gradient largely stay in L2: HBM sees less "
                          "than the algorithmic bytes"}

    # ---- end to end through the public API with host buffers --------------
    e2e = None
    if not args.no_e2e:
        # host queries in, host texels out through ntc_decode_host: chunks of
        # 2^20 queries, copies up and down overlapped with the decode; the
        # training step (independent state) runs on a second stream, joined
        # at the end of every step
        out_host = torch.empty((args.queries, DEC_C), dtype=torch.float16).pin_memory()
        loss_host = torch.empty(1, dtype=torch.float32).pin_memory()
        chunk = min(1 << 20, args.queries)
        ws = torch.empty(ntc.lib().ntc_decode_host_workspace_bytes(DEC_C, ntc.DTYPE_F16, chunk),
                         dtype=torch.uint8, device=dev)
        ts = torch.cuda.Stream()
        ntc.ntc_decode_host(mat, q_host, out_host=out_host, workspace=ws)
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_steps = min(args.steps, 20)
        for _ in range(e2e_steps):
            ts.wait_stream(stream)
            with torch.cuda.stream(ts):
                ntc.ntc_train_step(tr, target, args.batch, seed, stream=ts)
                loss_host.copy_(tr.loss, non_blocking=True)
            ntc.ntc_decode_host(mat, q_host, out_host=out_host, workspace=ws)
            stream.wait_stream(ts)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1), world)
        e2e = {"value": world * args.queries * e2e_steps / (e2e_ms / 1e3), "unit": "texels/s",
               "h2d_bytes_per_step": int(args.queries * 12),
               "d2h_bytes_per_step": int(args.queries * DEC_C * 2 + 4),
               "path": "ntc_decode_host (pinned host buffers, chunks of 2^20 queries, copies "
                       "overlapped with the decode) + ntc_train_step on a second stream + loss "
                       "read back, joined every step"}
        # this machine's host link (plain pinned copies of the step's output and
        # inputs), which bounds the end-to-end figure
        try:
            link = {}
            for name, fn, nb in (
                    ("d2h_gbs", lambda: out_host.copy_(out, non_blocking=True), out.numel() * 2),
                    ("h2d_gbs", lambda: q_dev.copy_(q_host, non_blocking=True), q_host.numel() * 4)):
                fn()
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(3):
                    fn()
                b.record(stream)
                torch.cuda.synchronize()
                link[name] = 3 * nb / (a.elapsed_time(b) / 1e3) / 1e9
            e2e["host_link"] = link
        except Exception as e:  # reported, never fatal to the headline line
            e2e["host_link"] = {"error": f"{type(e).__name__}: {e}"[:300]}

    # ---- the paper's crop sampler on the same trainer (Sec. 5.1) ----------
    crops = None
    if not args.no_extras and not args.multi_only:
        try:
            torch.cuda.synchronize()
            c0e, c1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0e.record(stream)
            for _ in range(CROP_STEPS):
                ntc.ntc_train_step(tr, target, args.batch, seed, flags=ntc.FLAG_CROPS)
            c1e.record(stream)
            torch.cuda.synchronize()
            cms = c0e.elapsed_time(c1e) / CROP_STEPS
            crops = {"sampler": "256x256 crops of one mip per batch (Sec. 5.1)", "train_ms": cms,
                     "samples_per_s": args.batch / (cms / 1e3), "status": ntc.ntc_device_status()}
        except Exception as e:  # reported, never fatal to the headline line
            crops = {"error": f"{type(e).__name__}: {e}"[:300]}

    # ---- the plain FP32 CUDA-core form on the same inputs ------------------
    fp32 = None
    if precision != "f32" and not args.no_fp32_compare:
        fp32 = {}
        if precision == "f16":
            mat32 = forms["f32"] if forms else mat.with_(
                weights=[w.float() for w in mat.weights], precision=ntc.PREC_F32)
            for _ in range(2):
                ntc.ntc_decode(mat32, q_dev, out=out)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                ntc.ntc_decode(mat32, q_dev, out=out)
            b.record(stream)
            torch.cuda.synchronize()
            fp32["decode_texels_per_s"] = 3 * args.queries / (a.elapsed_time(b) / 1e3)
            fp32["decode_speedup"] = value / world / fp32["decode_texels_per_s"]
            fp32["decode_tflops"] = flop_per_q * fp32["decode_texels_per_s"] / 1e12
            if mpeaks.get("fp32_fma_tflops"):
                fp32["decode_alu_frac_of_measured_fma"] = (fp32["decode_tflops"]
                                                           / mpeaks["fp32_fma_tflops"])
        if train_prec != "f32":
            tr32, _, _, _, _ = make_trainer("f32", 16)
            for _ in range(2):
                ntc.ntc_train_step(tr32, target, args.batch, seed)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                ntc.ntc_train_step(tr32, target, args.batch, seed)
            b.record(stream)
            torch.cuda.synchronize()
            fp32["train_samples_per_s"] = 3 * args.batch / (a.elapsed_time(b) / 1e3)
            fp32["train_speedup"] = train_rate / world / fp32["train_samples_per_s"]
            del tr32

    # ---- the FP8-E4M3 form of the same decode -------------------------------
    fp8 = None
    if precision == "f16" and forms and not args.no_fp32_compare:
        m8 = forms["f8"]
        for _ in range(2):
            ntc.ntc_decode(m8, q_dev, out=out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(5):
            ntc.ntc_decode(m8, q_dev, out=out)
        b.record(stream)
        torch.cuda.synchronize()
        ms8 = a.elapsed_time(b) / 5
        fp8 = {"decode_ms": ms8, "decode_texels_per_s": args.queries / (ms8 / 1e3),
               "decode_tflops": flop_per_q * args.queries / (ms8 / 1e3) / 1e12,
               "scales": [float(x) for x in m8.scale.cpu().numpy()],
               "scales_from": "ntc_f8_quantize_weights + ntc_f8_activation_scales (2^16 queries)"}
        if mpeaks.get("fp8_tflops"):
            fp8["tensor_frac_of_measured_fp8"] = fp8["decode_tflops"] / mpeaks["fp8_tflops"]
        fp8["vs_f16_decode_ms"] = statistics.mean(dec_ms)

    # ---- CPU oracle baseline (rank 0, N = 1) --------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, ns, threads, dt = oracle_decode_rate(grids_host, w_host, queries, args.cpu_seconds)
        trate, tn, tthreads, tdt = oracle_train_rate(chain, tgrids, tw, args.batch, args.cpu_seconds)
        cpu = {"value": rate, "unit": "texels/s", "cores": threads, "kind": "oracle",
               "sample": f"first {ns} of the 2^24 decode queries ({dt:.1f} s)",
               "train_samples_per_s": trate, "train_cores": tthreads,
               "train_sample": f"first {tn} of the 2^18 training texels ({tdt:.1f} s)"}

    render = None
    if not args.no_render:
        try:
            if forms is None:
                raise RuntimeError("the camera frame needs the trained decode material")
            render = render_eval(ntc, forms, grids_host, w_host, stream)
        except Exception as e:  # reported, never fatal to the headline line
            render = {"error": f"{type(e).__name__}: {e}"[:300]}

    paper_form = None
    if not args.no_extras and not args.multi_only:
        try:
            paper_form = paper_form_eval(ntc, q_dev, args.batch, stream)
        except Exception as e:  # reported, never fatal to the headline line
            paper_form = {"error": f"{type(e).__name__}: {e}"[:300]}

    u8 = None
    if not args.no_extras and not args.multi_only and precision != "f32":
        try:
            u8 = u8_output_eval(ntc, mat, q_dev, q_host, stream)
        except Exception as e:  # reported, never fatal to the headline line
            u8 = {"error": f"{type(e).__name__}: {e}"[:300]}

    vq = None
    if not args.no_extras and not args.multi_only:
        try:
            vq = vq_eval(ntc, q_dev, stream)
        except Exception as e:  # reported, never fatal to the headline line
            vq = {"error": f"{type(e).__name__}: {e}"[:300]}

    sqvq = None
    if not args.no_extras and not args.multi_only:
        try:
            sqvq = sq_vq_train_eval(ntc, chain, args.batch, seed, stream)
        except Exception as e:  # reported, never fatal to the headline line
            sqvq = {"error": f"{type(e).__name__}: {e}"[:300]}

    equal = None
    if not args.no_extras and not args.multi_only and not args.no_fp32_compare:
        try:
            equal = equal_psnr_eval(ntc, chain, args.batch, seed, stream)
        except Exception as e:  # reported, never fatal to the headline line
            equal = {"error": f"{type(e).__name__}: {e}"[:300]}

    multi = None
    if not args.no_multi:
        try:
            multi = multi_material_eval(ntc, 64, 1 << 20, 1 << 16, stream)
            multi["train_hbm_frac"] = multi["train_hbm_gbs_algorithmic"] / (
                peaks.get("hbm_gbs", 6773.2))
        except Exception as e:  # reported, never fatal to the headline line
            multi = {"error": f"{type(e).__name__}: {e}"[:300]}

    kernels_per_step = 1 + 4  # decode; train: noise pass, fused fwd/bwd, Adam, step counter
    line = {
        "metric": METRIC, "value": value, "unit": "texels/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "f16": "f16", "f8": "e4m3"}[precision], "data": "synthetic",
        "config": {"workload": "decode 4096^2x16 (13 mips, G0 1024^2x12 + G1 512^2x12 @4b, "
                               "MLP 48-64-64-16), 2^24 random (u,v,lod) queries + one train step "
                               "2048^2x12 (G0 512^2x16, G1 256^2x16 FP32, MLP 48-64-64-12), "
                               "2^18 texels", "queries": args.queries, "train_batch": args.batch,
                   "decode_model": (f"compressed by the library's FP16 trainer "
                                    f"({args.decode_train_steps} steps of {args.batch} texels) "
                                    "from a synthetic 4096^2x16 texture set"
                                    if dec_info.get("trained") else "random grids and weights"),
                   "decode_precision": precision, "train_precision": train_prec,
                   "l2": "inputs larger than L2 (0.74 GB streamed per decode pass)",
                   "parallelism": f"replicas x{world}"},
        "train_samples_per_s": train_rate, "train_loss": loss,
        "decode_ms": statistics.median(dec_ms), "train_ms": statistics.median(trn_ms),
        "roofline": roof, "train_roofline": train_roof, "tuning": tuning, "e2e": e2e, "fp32_path": fp32, "cpu_baseline": cpu,
        "render": render, "multi_material": multi, "paper_form": paper_form, "train_crops": crops,
        "fp8_path": fp8, "measured_peaks": mpeaks, "decode_material": dec_info,
        "equal_psnr_training": equal, "vq_decode": vq, "sq_vs_vq_training": sqvq,
        "u8_output": u8,
        "gpu_launches": kernels_per_step * args.steps,
        "clocks": clk.summary(), "wall_s": t_wall,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
