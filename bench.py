#!/usr/bin/env python
"""Throughput of the GB300 NGDBF decoder on the smoothed, adaptive high-rate workload.

Workload: a seeded progressive-edge-growth (6,32)-regular code, N=2048, M=384
(rank 383, rate 1665/2048), 10^6 frames of random information words at each
of Eb/N0 = 3.5, 4.0 and 4.5 dB (BPSK 0 -> +1, AWGN, FP32 samples), decoded by
SM-NGDBF with threshold adaptation and output smoothing: T = 300, W = 64,
theta = -0.7, eta = 0.65, lambda = 0.993, Y_max = 2.0, w = 0.1875 (the high-
rate parameter set of Fig. 5).  One step decodes the three 10^6-frame batches.

Reported: decoded frames/s (value), information Gbit/s, the ALU roofline
fraction of the decode kernel, clocks seen during the timed region, an
end-to-end number through the host-buffer C-ABI call (copies included), and
the FP32 reference decoder timed on the host cores on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import signal
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1402_2773_gb300 import workload as wl  # noqa: E402

FRAMES_PER_POINT = 1_000_000
EBN0_DB = (3.5, 4.0, 4.5)
PARAMS = dict(w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0, t_max=300, smooth_window=64,
              variant=3)
# precision name -> (NGDBF precision, q_bits, dtype label).  "fix8" holds 8-bit Eq. 8 samples
# and sums E_k in a finer fixed-point accumulator; "fix8-eq9" is the all-Q-bit metric of Eq. 9.
PRECISIONS = {"fp32": (0, 0, "f32"), "fp16": (1, 0, "f16"), "fix8": (3, 8, "i8"),
              "fix8-eq9": (2, 8, "i8")}
DATA_SEED = 2014          # information bits and channel noise
DECODER_SEED = 1          # Philox key of the perturbation
# Algorithmic lane operations per (symbol, iteration) of the FP32 path: Philox4x32-10 20 (per
# 4 symbols: 10 rounds of two wide multiplies, counted as 4, and 4 XOR) + inverse-CDF deviate 13
# (odd integer 1, leading zeros 1, normalize 1, segment index 2, table load 1, position v 3,
# cubic 3, sign 1) + perturbation 1 + inversion function 5 + decision bit 1 + penalty sum
# (2 d_v + 2) + threshold, adaptation, window and ballot 4 = 46 + 2 d_v, i.e. 58 for d_v = 6.


def ops_per_symbol_iter(dv: int) -> int:
    """Algorithmic lane operations per (symbol, iteration) of the FP32 path for symbol degree dv."""
    return 46 + 2 * int(dv)


OPS_PER_SYMBOL_ITER = ops_per_symbol_iter(6)
# Lane operations per symbol of the same-mix probe (ngdbf_mix_probe), by the same convention:
# Philox 20 + deviate 13 + perturbation 1 + inversion function 5 + decision bit 1 + threshold,
# adaptation, window and ballot 4 + the count lane's extraction 1 (the probe has no per-check
# penalty work: the decode forms those counts bit-sliced, once for 32 slots).
PROBE_OPS_PER_SYMBOL = 45
PROBE_GROUPS = 32768


def mix_probe(ngdbf, stream, reps=5, warmup=2):
    """Attainable lane-op rate of the decode's per-slot instruction mix (CUDA events, best of reps)."""
    import torch
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    threads = 0
    for _ in range(warmup):
        threads = ngdbf.ngdbf_mix_probe(PROBE_GROUPS, sink.data_ptr(), stream.cuda_stream)
    best = None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ngdbf.ngdbf_mix_probe(PROBE_GROUPS, sink.data_ptr(), stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    symbols = threads * PROBE_GROUPS * 4
    return {"lane_op_s": symbols * PROBE_OPS_PER_SYMBOL / (best / 1e3), "ms": best, "threads": threads,
            "symbols_per_launch": symbols, "ops_per_symbol": PROBE_OPS_PER_SYMBOL}
# DRAM bytes (read + write) per decoded frame of the decode kernel, from an ncu capture of
# this workload at 2*10^4 frames per Eb/N0 point (samples 164 MB per launch, larger than L2):
# 167.6 MB read + 8.0 MB written at 3.5 dB; traffic scales with frames, each frame's samples
# being read once.  Set to None when the kernel changes without a new capture.
DRAM_BYTES_PER_FRAME = 8_697


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def shard(rank: int, world: int, frames_per_gpu: int):
    """Frame ids of a rank: a disjoint range per rank (weak scaling, no data exchange)."""
    return rank * frames_per_gpu, frames_per_gpu


def max_over_ranks(value: float, device) -> float:
    """Largest value over all ranks (timing only; frames never cross ranks)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_blocks(ngdbf, tensors):
    """Page-locked blocks under `tensors`: bytes and the share the kernel backs with huge pages."""
    tot = huge = 0
    for t in tensors:
        try:
            b, h = ngdbf.ngdbf_host_block_info(t.data_ptr())
        except Exception:
            return None
        tot += b
        huge += max(h, 0)
    return {"bytes": tot, "huge_page_fraction": round(huge / tot, 4) if tot else None}


def make_inputs(code, frames, rank, world, pinned=False):
    """Seeded frames per Eb/N0 point; pinned=True puts them in page-locked host blocks from the
    library's allocator (huge-page backed, so copies from them run at the link rate)."""
    from paper_1402_2773_gb300 import ngdbf
    off, F = shard(rank, world, frames)
    ys, cws, sigmas = [], [], []
    for j, eb in enumerate(EBN0_DB):
        buf = ngdbf.host_empty((F, code.n), np.float32) if pinned else None
        y, cw, sig = wl.frames(code, F, eb, seed=DATA_SEED + j, frame_offset=off,
                               out=None if buf is None else buf.numpy())
        ys.append(buf if buf is not None else y)
        cws.append(cw)
        sigmas.append(sig)
    return off, ys, cws, sigmas


class ClockSampler:
    """nvidia-smi samples during the timed region (read only; changes no setting)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for ln in open(self.path):
                p = [x.strip() for x in ln.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_baseline(code, ys, cws, sigmas, gpu_outs, precision="fp32", target_s=15.0):
    """Reference decoder (same arithmetic) on all host cores, on a bounded sample of the same
    frames; also checks that the GPU decoded those frames identically."""
    import oracle
    O = oracle.load()
    prec, q_bits, _ = PRECISIONS[precision]
    op = oracle.make_params(**PARAMS, precision=prec, q_bits=q_bits)
    cores = os.cpu_count() or 1
    # calibrate on a small slice, then size the sample for about target_s seconds
    probe = max(cores, 64)
    t0 = time.perf_counter()
    O.decode_f32(code, np.asarray(ys[1][:probe]), sigmas[1], op, seed=DECODER_SEED + 1, threads=cores)
    per_frame = (time.perf_counter() - t0) / probe
    per_point = int(max(cores, min(20000, target_s / max(per_frame, 1e-7) / len(EBN0_DB))))
    total, secs, mism = 0, 0.0, 0
    for j in range(len(EBN0_DB)):
        y = np.ascontiguousarray(np.asarray(ys[j][:per_point]))
        t0 = time.perf_counter()
        b, it, ps = O.decode_f32(code, y, sigmas[j], op, seed=DECODER_SEED + j, frame_offset=0, threads=cores)
        secs += time.perf_counter() - t0
        total += per_point
        if gpu_outs is not None:
            gb, gi, gp = gpu_outs[j]
            mism += int(((gb[:per_point] != b).any(axis=1) | (gi[:per_point] != it) | (gp[:per_point] != ps)).sum())
    fps = total / secs
    return {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"first {per_point} frames of each of the {len(EBN0_DB)} Eb/N0 batches "
                      f"({total} frames, {precision} reference decoder, {cores} threads)",
            "info_gbit_s": fps * code.k / 1e9, "seconds": secs,
            "parity": {"frames": total, "mismatches": mism}}


def error_rates(code, outs, cws):
    res = {}
    info = code.encoder().info_pos
    for j, eb in enumerate(EBN0_DB):
        b, it, ps = outs[j]
        fe = (b != cws[j]).any(axis=1)
        xb = wl.unpack_bits(b, code.n)[:, info]
        tb = wl.unpack_bits(cws[j], code.n)[:, info]
        be = (xb != tb)
        n = b.shape[0]
        fer = float(fe.mean())
        half = 1.96 * math.sqrt(max(fer * (1 - fer), 1.0 / n) / n)
        res[str(eb)] = {"frames": n, "fer": fer, "fer_ci95": [max(0.0, fer - half), fer + half],
                        "ber_info": float(be.mean()), "avg_iters": float(it.mean()),
                        "pass_rate": float(ps.mean())}
    return res


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1402_2773_gb300 import ngdbf

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    ngdbf.load()
    code = wl.code_c2()
    off, ys_host, cws, sigmas = make_inputs(code, args.frames_per_point, rank, world, pinned=True)
    dc = ngdbf.DeviceCode.from_code(code)
    prec, q_bits, dtype = PRECISIONS[args.precision]
    gp = ngdbf.make_params(**PARAMS, precision=prec, q_bits=q_bits)
    ys = [y.cuda(non_blocking=False) for y in ys_host]
    F = args.frames_per_point
    nb = (code.n + 7) // 8
    outs = [(torch.empty((F, nb), dtype=torch.uint8, device="cuda"),
             torch.empty(F, dtype=torch.int32, device="cuda"),
             torch.empty(F, dtype=torch.uint8, device="cuda")) for _ in EBN0_DB]
    stream = torch.cuda.current_stream()

    def step(evs=None):
        for j in range(len(EBN0_DB)):
            if evs is not None:
                evs[j][0].record(stream)
            dc.decode(ys[j], sigmas[j], gp, seed=DECODER_SEED + j, frame_offset=off, out=outs[j], stream=stream)
            if evs is not None:
                evs[j][1].record(stream)

    for _ in range(args.warmup):
        step()
    launch = ngdbf.ngdbf_last_launch()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in EBN0_DB] for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t_start.record(stream)
        for s in range(args.steps):
            step(evs[s])
        t_end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    kernel_ms = [evs[s][j][0].elapsed_time(evs[s][j][1]) for s in range(args.steps) for j in range(len(EBN0_DB))]
    elapsed = max_over_ranks(elapsed, "cuda")
    frames_total = F * len(EBN0_DB) * args.steps * world
    fps = frames_total / elapsed

    host_outs = [(b.cpu().numpy(), i.cpu().numpy(), p.cpu().numpy()) for b, i, p in outs]
    with ClockSampler(local) as probe_clk:
        probe = mix_probe(ngdbf, stream)
    probe["clocks"] = probe_clk.summary()
    rates = error_rates(code, host_outs, cws)
    # roofline: algorithmic lane-ops of the iterations the frames needed, per launch
    sym_iters = [float(o[1].astype(np.int64).sum()) * code.n for o in host_outs]
    mean_launch_s = float(np.mean(kernel_ms)) / 1e3
    ops_per_launch = float(np.mean(sym_iters)) * OPS_PER_SYMBOL_ITER
    clocks = clk.summary()
    peak_mhz = clocks.get("sm_max_mhz") or measured_peaks().get("sm_max_mhz") or 2070.0
    sm_count = launch.get("sm_count") or 152
    peak_ops = sm_count * 128 * peak_mhz * 1e6      # 4 schedulers x 32 lanes issue per SM-clock
    achieved = ops_per_launch / mean_launch_s
    # the capture behind DRAM_BYTES_PER_FRAME is of the FP32 kernel
    traffic = DRAM_BYTES_PER_FRAME * F if (DRAM_BYTES_PER_FRAME and args.precision == "fp32") else None
    # the peak is the measured rate of the same instruction mix (probe), at the probe's clock
    # scaled to the decode's sampled clock; the nominal issue rate is kept beside it
    pclk = probe["clocks"].get("sm_mhz") or peak_mhz
    dclk = clocks.get("sm_mhz") or peak_mhz
    peak_meas = probe["lane_op_s"] * dclk / pclk
    rl = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_meas / 1e12, "unit": "Tlane-op/s",
          "frac": achieved / peak_meas, "traffic": traffic,
          "peak_basis": f"measured: same-mix probe (ngdbf_mix_probe, {PROBE_OPS_PER_SYMBOL} lane-ops per symbol) "
                        f"{probe['lane_op_s'] / 1e12:.2f} T at {pclk:.0f} MHz, scaled to the decode's median "
                        f"{dclk:.0f} MHz",
          "peak_nominal": peak_ops / 1e12, "frac_nominal": achieved / peak_ops,
          "peak_nominal_basis": f"{sm_count} SMs x 128 lanes x {peak_mhz:.0f} MHz (max SM clock)",
          "probe": {k: v for k, v in probe.items() if k != "clocks"} | {"sm_mhz": pclk},
          "kernel": "ngdbf_persistent_kernel<ADAPT,SMOOTH,state in smem>",
          "ops_per_symbol_iter": OPS_PER_SYMBOL_ITER,
          "ops_basis": "FP32 path" if args.precision == "fp32" else
                       "FP32 path count; the rounding or quantizing steps of this precision are not counted",
          "algorithmic_bytes_per_launch": F * (4 * code.n + nb + 5),
          "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum per frame on a 2*10^4-frame "
                           "capture, scaled to the launch's frames" if traffic else
                           "no capture of this precision's kernel",
          "symbol_iters_per_launch": float(np.mean(sym_iters)), "mean_launch_ms": mean_launch_s * 1e3}

    # end to end through the host-buffer C-ABI call: copies inside the timed region
    e2e_steps = max(1, args.steps)
    # the outputs of all points in one page-locked block (each array at a 256-byte offset)
    al = lambda v: (v + 255) // 256 * 256
    per = al(F * nb) + al(F * 4) + al(F)
    flat = ngdbf.host_empty(per * len(EBN0_DB), np.uint8)
    bits_p = [flat[j * per:j * per + F * nb].view(F, nb) for j in range(len(EBN0_DB))]
    it_p = [flat[j * per + al(F * nb):j * per + al(F * nb) + F * 4].view(torch.int32) for j in range(len(EBN0_DB))]
    ps_p = [flat[j * per + al(F * nb) + al(F * 4):j * per + al(F * nb) + al(F * 4) + F] for j in range(len(EBN0_DB))]
    dc.decode_host(ys_host[0][:4096], sigmas[0], gp, seed=DECODER_SEED, frame_offset=off,
                   out=(bits_p[0][:4096], it_p[0][:4096], ps_p[0][:4096]))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    host_stats = []
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for j in range(len(EBN0_DB)):
            dc.decode_host(ys_host[j], sigmas[j], gp, seed=DECODER_SEED + j, frame_offset=off,
                           out=(bits_p[j], it_p[j], ps_p[j]))
            host_stats.append(ngdbf.ngdbf_last_host_stats())
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, "cuda")
    e2e_ok = all(np.array_equal(bits_p[j].numpy(), host_outs[j][0]) for j in range(len(EBN0_DB)))
    tot = {k: sum(h[k] for h in host_stats) for k in ("h2d_bytes", "d2h_bytes", "h2d_ms", "kernel_ms", "d2h_ms",
                                                     "wall_ms", "chunks")}
    e2e = {"value": F * len(EBN0_DB) * e2e_steps * world / e2e_s, "unit": "frames/s",
           "h2d_bytes_per_step": F * code.n * 4 * len(EBN0_DB),
           "d2h_bytes_per_step": F * (nb + 4 + 1) * len(EBN0_DB), "steps": e2e_steps,
           "matches_device_run": bool(e2e_ok),
           "host_buffers": "page-locked, from ngdbf_host_alloc (huge pages requested)",
           "host_input_blocks": host_blocks(ngdbf, ys_host),
           # CUDA events around each chunk of ngdbf_decode_host (device clock)
           "h2d_gbs": tot["h2d_bytes"] / max(tot["h2d_ms"], 1e-9) / 1e6,
           "d2h_gbs": tot["d2h_bytes"] / max(tot["d2h_ms"], 1e-9) / 1e6,
           "chunks": tot["chunks"], "h2d_ms": tot["h2d_ms"], "kernel_ms": tot["kernel_ms"],
           "d2h_ms": tot["d2h_ms"], "event_wall_ms": tot["wall_ms"],
           "host_wall_ms": e2e_s * 1e3,
           "device_kernel_ms_same_frames": mean_launch_s * 1e3 * len(EBN0_DB) * e2e_steps}

    base = None
    if rank == 0 and not args.no_cpu_baseline:
        base = cpu_baseline(code, [y.numpy() for y in ys_host], cws, sigmas, host_outs, args.precision)

    if rank == 0:
        line = {
            "metric": "decoded frames/s", "value": fps, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic (seeded PEG code, random information words, AWGN)",
            "config": {"workload": "SM-NGDBF (adaptive, smoothed), PEG (6,32) N=2048 M=384 rate 1665/2048, "
                                   "10^6 frames at each of Eb/N0 3.5/4.0/4.5 dB per step",
                       "precision": args.precision,
                       "code": "peg(6,32) N=2048 M=384 seed 1", "frames_per_point": F,
                       "ebn0_db": list(EBN0_DB), "params": PARAMS, "decoder_seed": DECODER_SEED,
                       "l2": "inputs larger than L2 (8.2 GB of samples per batch)",
                       "parallelism": f"replicas x{world} (disjoint frame ranges)"},
            "info_gbit_s": fps * code.k / 1e9,
            "roofline": rl,
            "error_rates": rates,
            "launch": launch,
            "gpu_launches": len(EBN0_DB) * args.steps,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": base,
        }
        print(json.dumps(line))
    dc.close()
    if world > 1:
        dist.destroy_process_group()


# Uneven multi-code workload: five seeded PEG codes, frame counts from a seeded geometric
# distribution (mean 4096), per-code Eb/N0 in [3.5, 4.5] dB and T in 100..300, SM-NGDBF with
# the paper's parameter sets (rate 1/2: Figs. 2-4; (6,32): Fig. 5) and a d_v = 3 set for (3,15).
MULTI_CODES = [((3, 504, 252), "peg(3,6) N=504"), ((3, 1008, 504), "peg(3,6) N=1008"),
               ((4, 4096, 2048), "peg(4,8) N=4096"), ((6, 2048, 384), "peg(6,32) N=2048"),
               ((3, 8192, 1639), "peg(3,15) N=8192")]
MULTI_SEED = 404


def multicode_jobs(rank=0):
    rng = np.random.default_rng(MULTI_SEED)
    jobs = []
    for (dv, n, m), name in MULTI_CODES:
        F = int(rng.geometric(1.0 / 4096))
        eb = float(rng.uniform(3.5, 4.5))
        T = int(rng.integers(100, 301))
        code = wl.peg_code(n, m, dv, seed=1, name=name)
        if dv == 6:            # high-rate set of Fig. 5
            prm = dict(w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0)
        elif code.rate > 0.7:  # (3,15): a d_v = 3 code needs a larger weight (chosen on 48 frames)
            prm = dict(w=0.5, theta=-0.7, eta=0.8, lam=0.99, y_max=2.5)
        else:                  # rate 1/2 sets of Figs. 2-4
            prm = dict(w=0.75, theta=-0.9, eta=0.95 if dv == 3 else 0.7, lam=0.99, y_max=2.5)
        prm.update(t_max=T, smooth_window=64, variant=3)
        jobs.append(dict(code=code, frames=F, ebn0=eb, params=prm, offset=rank * 10 ** 7))
    return jobs


def run_multicode(args):
    """One persistent launch over the job table against one launch per code."""
    import torch
    from paper_1402_2773_gb300 import ngdbf

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    ngdbf.load()
    jobs = multicode_jobs(rank)
    dcs, ys, sig, gps = [], [], [], []
    for j, jb in enumerate(jobs):
        y, _, s_ = wl.frames(jb["code"], jb["frames"], jb["ebn0"], seed=DATA_SEED + 10 + j, frame_offset=jb["offset"])
        dcs.append(ngdbf.DeviceCode.from_code(jb["code"]))
        ys.append(torch.from_numpy(y).cuda())
        sig.append(s_)
        gps.append(ngdbf.make_params(**jb["params"]))
    stream = torch.cuda.current_stream()
    tune = args.shape is None
    batch = ngdbf.Batch([(dc, y, s_, gp, jb["offset"]) for dc, y, s_, gp, jb in zip(dcs, ys, sig, gps, jobs)],
                        seed=DECODER_SEED, flags=ngdbf.NGDBF_BATCH_GRAPH | (ngdbf.NGDBF_BATCH_TUNE if tune else 0))
    if not tune:
        batch.use_shape(args.shape)
    batch.launch(stream)
    launch = ngdbf.ngdbf_last_launch()
    shapes = batch.shapes()
    outs = [(torch.empty_like(o[0]), torch.empty_like(o[1]), torch.empty_like(o[2])) for o in batch.outputs]
    outs_it = [(torch.empty_like(o[0]), torch.empty_like(o[1]), torch.empty_like(o[2])) for o in batch.outputs]

    def plain():
        for dc, y, s_, gp, jb, o in zip(dcs, ys, sig, gps, jobs, outs):
            dc.decode(y, s_, gp, seed=DECODER_SEED, frame_offset=jb["offset"], out=o, stream=stream)

    def plain_iter():
        for dc, y, s_, gp, jb, o in zip(dcs, ys, sig, gps, jobs, outs_it):
            dc.decode_plain(y, s_, gp, seed=DECODER_SEED, frame_offset=jb["offset"], out=o, stream=stream)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3

    with ClockSampler(local) as clk:
        t_iter = max_over_ranks(timed(plain_iter), "cuda")
        iter_launches = sum(3 * jb["params"]["t_max"] + 3 for jb in jobs)
        t_plain = max_over_ranks(timed(plain), "cuda")
        t_batch = max_over_ranks(timed(lambda: batch.launch(stream)), "cuda")
        probe = mix_probe(ngdbf, stream)
    same = all(all(torch.equal(a, b) for a, b in zip(o1, o2)) for o1, o2 in zip(batch.outputs, outs))
    same_iter = all(all(torch.equal(a, b) for a, b in zip(o1, o2)) for o1, o2 in zip(batch.outputs, outs_it))
    frames = sum(jb["frames"] for jb in jobs)
    fps = frames * args.steps * world / t_batch
    fps_plain = frames * args.steps * world / t_plain
    fps_iter = frames * args.steps * world / t_iter
    host = [tuple(t.cpu().numpy() for t in o) for o in batch.outputs]
    per_code = []
    ops = 0.0
    for jb, o in zip(jobs, host):
        it = o[1].astype(np.int64)
        dv = jb["code"].dense().sum(axis=0).max()
        ops += float(it.sum()) * jb["code"].n * ops_per_symbol_iter(dv)
        per_code.append({"code": jb["code"].name, "frames": jb["frames"], "ebn0_db": round(jb["ebn0"], 3),
                         "t_max": jb["params"]["t_max"], "avg_iters": float(it.mean()),
                         "pass_rate": float(o[2].mean())})
    clocks = clk.summary()
    peak_nominal = (launch.get("sm_count") or 152) * 128 * (clocks.get("sm_max_mhz") or 2070.0) * 1e6
    peak = probe["lane_op_s"]
    achieved = ops / (t_batch / args.steps)
    if rank == 0:
        print(json.dumps({
            "metric": "decoded frames/s", "value": fps, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded PEG codes, random information words, AWGN)",
            "config": {"workload": "uneven multi-code batch: five PEG codes, geometric frame counts "
                                   "(mean 4096), per-code Eb/N0 and T, SM-NGDBF, one persistent launch "
                                   "(CUDA graph; shape tuned over block size x cluster size x table placement)"
                                   if tune else f"... candidate shape {args.shape} (not tuned)",
                       "codes": per_code, "tuned_shape": batch.shape(), "candidate_shapes": len(shapes),
                       "l2": "inputs and slot state smaller than L2 between launches (both arms alike)"},
            "plain_per_iteration": {"value": fps_iter, "unit": "frames/s", "ms_per_step": t_iter / args.steps * 1e3,
                                    "launches_per_step": iter_launches,
                                    "form": "ngdbf_decode_plain per code: syndrome, retire and update kernels per "
                                            "iteration, one byte per decision"},
            "plain_per_code": {"value": fps_plain, "unit": "frames/s", "ms_per_step": t_plain / args.steps * 1e3,
                               "launches_per_step": len(jobs),
                               "form": "one persistent ngdbf_decode per code"},
            "speedup_vs_plain": fps / fps_plain, "speedup_vs_plain_per_iteration": fps / fps_iter,
            "results_identical": bool(same and same_iter),
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tlane-op/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_basis": f"measured: same-mix probe ({PROBE_OPS_PER_SYMBOL} lane-ops per symbol)",
                         "peak_nominal": peak_nominal / 1e12, "frac_nominal": achieved / peak_nominal,
                         "kernel": "ngdbf_multi_cluster_kernel / ngdbf_multi_kernel (tuned)"},
            "launch": launch, "gpu_launches": args.steps, "clocks": clocks,
        }))
    batch.close()
    for dc in dcs:
        dc.close()


SERVE_SEED = 505
SERVE_BINS = (3.0, 3.5, 4.0, 4.5, 5.0)      # Eb/N0 of the input pools; a request takes the nearest
SERVE_POOL = 4096                          # frames per (code, Eb/N0) pool


def serving_trace(n_req, rate, n_codes):
    """Seeded Poisson arrivals of requests: (arrival s, code, frames 1..4096, pool bin, start, Eb/N0)."""
    rng = np.random.default_rng(SERVE_SEED)
    t = np.cumsum(rng.exponential(1.0 / rate, n_req))
    out = []
    for k in range(n_req):
        c = int(rng.integers(n_codes))
        F = int(rng.integers(1, SERVE_POOL + 1))
        eb = float(rng.uniform(3.0, 5.0))
        b = int(np.argmin([abs(eb - x) for x in SERVE_BINS]))
        start = int(rng.integers(0, SERVE_POOL - F + 1))
        out.append((float(t[k]), c, F, b, start, eb))
    return out


def run_serving(args):
    """Continuous-batching server against one synchronous decode per request, same arrival trace."""
    import threading
    import torch
    from paper_1402_2773_gb300 import ngdbf

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    ngdbf.load()
    specs = multicode_jobs(rank)
    codes = [jb["code"] for jb in specs]
    dvs = [int(c.dense().sum(axis=0).max()) for c in codes]
    dcs = [ngdbf.DeviceCode.from_code(c) for c in codes]
    params = [ngdbf.make_params(**jb["params"]) for jb in specs]
    # every input pool in one page-locked block from the library's allocator
    pools = {}
    flat = ngdbf.host_empty(sum(SERVE_POOL * code.n for code in codes) * len(SERVE_BINS), np.float32)
    pos = 0
    for c, code in enumerate(codes):
        for b, eb in enumerate(SERVE_BINS):
            buf = flat[pos:pos + SERVE_POOL * code.n].view(SERVE_POOL, code.n)
            pos += SERVE_POOL * code.n
            _, _, sig = wl.frames(code, SERVE_POOL, eb, seed=DATA_SEED + 100 * c + b, out=buf.numpy())
            pools[(c, b)] = (buf, sig)
    pool_blocks = host_blocks(ngdbf, [flat])

    def outputs(trace):
        return [(torch.empty((F, (codes[c].n + 7) // 8), dtype=torch.uint8, pin_memory=True),
                 torch.empty(F, dtype=torch.int32, pin_memory=True), torch.empty(F, dtype=torch.uint8, pin_memory=True))
                for _, c, F, _, _, _ in trace]

    def run_server(trace):
        srv = ngdbf.Server(8 << 30, max_inflight=4, max_jobs=256, seed=DECODER_SEED)
        outs = outputs(trace)
        sub = [0.0] * len(trace)
        t0 = time.perf_counter()
        for k, (ta, c, F, b, st, _) in enumerate(trace):
            d = t0 + ta - time.perf_counter()
            if d > 0:
                time.sleep(d)
            sub[k] = time.perf_counter() - t0
            buf, sig = pools[(c, b)]
            srv.submit(dcs[c], buf[st:st + F], sig, params[c], frame_offset=10 ** 9 * (k + 1), out=outs[k])
        srv.wait(3600)
        done = {rid: (lat, stt) for rid, lat, stt in srv.poll()}
        stats = srv.stats()
        srv.close()
        lat = np.array([done[k + 1][0] for k in range(len(trace))])
        assert all(done[k + 1][1] == 0 for k in range(len(trace)))
        end = max(sub[k] + lat[k] for k in range(len(trace)))
        return lat, end - sub[0], stats, outs

    def run_plain(trace):
        outs = outputs(trace)
        lat = []
        t0 = time.perf_counter()
        for k, (ta, c, F, b, st, _) in enumerate(trace):
            d = t0 + ta - time.perf_counter()
            if d > 0:
                time.sleep(d)
            buf, sig = pools[(c, b)]
            dcs[c].decode_host(buf[st:st + F], sig, params[c], seed=DECODER_SEED, frame_offset=10 ** 9 * (k + 1),
                               out=outs[k])
            lat.append(time.perf_counter() - t0 - ta)
        return np.array(lat), time.perf_counter() - t0 - trace[0][0], outs

    n_req = args.requests
    frames = None
    res = {}
    with ClockSampler(local) as clk:
        warm = serving_trace(8, 1e9, len(codes))
        run_server(warm)
        for label, rate in (("offered", args.rate), ("at_load", None)):
            if rate is None:      # 60 % of the capacity measured at the offered rate
                rate = 0.6 * res["offered"]["server_requests_per_s"]
            trace = serving_trace(n_req, rate, len(codes))
            frames = sum(F for _, _, F, _, _, _ in trace)
            lat_s, span_s, stats, outs_s = run_server(trace)
            lat_p, span_p, outs_p = run_plain(trace)
            same = all(all(torch.equal(a, b) for a, b in zip(x, y)) for x, y in zip(outs_s, outs_p))
            # algorithmic lane operations of the iterations the frames needed (FP32 count)
            ops = sum(float(o[1].numpy().astype(np.int64).sum()) * codes[c].n * ops_per_symbol_iter(dvs[c])
                      for (_, c, _, _, _, _), o in zip(trace, outs_s))
            res[label] = {
                "rate_requests_per_s": rate, "requests": n_req, "frames": frames,
                "server_frames_per_s": frames / span_s, "server_requests_per_s": n_req / span_s,
                "server_latency_ms": {"p50": float(np.percentile(lat_s, 50)) * 1e3,
                                      "p99": float(np.percentile(lat_s, 99)) * 1e3},
                "plain_frames_per_s": frames / span_p,
                "plain_latency_ms": {"p50": float(np.percentile(lat_p, 50)) * 1e3,
                                     "p99": float(np.percentile(lat_p, 99)) * 1e3},
                "results_identical": bool(same), "server_stats": stats,
                "server_lane_op_s": ops / span_s}
        probe = mix_probe(ngdbf, torch.cuda.current_stream())
    clocks = clk.summary()
    for label in res:
        res[label]["server_alu_frac"] = res[label]["server_lane_op_s"] / probe["lane_op_s"]
    if rank == 0:
        off = res["offered"]
        print(json.dumps({
            "metric": "decoded frames/s", "value": off["server_frames_per_s"], "unit": "frames/s", "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": frames / off["server_frames_per_s"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded PEG codes, random information words, AWGN)",
            "config": {"workload": f"serving: Poisson arrivals of {n_req} requests of 1-4096 frames over five PEG "
                                   "codes, Eb/N0 uniform 3-5 dB, SM-NGDBF, 8 GiB device budget, 4 streams, "
                                   "up to 256 requests per launch; input pools page-locked (ngdbf_host_alloc)",
                       "codes": [c.name for c in codes]},
            "serving": res, "clocks": clocks, "input_pool_blocks": pool_blocks,
            "e2e": {"value": off["server_frames_per_s"], "unit": "frames/s",
                    "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                    "note": "serving is measured end to end (host buffers, copies included)"},
        }))
    for dc in dcs:
        dc.close()


def run_reference(args):
    """The FP32 reference decoder on the host cores: same workload, metric and unit."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle
    O = oracle.load()
    code = wl.code_c2()
    cores = os.cpu_count() or 1
    op = oracle.make_params(**PARAMS)
    # per step: a bounded sample of each Eb/N0 batch, sized so the run ends within minutes
    per_point = int(os.environ.get("NGDBF_REF_FRAMES", "0"))
    ys, sig = [], []
    if per_point <= 0:
        # about 6 s of decoding per step, from a timed probe at the middle Eb/N0
        y, _, s = wl.frames(code, 4 * cores, 4.0, seed=DATA_SEED + 1)
        t0 = time.perf_counter()
        O.decode_f32(code, y, s, op, seed=DECODER_SEED + 1, threads=cores)
        per_frame = (time.perf_counter() - t0) / (4 * cores)
        per_point = int(min(5000, 6.0 / max(per_frame, 1e-7) / len(EBN0_DB)))
    per_point = max(cores, per_point)
    for j, eb in enumerate(EBN0_DB):
        y, _, s = wl.frames(code, per_point, eb, seed=DATA_SEED + j)
        ys.append(y)
        sig.append(s)

    def step():
        for j in range(len(EBN0_DB)):
            O.decode_f32(code, ys[j], sig[j], op, seed=DECODER_SEED + j, threads=cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    secs = time.perf_counter() - t0
    fps = per_point * len(EBN0_DB) * args.steps / secs
    sample = (f"first {per_point} frames of each of the {len(EBN0_DB)} Eb/N0 batches per step, "
              f"FP32 reference decoder, {cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": "decoded frames/s", "value": fps, "unit": "frames/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded PEG code, random information words, AWGN)",
        "config": {"workload": "SM-NGDBF (adaptive, smoothed), PEG (6,32) N=2048 M=384 rate 1665/2048, "
                               "10^6 frames at each of Eb/N0 3.5/4.0/4.5 dB per step",
                   "code": "peg(6,32) N=2048 M=384 seed 1", "frames_per_point": per_point,
                   "ebn0_db": list(EBN0_DB), "params": PARAMS},
        "info_gbit_s": fps * code.k / 1e9,
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["sm-ngdbf-6x32", "multicode", "serving"], default="sm-ngdbf-6x32",
                    help="the benchmark workload (default) or the uneven multi-code batch")
    ap.add_argument("--requests", type=int, default=300, help="serving workload: requests per run")
    ap.add_argument("--rate", type=float, default=2e5, help="serving workload: offered requests/s")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp32",
                    help="arithmetic of the held samples and E_k (the perturbation stays FP32)")
    ap.add_argument("--shape", type=int, default=None,
                    help="multicode workload: use candidate launch shape K of the job table instead of tuning")
    ap.add_argument("--frames-per-point", type=int, default=FRAMES_PER_POINT,
                    help="frames per Eb/N0 batch (the benchmark workload is 10^6; smaller only for profiling)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "multicode":
        run_multicode(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
