#!/usr/bin/env python
"""Benchmark of the CT volume ray caster on one GPU per rank (replicas; weak scaling).

Default workload: a 512 x 512 x 400 int16 synthetic CT resident in HBM, rendered to 1024^2
perspective images (30 degree field of view) from 16 seeded orbit cameras, step 0.5 voxel,
8^3 brick empty-space leaping, early ray termination at opacity 0.999. One step = rebuild the
brick min/max table, rebuild the occupancy for the transfer function, render the 16 frames.
L2 is flushed (a 256 MB write) before every step, outside the step's events.

Printed: one JSON line on rank 0. `value` is executed samples per second (Gsamples/s, all
ranks; executed = samples in occupied bricks up to termination, the oracle's count); Mrays/s
and nominal Gsamples/s ride along. `roofline` reports one render call (the split render's two
kernels) against the stencil's bound max(N F / P_fp32, N G / BW_L1): F = 230 flop and G = 128
bytes (64 int16 taps) per sample, P_fp32 and BW_L1 the lower of this device's measured rates
(vrc_microbench) and its unit counts (152 SMs x 128 lanes x 2 flop, x 128 bytes, at 2.07 GHz);
`frac` counts executed samples, `frac_resampled` only those resampled. `dense_tf` repeats the
frames with a transfer function that makes soft tissue semi-transparent (long rays, nearly all
samples resampled). `cpu_baseline` times the FP64 oracle on host cores on a bounded sample of
the same workload. `e2e` repeats the measurement through vrc_render_host_batch (each step's
images read back to pinned host memory inside the timed region, each frame's copy overlapping
the next frame's render).

`--impl reference` times the FP64 CPU oracle itself on the same workload (bounded samples).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_SAMPLE = 230        # algorithmic FP32 flops per sample (FMA = 2)
GATHER_BYTES_PER_SAMPLE = 128  # 64 int16 taps: the least a sample reads from on-chip memory
ADJ_FLOPS_PER_SAMPLE = 400     # reverse mode: forward recompute 230 + backward chain about 170
ADJ_ATOMIC_BYTES_PER_SAMPLE = 256  # 64 voxel-gradient float atomics per resampled sample
FP32_LANES = 128
L1_BYTES_PER_CLK = 128
SM_MAX_MHZ = 2070.0
METRIC = ("Gsamples/s & Mrays/s (512²×400 CT, 1024² img) vs roofline; "
          "p50/p99 req latency")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="vrc", choices=["vrc", "reference"])
    p.add_argument("--brick", type=int, default=8)
    p.add_argument("--cameras", type=int, default=16)
    p.add_argument("--kernel", type=int, default=0)
    p.add_argument("--no-dense", action="store_true")
    p.add_argument("--tf", default="ct", choices=["ct", "dense"],
                   help="transfer function of the headline frames (dense: soft tissue "
                        "semi-transparent)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--mode", default="render",
                   choices=["render", "serve", "adjoint", "large", "variants", "sortlast"])
    p.add_argument("--serve-seconds", type=float, default=10.0)
    p.add_argument("--grid", default="1,1,1;2,2,2;3,3,3;4,4,4",
                   help="--mode sortlast: piece grids gx,gy,gz separated by ';'")
    return p.parse_args()


def workload_config(args):
    tf = "" if getattr(args, "tf", "ct") == "ct" else "_densetf"
    return {"workload": f"ct512x512x400_i16_to_1024sq_persp30_step0.5_B{args.brick}_ert0.999_"
                        f"{args.cameras}cams{tf}",
            "transfer_function": getattr(args, "tf", "ct"),
            "volume": [512, 512, 400], "volume_dtype": "int16", "image": [1024, 1024],
            "fovy_deg": 30.0, "step": 0.5, "brick": args.brick, "ert": 0.999,
            "cameras": args.cameras, "ct_seed": 3, "camera_seed": 4,
            "l2": "flushed (256 MB write) before every step",
            "parallelism": f"replicas x{args.gpus}"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None
        self.active = False
        self.lock = threading.Lock()

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            with self.lock:
                if self.active:
                    self.rows.append([x.strip() for x in line.split(",")])

    def mark(self, on: bool):
        with self.lock:
            self.active = on

    def rows_clear(self):
        with self.lock:
            self.rows = []

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        with self.lock:
            rows = list(self.rows)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if args.impl == "vrc" else "gloo")
    return rank, world, local


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks of the default process group (the value itself
    without one): the timed region of a replicated run ends when its slowest rank ends."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_sample(vol, tf, cams, rows_every: int, brick: int):
    """Times the oracle on rows 0, k, 2k, ... of the first camera; returns (seconds,
    executed samples, rays, threads)."""
    import numpy as np

    import oracle
    from paper_2005_01442_gb300 import synth
    try:
        ncores = len(os.sched_getaffinity(0))
    except Exception:
        ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    cam = cams[0]
    rows = np.arange(0, cam.height, rows_every)
    pix = np.stack(np.meshgrid(np.arange(cam.width), rows), -1).reshape(-1, 2)
    t0 = time.perf_counter()
    _, counts = oracle.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, ert=0.999,
                              brick=brick, pixels=pix, return_counts=True)
    dt = time.perf_counter() - t0
    return dt, counts[1], counts[0], pix.shape[0], oracle.get_threads()


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle timed on host cores (rank 0 only)."""
    if rank != 0:
        return
    from paper_2005_01442_gb300 import synth
    vol = synth.ct_volume()
    tf = synth.tf_ct()
    cams = synth.orbit_cameras(4, args.cameras, synth.dims_of(vol), 1024, 1024)
    rows_every = 4
    times, ex, nom, rays = [], 0, 0, 0
    threads = 1
    for i in range(args.warmup + args.steps):
        dt, e, n, r, threads = cpu_sample(vol, tf, [cams[i % len(cams)]], rows_every, args.brick)
        if i >= args.warmup:
            times.append(dt)
            ex += e
            nom += n
            rays += r
    total = sum(times)
    value = ex / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gsamples/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "mrays_per_s": rays / total / 1e6, "gsamples_nominal_per_s": nom / total / 1e9,
            "cpu_baseline": {"value": value, "unit": "Gsamples/s", "cores": threads,
                             "kind": "oracle",
                             "sample": f"each step: every {rows_every}th row of one 1024^2 "
                                       "frame (cameras in turn), ESL+ERT on"},
            "e2e": {"value": value, "unit": "Gsamples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_peaks(R, sms: int) -> dict:
    """The stencil's two roofs on this device: measured (vrc_microbench) and unit-count figures,
    and the lower of the two, which the roofline divides by."""
    spec_fp32 = sms * FP32_LANES * 2 * SM_MAX_MHZ * 1e6
    spec_l1 = sms * L1_BYTES_PER_CLK * SM_MAX_MHZ * 1e6
    fma, l1, lds = R.microbench(0), R.microbench(1), R.microbench(2)
    return {"fp32_tflops": min(fma, spec_fp32) / 1e12, "fp32_tflops_measured": fma / 1e12,
            "fp32_tflops_spec": spec_fp32 / 1e12,
            "l1_gbs": min(l1, spec_l1) / 1e9, "l1_gbs_measured": l1 / 1e9,
            "lds_gbs_measured": lds / 1e9, "l1_gbs_spec": spec_l1 / 1e9,
            "source": "min(measured vrc_microbench, unit count at 2070 MHz); "
                      f"{sms} SMs"}


def roofline(executed: int, resampled: int, launch_ms: float, peaks: dict, kernel: str) -> dict:
    """Roofline of one render call: max(N F / P_fp32, N G / BW_L1) over its CUDA-event time,
    N = executed samples (`frac`) or resampled samples (`frac_resampled`)."""
    t = launch_ms / 1e3
    p_alu, p_l1 = peaks["fp32_tflops"] * 1e12, peaks["l1_gbs"] * 1e9
    alu, gat = FLOPS_PER_SAMPLE * executed / t, GATHER_BYTES_PER_SAMPLE * executed / t
    alu_r, gat_r = FLOPS_PER_SAMPLE * resampled / t, GATHER_BYTES_PER_SAMPLE * resampled / t
    l1_binds = gat / p_l1 >= alu / p_alu
    return {"bound": "l1_gather" if l1_binds else "alu",
            "achieved": gat / 1e9 if l1_binds else alu / 1e12,
            "peak": peaks["l1_gbs"] if l1_binds else peaks["fp32_tflops"],
            "unit": "GB/s" if l1_binds else "TFLOP/s",
            "frac": max(gat / p_l1, alu / p_alu),
            "traffic": None,
            "alu_frac": alu / p_alu, "gather_frac": gat / p_l1,
            "frac_resampled": max(gat_r / p_l1, alu_r / p_alu),
            "alu_frac_resampled": alu_r / p_alu, "gather_frac_resampled": gat_r / p_l1,
            "executed_per_launch": executed, "resampled_per_launch": resampled,
            "launch_ms": launch_ms, "kernel": kernel,
            "basis": f"{FLOPS_PER_SAMPLE} flop and {GATHER_BYTES_PER_SAMPLE} B (64 int16 taps) "
                     "per sample; peaks measured on this device (of measured)",
            "traffic_note": "DRAM bytes per launch come from ncu captures, not from this run",
            "peaks": peaks}


SERVE_SIZES = [(512, 512), (1024, 1024), (2048, 2048)]
SERVE_HBM_BUDGET = 8 << 30  # device bytes of the requests in flight (images + ray queues)
SERVE_P99_CAP_MS = 33.0     # latency cap of the rate sweep: one frame at 30 frames/s
# one launch per request; one persistent launch whose warps render (mode 0); one persistent
# scheduler launch that starts each request's render on the device (mode 1)
SERVE_KINDS = ("plain", "batched", "launching")


def serve_bench(R, torch, vols, tids, runs, brick, seed, p99_cap_ms=SERVE_P99_CAP_MS):
    """Open-loop Poisson load (seeded) of mixed volumes, transfer functions, orbit cameras and
    image sizes, replayed against the one-launch-per-request server and the two persistent
    batched servers (SERVE_KINDS) for each (offered rate, seconds, warm-up seconds) run; admission by an HBM
    budget for the requests in flight. For each server, `best_at_p99_cap` is the highest
    images/s of a run whose p99 latency stays under the cap."""
    from paper_2005_01442_gb300 import serve, synth

    def cam_fn(rng, v, w, h):
        return synth.orbit_camera(rng, vols[v], w, h)

    for v in vols:
        for t in tids:
            R.build_occupancy(v, t, brick)
    torch.cuda.synchronize()
    out = {"volumes": [list(d) for d in vols.values()], "transfer_functions": len(tids),
           "images": [f"{w}x{h}" for w, h in SERVE_SIZES], "brick": brick,
           "hbm_budget_bytes": SERVE_HBM_BUDGET, "p99_cap_ms": p99_cap_ms, "runs": []}
    for rate, seconds, warm in runs:
        reqs = serve.poisson_requests(seed, rate, seconds + warm, list(vols), tids,
                                      SERVE_SIZES, cam_fn, brick=brick)
        for kind in SERVE_KINDS:
            srv = serve.PlainServer(R) if kind == "plain" else \
                serve.BatchedServer(R, max_slots=1024, mode=1 if kind == "launching" else 0)
            budget = serve.ImageBudget(SERVE_HBM_BUDGET, lambda h, w: torch.empty(
                (h, w, 4), dtype=torch.float32, device="cuda"), srv.extra_bytes_per_pixel)
            res = serve.run_open_loop(srv, reqs, budget, warmup=warm)
            srv.close()
            res.pop("latencies_s")
            res.pop("records")
            res["offered_rate"] = rate
            res["seconds"] = seconds
            res["warmup_s"] = warm
            out["runs"].append(res)
    best = {}
    for kind in SERVE_KINDS:
        ok = [r for r in out["runs"] if r["server"] == kind and r["p99_ms"] <= p99_cap_ms]
        top = max(ok, key=lambda r: r["images_per_s"]) if ok else None
        best[kind] = ({"images_per_s": top["images_per_s"], "p99_ms": top["p99_ms"],
                       "p50_ms": top["p50_ms"], "offered_rate": top["offered_rate"]}
                      if top else None)
    out["best_at_p99_cap"] = best
    for kind in SERVE_KINDS[1:]:
        if best["plain"] and best[kind]:
            out[f"{kind}_over_plain_at_p99_cap"] = (best[kind]["images_per_s"] /
                                                    best["plain"]["images_per_s"])
    return out


def serve_volumes(R, synth, B, resident=None):
    """The serving workload's resident volumes: 256^3, 512^2 x 400 and 512^2 x 1200 int16 CTs
    (seeds 5, 3, 6); `resident` = (id, dims) of an already resident 512^2 x 400 seed-3 CT."""
    vols = {}
    for shape, seed in [((256, 256, 256), 5), ((400, 512, 512), 3), ((1200, 512, 512), 6)]:
        if resident is not None and shape == (400, 512, 512) and seed == 3:
            vols[resident[0]] = resident[1]
            continue
        v = synth.ct_volume(shape, seed=seed)
        vid = R.upload_volume(v)
        R.build_bricks(vid, B)
        vols[vid] = synth.dims_of(v)
        del v
    return vols


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    from paper_2005_01442_gb300 import build as vbuild
    from paper_2005_01442_gb300 import synth
    from paper_2005_01442_gb300.renderer import Renderer

    torch.cuda.set_device(local)
    if rank == 0:
        vbuild.build()
    if world > 1:
        torch.distributed.barrier()
    vbuild.build()
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    gpu_id = f"GPU-{uuid}" if uuid is not None else str(local)
    if args.mode != "render":
        global _SAMPLER
        _SAMPLER = ClockSampler(gpu_id)
        _SAMPLER.start()
        time.sleep(0.5)
        R = Renderer(local)
        run_mode(args, torch, R, synth)
        R.close()
        _SAMPLER.stop()
        return

    vol = synth.ct_volume()
    tf = synth.tf_ct() if args.tf == "ct" else synth.tf_ct_dense()
    dims = synth.dims_of(vol)
    cams = synth.orbit_cameras(4 + 1000 * rank, args.cameras, dims, 1024, 1024)
    R = Renderer(local)
    vid = R.upload_volume(vol)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    B = args.brick
    stream = torch.cuda.current_stream(dev)
    out = torch.empty((args.cameras, 1024, 1024, 4), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # sample counts (deterministic; measured once, outside the timed region)
    R.build_bricks(vid, B)
    cnt = torch.zeros((args.cameras, 3), dtype=torch.int64, device=dev)
    for i, cam in enumerate(cams):
        R.render(vid, tid, cam, ert=0.999, brick=B, out=out[i], counters=cnt[i],
                 kernel=args.kernel)
    torch.cuda.synchronize()
    nominal, executed, resampled = [int(x) for x in cnt.sum(0).tolist()]
    rays_per_step = args.cameras * 1024 * 1024

    def one_step(ev_frames=None):
        R.build_bricks(vid, B)
        R.build_occupancy(vid, tid, B)
        for i, cam in enumerate(cams):
            if ev_frames is not None:
                ev_frames[i][0].record(stream)
            R.render(vid, tid, cam, ert=0.999, brick=B, out=out[i], kernel=args.kernel)
            if ev_frames is not None:
                ev_frames[i][1].record(stream)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        one_step()
    torch.cuda.synchronize()

    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.5)
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    frame_ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in cams] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.mark(True)
    for s in range(args.steps):
        flush.fill_(float(s))
        step_ev[s][0].record(stream)
        one_step(frame_ev[s])
        step_ev[s][1].record(stream)
    torch.cuda.synchronize()
    sampler.mark(False)
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    frame_ms = [a.elapsed_time(b) for fr in frame_ev for a, b in fr]
    total_ms = max_over_ranks(sum(step_ms), dev)
    secs = total_ms / 1e3
    value = world * executed * args.steps / secs / 1e9

    # end to end through the public host-buffer call
    e2e = None
    if not args.no_e2e:
        host = torch.empty((args.cameras, 1024, 1024, 4), dtype=torch.float32, pin_memory=True)
        for _ in range(2):
            R.build_bricks(vid, B)
            R.render_host_batch(vid, tid, cams, out=host, ert=0.999, brick=B, kernel=args.kernel)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            R.build_bricks(vid, B)
            R.render_host_batch(vid, tid, cams, out=host, ert=0.999, brick=B, kernel=args.kernel)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
        e2e = {"value": world * executed * args.steps / e2e_s / 1e9, "unit": "Gsamples/s",
               "h2d_bytes_per_step": args.cameras * 60,  # vrc_camera records passed by value
               "d2h_bytes_per_step": args.cameras * 1024 * 1024 * 16,
               "api": "vrc_render_host_batch (the step's cameras in one call; pinned host "
                      "images, each read back while the next frame renders, inside the timed "
                      "region)"}

    clocks = sampler.summary()
    sms = props.multi_processor_count
    kernel_ms = statistics.mean(frame_ms)
    kname = ("one render call: split_head_kernel + split_tail_kernel" if args.kernel in (0, 6)
             else f"render kernel {args.kernel}")
    # the other workload (the dense transfer function) and the other kernel (TMA-staged), A/B
    legs = []
    if not args.no_dense:
        other_tf = "dense" if args.tf == "ct" else "ct"
        other_k = 7 if args.kernel in (0, 6) else 0
        for tfk, k in ((args.tf, other_k), (other_tf, args.kernel), (other_tf, other_k)):
            legs.append(frames_leg(args, torch, R, synth, vid, cams, out, flush, stream, sampler,
                                   world, dev, tfk, k))
    line = None
    if rank == 0:
        peaks = measure_peaks(R, sms)  # after the timed regions
        roof = roofline(executed // args.cameras, resampled // args.cameras, kernel_ms, peaks,
                        kname)
        for leg in legs:
            leg["roofline"] = roofline(leg.pop("_executed"), leg.pop("_resampled"),
                                       leg["ms_per_frame"], peaks, leg["kernel_name"])
        sgemm = fp32_sgemm_tflops(torch, dev)
        cpu = None
        if not args.no_cpu_baseline:
            # a bounded sample of the step (~10 s of host work): whole frames, cameras in
            # turn, until 10 s have passed
            dt = ex = 0.0
            nframes = 0
            threads = 1
            while dt < 10.0 and nframes < 64:
                d, e, _, _, threads = cpu_sample(vol, tf, [cams[nframes % len(cams)]], 1, B)
                dt += d
                ex += e
                nframes += 1
            cpu = {"value": ex / dt / 1e9, "unit": "Gsamples/s", "cores": threads,
                   "kind": "oracle",
                   "sample": f"{nframes} whole 1024^2 frames, the step's cameras in turn, "
                             f"ESL B={B} + ERT, {dt:.1f} s"}
        line = {
            "metric": METRIC, "value": value, "unit": "Gsamples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(args),
            "mrays_per_s": world * rays_per_step * args.steps / secs / 1e6,
            "gsamples_nominal_per_s": world * nominal * args.steps / secs / 1e9,
            "samples_per_step": {"nominal": nominal, "executed": executed,
                                 "resampled": resampled},
            "render_kernel_ms": kernel_ms,
            "roofline": roof,
            "fp32_sgemm_tflops_measured": sgemm,
            "other_workloads_and_kernels": legs,
            "cpu_baseline": cpu, "e2e": e2e,
            # bricks, occupancy, 3 summed-volume passes, distance, cell mask; per frame the
            # split render's two kernels (one for the per-ray kernel)
            "gpu_launches": args.steps * (7 + args.cameras * (2 if args.kernel in (0, 6) else 1)),
            "clocks": clocks,
        }
        if not args.no_serve:
            # the serving workload: three resident CTs, four transfer functions, 512^2 /
            # 1024^2 / 2048^2 images; the nominal 200 req/s stream, then a rate sweep
            vols = serve_volumes(R, synth, B, resident=(vid, dims) if args.tf == "ct" else None)
            tids = [R.set_tf(synth.tf_ct(k), synth.CT_LO, synth.CT_HI) for k in (None, 1, 2, 3)]
            sweep = [(r, 4.0, 1.0) for r in (400.0, 800.0, 1200.0, 1400.0, 1600.0)]
            sampler.rows_clear()  # clock record of the serving runs
            sampler.mark(True)
            line["serving"] = serve_bench(R, torch, vols, tids,
                                          [(200.0, args.serve_seconds, 2.0)] + sweep, B,
                                          seed=5)
            sampler.mark(False)
            line["serving"]["clocks"] = sampler.summary()
        print(json.dumps(line), flush=True)
    sampler.stop()
    R.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def frames_leg(args, torch, R, synth, vid, cams, out, flush, stream, sampler, world, dev,
               tf_kind: str, kernel: int):
    """The headline volume and cameras with transfer function `tf_kind` ("ct" or "dense": soft
    tissue semi-transparent) rendered by `kernel`: frame time of the render call (CUDA events,
    L2 flushed before each group of frames), its sample counts and its own clock record."""
    B = args.brick
    tf = synth.tf_ct() if tf_kind == "ct" else synth.tf_ct_dense()
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    R.build_occupancy(vid, tid, B)
    cnt = torch.zeros((len(cams), 3), dtype=torch.int64, device=dev)
    for i, cam in enumerate(cams):
        R.render(vid, tid, cam, ert=0.999, brick=B, out=out[i], counters=cnt[i], kernel=kernel)
    torch.cuda.synchronize()
    nominal, executed, resampled = [int(x) for x in cnt.sum(0).tolist()]
    steps = max(1, min(args.steps, 5))
    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        for i, cam in enumerate(cams):
            R.render(vid, tid, cam, ert=0.999, brick=B, out=out[i], kernel=kernel)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in cams] for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.rows_clear()
    sampler.mark(True)
    for s in range(steps):
        flush.fill_(float(s))
        for i, cam in enumerate(cams):
            ev[s][i][0].record(stream)
            R.render(vid, tid, cam, ert=0.999, brick=B, out=out[i], kernel=kernel)
            ev[s][i][1].record(stream)
    torch.cuda.synchronize()
    sampler.mark(False)
    ms = statistics.mean(a.elapsed_time(b) for fr in ev for a, b in fr)
    R.free_tf(tid)
    nf = len(cams)
    return {"transfer_function": ("CT (transparent below 150 HU; vessels, bone)" if tf_kind == "ct"
                                  else "dense: soft tissue semi-transparent (about 0.01-0.02 "
                                       "opacity per voxel), vessels and bone more opaque"),
            "kernel": kernel, "kernel_name": KERNEL_NAMES.get(kernel, str(kernel)),
            "ms_per_frame": ms, "frames_timed": steps * nf,
            "gsamples_per_s": executed / nf / (ms / 1e3) / 1e9,
            "gsamples_resampled_per_s": resampled / nf / (ms / 1e3) / 1e9,
            "mrays_per_s": 1024 * 1024 / (ms / 1e3) / 1e6,
            "samples_per_frame": {"nominal": nominal // nf, "executed": executed // nf,
                                  "resampled": resampled // nf},
            "clocks": sampler.summary(),
            "_executed": executed // nf, "_resampled": resampled // nf}


KERNEL_NAMES = {0: "split render (split_head_kernel + split_tail_kernel)",
                6: "split render (split_head_kernel + split_tail_kernel)",
                1: "one ray per thread (render_ray_kernel)",
                7: "TMA-staged boxes in shared memory (render_tma_kernel)"}


def _gauss_blur(a, sigma=1.5, radius=5):
    import numpy as np
    x = np.arange(-radius, radius + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    k /= k.sum()
    pad = np.pad(a, radius, mode="reflect")
    tmp = sum(k[i] * pad[i:i + a.shape[0], :] for i in range(k.size))
    return sum(k[i] * tmp[:, i:i + a.shape[1]] for i in range(k.size))


def image_quality(img, ref):
    """(PSNR in dB, mean SSIM) of an RGBA image against a reference, values in [0, 1];
    SSIM with the usual 11-tap Gaussian window (sigma 1.5), K1 = 0.01, K2 = 0.03, averaged
    over the four channels."""
    import numpy as np
    mse = float(np.mean((img - ref) ** 2))
    psnr = float("inf") if mse == 0.0 else 10.0 * np.log10(1.0 / mse)
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    ss = []
    for ch in range(img.shape[-1]):
        a, b = img[..., ch], ref[..., ch]
        ma, mb = _gauss_blur(a), _gauss_blur(b)
        va = _gauss_blur(a * a) - ma * ma
        vb = _gauss_blur(b * b) - mb * mb
        cab = _gauss_blur(a * b) - ma * mb
        m = ((2 * ma * mb + c1) * (2 * cab + c2)) / ((ma * ma + mb * mb + c1) * (va + vb + c2))
        ss.append(float(m.mean()))
    return psnr, float(np.mean(ss))


def fp32_sgemm_tflops(torch, dev, n=8192, reps=5):
    """Measured FP32 FMA rate of the CUDA cores: a cuBLAS SGEMM with TF32 off (context for the
    ALU roof, which stays the unit-count figure)."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        a = torch.randn(n, n, device=dev)
        b = torch.randn(n, n, device=dev)
        for _ in range(2):
            a @ b
        ms = _timed(torch, lambda: a @ b, reps)
        del a, b
        return 2.0 * n ** 3 / (ms / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


_SAMPLER = None  # clock sampler of the --mode runs (marks the timed regions)


def _mark(on: bool):
    if _SAMPLER is not None:
        _SAMPLER.mark(on)


def _clocks():
    return _SAMPLER.summary() if _SAMPLER is not None else None


def _timed(torch, fn, reps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    _mark(True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    _mark(False)
    return e0.elapsed_time(e1) / reps


def run_mode(args, torch, R, synth):
    """--mode serve | adjoint | large | variants: the serving, differentiation and large
    workloads and the interpolation / classification variants; one JSON line each (not the
    headline metric)."""
    import numpy as np
    dev = torch.device("cuda", 0)
    if args.mode == "serve":
        vols = serve_volumes(R, synth, args.brick)
        tids = [R.set_tf(synth.tf_ct(k), synth.CT_LO, synth.CT_HI) for k in (None, 1, 2, 3)]
        _mark(True)
        res = serve_bench(R, torch, vols, tids,
                          [(200.0, 60.0, 5.0)] + [(r, 10.0, 2.0) for r in
                                                  (400.0, 800.0, 1200.0, 1400.0, 1600.0, 2000.0)],
                          args.brick, seed=5)
        _mark(False)
        print(json.dumps({"mode": "serve", "metric": "p50/p99 request latency (ms) and images/s",
                          "data": "synthetic", "serving": res, "clocks": _clocks()}), flush=True)
        return
    if args.mode == "adjoint":
        vol = synth.ct_float_downsampled(7)
        dims = synth.dims_of(vol)
        cams = synth.orbit_cameras(7, 8, dims, 512, 512)
        vid = R.upload_volume(vol)
        R.build_bricks(vid, args.brick)
        tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
        tgt_tf = R.set_tf(synth.tf_ct(8), synth.CT_LO, synth.CT_HI)
        targets = [R.render(vid, tgt_tf, c, brick=args.brick).clone() for c in cams]
        imgs = [torch.empty((512, 512, 4), device=dev) for _ in cams]
        gtf = torch.zeros((256, 4), device=dev)
        gvol = torch.zeros(vol.shape, device=dev)
        cnt = torch.zeros(3, dtype=torch.int64, device=dev)
        for c, im in zip(cams, imgs):
            R.render(vid, tid, c, brick=args.brick, out=im, counters=cnt)
        torch.cuda.synchronize()
        executed, resampled = int(cnt[1]), int(cnt[2])

        # the forward records each camera's checkpoints; the adjoint reads them
        cks = [R.ckpt_buffer(vid, c, 0.5, 64) for c in cams]

        def fwd():
            for c, im, ck in zip(cams, imgs, cks):
                R.render(vid, tid, c, brick=args.brick, out=im, ckpt=ck)

        def bwd():
            for c, im, t, ck in zip(cams, imgs, targets, cks):
                R.render_backward(vid, tid, c, 2.0 * (im - t), gtf, gvol, brick=args.brick,
                                  ckpt=ck)

        for _ in range(args.warmup):
            fwd()
            bwd()
        f_ms = _timed(torch, fwd, args.steps)
        b_ms = _timed(torch, bwd, args.steps)
        loss = float(sum(((im - t) ** 2).sum() for im, t in zip(imgs, targets)))
        # roofline of the adjoint launches: every resampled sample is recomputed from its
        # segment checkpoint (230 flop) and walked back (about 170 flop: classification and
        # opacity chain, 64 tap weights times the value gradient), and adds 64 float gradients
        # (256 bytes of vector atomics) into the voxel gradients
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        fma = min(R.microbench(0), sms * FP32_LANES * 2 * SM_MAX_MHZ * 1e6)
        red = R.microbench(3)
        t_b = b_ms / 1e3
        alu = ADJ_FLOPS_PER_SAMPLE * resampled / t_b
        atom = ADJ_ATOMIC_BYTES_PER_SAMPLE * resampled / t_b
        adj_roof = {"bound": "atomics" if atom / red >= alu / fma else "alu",
                    "alu_frac": alu / fma, "atomic_frac": atom / red,
                    "frac": max(alu / fma, atom / red),
                    "achieved_tflops": alu / 1e12, "achieved_atomic_gbs": atom / 1e9,
                    "peak_fp32_tflops": fma / 1e12, "peak_atomic_gbs_measured": red / 1e9,
                    "basis": f"{ADJ_FLOPS_PER_SAMPLE} flop and {ADJ_ATOMIC_BYTES_PER_SAMPLE} B of "
                             "float atomics per resampled sample over the adjoint launches' time; "
                             "atomic peak = vrc_microbench kind 3 (of measured)"}
        print(json.dumps({
            "mode": "adjoint", "metric": "forward+adjoint Gsamples/s", "data": "synthetic",
            "config": {"volume": [256, 256, 256], "volume_dtype": "float32",
                       "cameras": 8, "image": [512, 512], "step": 0.5, "brick": args.brick,
                       "loss": "L2 vs targets rendered with transfer function seed 8"},
            "forward_ms_per_step": f_ms, "backward_ms_per_step": b_ms,
            "forward": "split render recording checkpoints (seg_len 64)",
            "checkpoint_bytes_per_camera": int(cks[0].numel()),
            "executed_samples_per_step": executed, "resampled_samples_per_step": resampled,
            "loss": loss, "adjoint_roofline": adj_roof,
            "value": executed / ((f_ms + b_ms) / 1e3) / 1e9, "unit": "Gsamples/s",
            "gpu_launches": 8 * args.steps * 3, "clocks": _clocks()}), flush=True)
        return
    if args.mode == "variants":
        # the paper's Fig. 4 comparison on the headline workload: frame time of each
        # interpolation / classification variant and its PSNR / SSIM against the tricubic
        # post-classified image
        vol = synth.ct_volume()
        dims = synth.dims_of(vol)
        cams = synth.orbit_cameras(4, args.cameras, dims, 1024, 1024)
        vid = R.upload_volume(vol)
        R.build_bricks(vid, args.brick)
        tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
        out = torch.empty((len(cams), 1024, 1024, 4), device=dev)
        rows, ref = [], None
        for interp, preclass, phong, preint, name in [
                (0, 0, None, 0, "tricubic post-classification"),
                (1, 0, None, 0, "trilinear post-classification"),
                (0, 1, None, 0, "tricubic pre-classification"),
                (1, 1, None, 0, "trilinear pre-classification"),
                (0, 0, (0.3, 0.7, 0.25, 16.0), 0, "tricubic post-classification + Phong"),
                (0, 0, None, 0, "tricubic post-classification, no skipping"),
                (0, 0, None, 1, "pre-integrated (slabs), no skipping")]:
            brick = 0 if "no skipping" in name else args.brick

            def frames():
                for i, c in enumerate(cams):
                    R.render(vid, tid, c, ert=0.999, brick=brick, out=out[i], interp=interp,
                             preclass=preclass, phong=phong, preint=preint)
            for _ in range(args.warmup):
                frames()
            ms = _timed(torch, frames, args.steps) / len(cams)
            imgs = out[:4].cpu().numpy().astype(np.float64)  # quality on the first 4 frames
            if ref is None:
                ref = imgs.copy()
            q = [image_quality(a, b) for a, b in zip(imgs, ref)]
            rows.append({"variant": name, "interp": interp, "preclass": preclass,
                         "phong": phong, "preint": preint, "brick": brick,
                         "ms_per_frame": ms, "mrays_per_s": 1024 * 1024 / (ms / 1e3) / 1e6,
                         "psnr_db": (None if all(math.isinf(x[0]) for x in q)  # identical
                                     else float(np.mean([x[0] for x in q]))),
                         "ssim": float(np.mean([x[1] for x in q]))})
        print(json.dumps({
            "mode": "variants", "metric": "ms per frame; PSNR / SSIM vs tricubic "
            "post-classification (RGBA, peak 1)", "data": "synthetic",
            "config": workload_config(args), "variants": rows,
            "gpu_launches": 7 * (args.warmup + args.steps) * len(cams) * 2, "clocks": _clocks()}), flush=True)
        return
    if args.mode == "sortlast":
        # object-order rendering: the headline workload cut into grids of pieces of whole
        # bricks, each piece rendered into the rectangle of its visible box, then blended in
        # visibility order; frame time against the one-pass render, and the blend kernel
        # timed alone against the HBM roofline (bytes: every partial pixel read once, every
        # image pixel written once)
        from paper_2005_01442_gb300 import native
        vol = synth.ct_volume()
        dims = synth.dims_of(vol)
        cams = synth.orbit_cameras(4, args.cameras, dims, 1024, 1024)
        vid = R.upload_volume(vol)
        R.build_bricks(vid, args.brick)
        tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
        out = torch.empty((1024, 1024, 4), device=dev)
        ref = torch.empty_like(out)
        try:
            hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
            hbm_src = "measured"
        except (OSError, KeyError, ValueError):
            hbm, hbm_src = 6800.0, "fallback"

        def one_pass():
            for c in cams:
                R.render(vid, tid, c, ert=0.999, brick=args.brick, out=out)
        for _ in range(args.warmup):
            one_pass()
        base_ms = _timed(torch, one_pass, args.steps) / len(cams)
        rows = []
        for grid in [tuple(int(x) for x in g.split(",")) for g in args.grid.split(";")]:
            plan = R.build_pieces(vid, tid, args.brick, grid)
            pieces, _ = R.pieces(plan)

            def frames():
                for c in cams:
                    R.render_sortlast(plan, c, ert=0.999, brick=args.brick, out=out)
            for _ in range(args.warmup):
                frames()
            ms = _timed(torch, frames, args.steps) / len(cams)

            def ordered():
                for c in cams:
                    R.render_ordered(plan, c, ert=0.999, brick=args.brick, out=out)
            for _ in range(args.warmup):
                ordered()
            ord_ms = _timed(torch, ordered, args.steps) / len(cams)
            # the blend alone, on the partials of the first camera
            cam = cams[0]
            order = native.grid_order(cam, grid, R.pieces(plan)[1])
            rects, parts = [], []
            for k, p in enumerate(pieces):
                lo = [max(float(p["vis_lo"][a]), -0.5) for a in range(3)]
                hi = [min(float(p["vis_hi"][a]), dims[a] - 0.5) for a in range(3)]
                r = native.box_rect(cam, lo, hi)
                rects.append(r)
                parts.append(R.render_piece(plan, k, cam, r, ert=0.999, brick=args.brick)
                             if r[2] and r[3] else None)
            flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MB > L2
            c_ms = 0.0
            for rep in range(23):  # 3 warm-up launches, then 20 timed, L2 flushed before each
                flush.fill_(float(rep))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                R.composite(parts, rects, order, 1024, 1024, out=out)
                e1.record()
                torch.cuda.synchronize()
                if rep >= 3:
                    c_ms += e0.elapsed_time(e1) / 20
            del flush
            nbytes = 16 * (sum(r[2] * r[3] for r in rects) + 1024 * 1024)
            # agreement with the one-pass render on the first four cameras
            d_off = d_on = d_ord = 0.0
            for c in cams[:4]:
                R.render(vid, tid, c, ert=1.0, brick=args.brick, out=ref)
                R.render_sortlast(plan, c, ert=1.0, brick=args.brick, out=out)
                d_off = max(d_off, float((out - ref).abs().max()))
                R.render(vid, tid, c, ert=0.999, brick=args.brick, out=ref)
                R.render_sortlast(plan, c, ert=0.999, brick=args.brick, out=out)
                d_on = max(d_on, float((out - ref).abs().max()))
                R.render_ordered(plan, c, ert=0.999, brick=args.brick, out=out)
                d_ord = max(d_ord, float((out - ref).abs().max()))
            rows.append({
                "grid": list(grid), "pieces": len(pieces),
                "visible_pieces": sum(p["vis_hi"] != (0, 0, 0) for p in pieces),
                "sortlast_ms_per_frame": ms, "sortlast_vs_one_pass": ms / base_ms,
                "ordered_ms_per_frame": ord_ms, "ordered_vs_one_pass": ord_ms / base_ms,
                "partial_pixels_first_camera": sum(r[2] * r[3] for r in rects),
                "composite_us": c_ms * 1e3, "composite_gbs": nbytes / (c_ms / 1e3) / 1e9,
                "composite_frac_of_hbm": nbytes / (c_ms / 1e3) / 1e9 / hbm,
                "max_abs_diff_vs_one_pass_no_ert": d_off,
                "max_abs_diff_vs_one_pass_ert": d_on,
                "max_abs_diff_ordered_vs_one_pass_ert": d_ord})
            R.free_pieces(plan)
        print(json.dumps({
            "mode": "sortlast", "metric": "ms per frame of the object-order paths (sort-last: "
            "pieces + blend; ordered: pieces front to back) vs the one-pass render",
            "data": "synthetic", "config": workload_config(args),
            "one_pass_ms_per_frame": base_ms, "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_src,
            "grids": rows, "clocks": _clocks()}), flush=True)
        return
    if args.mode == "large":
        vol = synth.ct_volume((2000, 512, 512), seed=9)
        dims = synth.dims_of(vol)
        vid = R.upload_volume(vol)
        del vol
        B = 16
        R.build_bricks(vid, B)
        tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
        cam = synth.orbit_cameras(9, 1, dims, 4096, 4096)[0]
        img = torch.empty((4096, 4096, 4), device=dev)
        cnt = torch.zeros(3, dtype=torch.int64, device=dev)
        R.render(vid, tid, cam, step=0.25, ert=0.999, brick=B, out=img, counters=cnt)
        torch.cuda.synchronize()
        nominal, executed, resampled = (int(x) for x in cnt.tolist())
        g = torch.rand((4096, 4096, 4), device=dev) - 0.5
        gtf = torch.zeros((256, 4), device=dev)
        gvol = torch.zeros((dims[2], dims[1], dims[0]), device=dev)
        ck = R.ckpt_buffer(vid, cam, 0.25, 64)  # caller-owned checkpoints (about 9 GB)
        plain = lambda: R.render(vid, tid, cam, step=0.25, ert=0.999, brick=B, out=img)  # noqa
        fwd = lambda: R.render(vid, tid, cam, step=0.25, ert=0.999, brick=B, out=img,  # noqa
                               ckpt=ck, seg_len=64)
        bwd = lambda: R.render_backward(vid, tid, cam, g, gtf, gvol, step=0.25,  # noqa
                                        ert=0.999, brick=B, seg_len=64, ckpt=ck)
        plain()
        fwd()
        bwd()
        reps = max(1, min(args.steps, 3))
        p_ms = _timed(torch, plain, reps)
        f_ms = _timed(torch, fwd, reps)
        b_ms = _timed(torch, bwd, reps)
        print(json.dumps({
            "mode": "large", "metric": "forward and adjoint time, Gsamples/s", "data": "synthetic",
            "config": {"volume": [512, 512, 2000], "volume_dtype": "int16", "image": [4096, 4096],
                       "step": 0.25, "brick": B, "ert": 0.999, "seg_len": 64},
            "nominal_samples": nominal, "executed_samples": executed,
            "resampled_samples": resampled, "checkpoint_bytes": int(ck.numel()),
            "render_ms": p_ms, "forward_with_checkpoints_ms": f_ms, "backward_ms": b_ms,
            "forward_gsamples_per_s": executed / (p_ms / 1e3) / 1e9,
            "mrays_per_s": 4096 * 4096 / (p_ms / 1e3) / 1e6, "clocks": _clocks()}), flush=True)
        return


if __name__ == "__main__":
    main()
