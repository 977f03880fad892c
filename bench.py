#!/usr/bin/env python
"""Benchmark of the EPO hot path on GB300: one optimisation step = pair setup, fused
loss + gradient edge kernel, FP64 finalize, FP64 Adam + Exp retraction (one CUDA-graph
replay).  Prints one JSON line.

Workloads (--workload; seeded synthetic scenes, records and maps built on the fly):
  batch64  (default) 64 independent scenes (8..120 views, 256x192 / 518x392 / 518x518, 8
           neighbours, 2-8 % edge density; 4,305 views, 34,440 pairs, 3.2e8 evaluations per
           step) batched in one launch per stage, FP32 records and maps: the largest workload
           at the paper's FP32 precision.  Adds the plain per-scene form (64 handles, kernels
           launched one by one) at equal final pose accuracy.  --scenes N keeps the first N
           scenes (a smaller case of the same kernel, for profiling).
  ring32   32 views at 518x392 on a ring, each paired with its 8 nearest views
           (256 directed pairs), ~20,000 edge pixels per view, FP32 records and maps.
  walk200  200 views at 518x392 on a random walk, 10 neighbours (2,000 pairs), ~30,000 edge
           pixels per view (6e7 evaluations per step); adds the autograd forward + adjoint
           timing and the device memory against a stored-Jacobian variant.
  ring500  500 views at 518x518, 12 neighbours (6,000 pairs), BF16 maps and FP16 depth;
           adds the FP32 form of the same scene and both forms' final pose errors.
Metric: edge-pixel x pair evaluations per second of the loss + gradient step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]
                  [--scenes N] [--schedule GATHER/BLOCK/RPT] [--no-legs] [--no-cpu-baseline]

--impl reference times the FP64 CPU oracle (the reference arm for this build) on the host
cores on the same workload and metric.  For N > 1 (torchrun) every rank runs an
independent replica of the workload (the path shards by scene with no exchange); rank 0
prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edge-pixel*pair evals/s (loss+grad step)"
UNIT = "evals/s"
WORKLOADS = {
    "ring32": "ring32_518x392_k8_20k_f32",
    "walk200": "walk200_518x392_k10_30k_f32",
    "batch64": "batch64_uneven_8to120views_k8_f32",
    "ring500": "ring500_518x518_k12_40k_bf16map_f16depth",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch64", choices=sorted(WORKLOADS))
    ap.add_argument("--scenes", type=int, default=0,
                    help="batch64 only: keep the first N scenes (0 = all 64)")
    ap.add_argument("--schedule", default="",
                    help="fixed edge-kernel schedule gather/block/records_per_thread, e.g. tex/128/2 "
                         "(default: autotuned)")
    ap.add_argument("--no-legs", action="store_true", help="skip the workload's comparison legs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Workload:
    """Seeded synthetic scenes of one benchmark workload, with the stored dtypes."""

    def __init__(self, key, n_scenes=0):
        import synth
        self.key = key
        self.name = WORKLOADS[key]
        if key == "batch64" and n_scenes:
            self.name = f"batch64_uneven_first{n_scenes}of64_8to120views_k8_f32"
        if key == "ring32":
            self.scenes = [synth.make_scene(synth.RING32_518x392, keep_depth=True)]
        elif key == "walk200":
            self.scenes = [synth.make_scene(synth.WALK200_518x392)]
        elif key == "batch64":
            specs = synth.batch64_uneven_specs()
            self.scenes = [synth.make_scene(sp) for sp in (specs[:n_scenes] if n_scenes else specs)]
        elif key == "ring500":
            self.scenes = [synth.make_scene(synth.RING500_518x518)]
        else:
            raise ValueError(key)
        self.mixed = key == "ring500"  # BF16 maps, FP16 depth records

    @property
    def T_init(self):
        return np.concatenate([sc.T_init for sc in self.scenes])

    def parts(self, epo, torch, mixed=None):
        """Scene parts with device-resident records and maps; the maps are the library's
        GPU distance fields (rounded to BF16 on the GPU for the mixed form)."""
        mixed = self.mixed if mixed is None else mixed
        import synth
        out = []
        for sc in self.scenes:
            maps = [epo.distance_field(torch.from_numpy(e).cuda()) for e in sc.edges]
            if mixed:
                maps = [epo.round_bf16(m) for m in maps]
                rec = torch.from_numpy(synth.records_f16(sc.rec).view(np.int16)).cuda()
            else:
                rec = torch.from_numpy(sc.rec).cuda()
            out.append(dict(W=sc.W, H=sc.H, K=sc.K, rec_off=sc.rec_off, rec=rec, maps=maps, pairs=sc.pairs,
                            fixed=sc.fixed))
        return out

    def dtypes(self, epo, mixed=None):
        mixed = self.mixed if mixed is None else mixed
        return (epo.EPO_F16, epo.EPO_BF16) if mixed else (epo.EPO_F32, epo.EPO_F32)


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def captured_traffic(workload, gather, block, rpt, evals):
    """DRAM bytes per edge-kernel launch from the committed ncu capture, or None when the
    kernel source changed since the capture or this schedule was not captured.  A capture
    of a smaller case of the same workload (its first scenes) is scaled to a full launch by
    the evaluations it processed."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "edge_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    key = f"{ {1: 'ldg', 2: 'tex', 3: 'mix'}.get(gather, '?') }/{block}/{rpt}"
    for c in d.get("captures", []):
        srcs = c["kernel_sources_sha256"]
        ok = True
        for path, sha in srcs.items():
            with open(os.path.join(ROOT, path), "rb") as f:
                ok = ok and hashlib.sha256(f.read()).hexdigest() == sha
        if not ok or c.get("workload") != workload or key not in c["dram_bytes_per_launch"]:
            continue
        v = c["dram_bytes_per_launch"][key]
        return int(round(v * evals / c["evals_per_launch"]))
    return None


# ------------------------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and the reference arm)
# ------------------------------------------------------------------------------------------
def _bf16_widened(x):
    """float32 -> nearest bfloat16 (ties to even) -> float32, for finite inputs."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + ((b >> 16) & 1) + 0x7FFF) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


def oracle_for_pairs(sc, pair_ids, mixed):
    """The oracle scene of the given pairs of one synthetic scene: only the views they touch
    (renumbered), their records and their maps as the GPU stores them (widened)."""
    import oracle
    import synth
    pairs = sc.pairs[pair_ids]
    views = np.unique(pairs)
    new_id = -np.ones(sc.n_views, dtype=np.int64)
    new_id[views] = np.arange(len(views))
    recs, offs = [], [0]
    for v in views:
        a, b = sc.rec_off[v], sc.rec_off[v + 1]
        recs.append(sc.rec[a:b])
        offs.append(offs[-1] + (b - a))
    rec = np.concatenate(recs, axis=0)
    maps = [oracle.edt(sc.edges[v]).astype(np.float32) for v in views]
    if mixed:
        rec = synth.records_f16_widened(rec)
        maps = [_bf16_widened(m) for m in maps]
    osc = oracle.OracleScene(sc.W[views], sc.H[views], sc.K[views], np.array(offs, dtype=np.int64), rec,
                             [m.astype(np.float64) for m in maps], new_id[pairs])
    evals = int(np.diff(sc.rec_off)[pairs[:, 0]].sum())
    return osc, sc.T_init[views].copy(), sc.fixed[views].copy(), evals


def oracle_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def time_oracle_steps(osc, T, fixed, n_steps, step0=0, m=None, v=None):
    """n_steps oracle optimisation steps (loss + gradient + Adam/Exp); returns (seconds, state)."""
    t0 = time.perf_counter()
    out = osc.optimize(T, fixed, n_steps, lr_rot=2e-3, lr_trans=2e-2, step0=step0, m=m, v=v)
    return time.perf_counter() - t0, out


def oracle_sample(wl, budget_s, seed=0):
    """A pair subset of the workload's first scene whose one oracle step takes about
    budget_s (all pairs when a step takes less): (oracle scene, T, fixed, evals, n_pairs)."""
    sc = wl.scenes[0]
    rng = np.random.default_rng(seed)
    order = rng.permutation(sc.n_pairs)
    pilot = np.sort(order[: min(8, sc.n_pairs)])
    osc, T, fx, ev = oracle_for_pairs(sc, pilot, wl.mixed)
    time_oracle_steps(osc, T, fx, 1)
    dt, _ = time_oracle_steps(osc, T, fx, 1)
    rate = ev / max(dt, 1e-6)
    cnt = np.diff(sc.rec_off)[sc.pairs[order, 0]]
    n = int(np.searchsorted(np.cumsum(cnt), rate * budget_s)) + 1
    ids = np.sort(order[: min(max(n, 1), sc.n_pairs)])
    osc, T, fx, ev = oracle_for_pairs(sc, ids, wl.mixed)
    return osc, T, fx, ev, len(ids)


def cpu_baseline(wl, budget_s=12.0):
    """The oracle on all host cores (the reported value), and on one thread for reference."""
    import oracle
    cores = oracle.set_threads(oracle_threads())
    osc, T, fx, ev, n_pairs = oracle_sample(wl, budget_s / 4)
    dt1, _ = time_oracle_steps(osc, T, fx, 1)
    n = max(1, int(0.75 * budget_s / max(dt1, 1e-3)))
    dt, _ = time_oracle_steps(osc, T, fx, n)
    oracle.set_threads(1)
    dts, _ = time_oracle_steps(osc, T, fx, 1)
    oracle.set_threads(cores)
    return {"value": ev * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread_value": ev / dts,
            "sample": f"{n} oracle optimisation steps (FP64, OpenMP over pairs) on {n_pairs} of the "
                      f"{wl.scenes[0].n_pairs} pairs of the {'first scene of the ' if len(wl.scenes) > 1 else ''}"
                      f"{wl.name} workload ({ev} evals per step), {ev * n} evals in {dt:.2f} s; "
                      f"single_thread_value: one such step on 1 thread in {dts:.2f} s"}


def job_throughput(units, ms, device="cpu"):
    """Whole-job rate over the ranks of the default process group (or this process alone):
    the units all ranks processed divided by the slowest rank's time."""
    import torch
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return units / (ms * 1e-3), ms
    import torch.distributed as dist
    t = torch.tensor([float(units), float(ms)], dtype=torch.float64, device=device)
    u = t[:1].clone()
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    m = t[1:].clone()
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(u.item()) / (float(m.item()) * 1e-3), float(m.item())


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = Workload(args.workload, args.scenes)
    # each timed step is a bounded sample: a pair subset sized so that the run stays short
    per_step_budget = 150.0 / max(args.steps + args.warmup, 1)
    osc, T, fx, evals, n_pairs = oracle_sample(wl, per_step_budget)
    m = v = None
    step = 0
    for _ in range(args.warmup):
        _, (T, m, v, _) = time_oracle_steps(osc, T, fx, 1, step, m, v)
        step += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, (T, m, v, _) = time_oracle_steps(osc, T, fx, 1, step, m, v)
        step += 1
    dt = time.perf_counter() - t0
    val = evals * args.steps / dt
    sample = (f"each step = oracle loss+grad+Adam/Exp on {n_pairs} of {wl.scenes[0].n_pairs} pairs "
              f"({evals} evals) of the {wl.name} workload")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------
def pose_errors(T, scenes):
    """Mean rotation error (degrees) and mean camera-centre error (fraction of the scene
    scale) of stacked poses T against the scenes' ground truth."""
    rot, tr, off = [], [], 0
    for sc in scenes:
        for v in range(sc.n_views):
            A = T[off + v].reshape(3, 4)
            G = sc.T_gt[v].reshape(3, 4)
            c = (np.trace(A[:, :3] @ G[:, :3].T) - 1) / 2
            rot.append(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))
            ca, cg = -A[:, :3].T @ A[:, 3], -G[:, :3].T @ G[:, 3]
            tr.append(np.linalg.norm(ca - cg) / sc.scale)
        off += sc.n_views
    return float(np.mean(rot)), float(np.mean(tr))


def time_steps(h, n, flush_l2, stream, torch):
    """n flushed, event-timed graph steps of handle h; returns per-step ms."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for k in range(n):
        flush_l2(k)
        ev[k][0].record(stream)
        h.step_async(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    h.check()
    return [x.elapsed_time(y) for x, y in ev]


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2607_00579_gb300 as epo

    wl = Workload(args.workload, args.scenes)
    stream = torch.cuda.current_stream()
    T_init = wl.T_init
    # distance transform fields built on the GPU by the library (construction step)
    parts = wl.parts(epo, torch)
    rd, md = wl.dtypes(epo)
    lr = dict(lr_rot=2e-3, lr_trans=2e-2)

    def scene(options, prts=parts, dt=(rd, md)):
        return epo.Scene(prts, record_dtype=dt[0], map_dtype=dt[1], options=options, on_device=True)

    if args.schedule:
        g, b, r = args.schedule.split("/")
        fixed = dict(gather={"ldg": epo.EPO_GATHER_LDG, "tex": epo.EPO_GATHER_TEX, "mix": epo.EPO_GATHER_MIX}[g],
                     block_threads=int(b),
                     records_per_thread=int(r))
        s = scene(epo.default_options(**lr, **fixed))
        s.set_poses(T_init)
    else:
        s = scene(epo.default_options(autotune=2, **lr))
        s.set_poses(T_init)
        s.autotune()
    info = s.info()
    evals = info.evals_per_step
    # a second handle on the same workload and schedule, with CUDA events captured around
    # each stage inside its graph: kernel and stage times come from it, so that the events
    # do not perturb the headline step time
    sched = dict(gather=info.gather, block_threads=info.block_threads, records_per_thread=info.records_per_thread)
    st_ = scene(epo.default_options(timing=1, **lr, **sched))
    # L2 flush between timed steps: write a 512 MB buffer (4x the L2), then read half of it
    # back, so that the step starts with an L2 full of clean lines unrelated to its inputs
    # (a write alone would leave 126 MB of dirty lines whose write-backs the step would pay)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_sink = torch.empty(1, dtype=torch.float32, device="cuda")

    def flush_l2(k):
        flush.fill_(float(k))
        flush_sink.copy_(flush[: flush.numel() // 2].sum().reshape(1))

    for h in (s, st_):
        h.set_poses(T_init)
        for _ in range(args.warmup):
            h.step_async(1)
        torch.cuda.synchronize()
        h.set_poses(T_init)
        h.set_state(0)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    step_ms = time_steps(s, args.steps, flush_l2, stream, torch)
    t_wall = time.perf_counter() - t_wall0
    # kernel and stage times over the same number of flushed steps on the timed handle
    kern_ms, stages = [], []
    for k in range(args.steps):
        flush_l2(k)
        st_.step_async(1)
        kern_ms.append(epo._binding.epo_kernel_time(st_.handle))
        stages.append(epo._binding.epo_stage_times(st_.handle))
    st_.check()
    clk = clocks.stop()
    value, tot_ms = job_throughput(evals * args.steps, float(np.sum(step_ms)), "cuda")

    # end to end through the public API with host buffers: pinned poses in, step, poses + loss
    # out; each step's output poses are the next step's input (two buffers in turn, passed by
    # address)
    T_host = torch.from_numpy(T_init.copy()).pin_memory()
    T_out = torch.empty_like(T_host).pin_memory()
    loss_out = torch.empty(info.n_scenes, dtype=torch.float64).pin_memory()
    io = (T_host.data_ptr(), T_out.data_ptr())
    e2e_steps = max(10, args.steps // 2)
    # untimed warm-up: the first call captures the host-step graph
    for _ in range(3):
        epo._binding.epo_step_host(s.handle, io[0], io[1], loss_out.data_ptr())
    T_host.copy_(torch.from_numpy(T_init))
    lp = loss_out.data_ptr()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        # one public call per step: poses in, the step, poses and loss out, one sync (the
        # step's graph reads and writes the scene's mapped pinned staging)
        epo._binding.epo_step_host(s.handle, io[k & 1], io[(k + 1) & 1], lp)
    e2e_dt = time.perf_counter() - t0
    e2e = {"value": world * evals * e2e_steps / e2e_dt, "unit": UNIT,
           "h2d_bytes_per_step": int(T_host.numel() * 8),
           "d2h_bytes_per_step": int(T_out.numel() * 8 + loss_out.numel() * 8 + 8)}  # + the status word

    # roofline of the dominant kernel (fused loss + gradient edge kernel)
    peak, peak_src = measured_peaks()
    kern_avg = float(np.mean(kern_ms))
    traffic = captured_traffic(wl.name, info.gather, info.block_threads, info.records_per_thread, evals)
    gather_roof = gather_roofline(epo, wl, info, evals, kern_avg, peak)
    roof = roofline_line(wl, info, evals, kern_avg, gather_roof, traffic, peak, peak_src)
    st_avg = np.mean(np.array(stages), axis=0)
    queued, overflow = epo._binding.epo_fixup_stats(st_.handle)
    # samples of the last evaluated step that were valid (in front, inside the target image):
    # the footprints the gathers had to serve
    valid_evals = int(round(float(st_.pair_stats()[:, 1].sum())))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16/f16 gathers, f32" if wl.mixed else "f32",
            "data": "synthetic",
            "config": {"workload": wl.name, "scenes": info.n_scenes, "views": info.n_views,
                       "pairs": info.n_pairs, "records": info.n_records, "evals_per_step": evals,
                       "l2": "flushed between timed steps (512 MB write, then 256 MB read back)",
                       "schedule": {"gather": info.gather, "block": info.block_threads,
                                    "records_per_thread": info.records_per_thread,
                                    "grid": info.grid_blocks, "tail_pairs": info.tail_pairs,
                                    "work_items": info.n_tiles},
                       "parallelism": f"replicas x{world}" if world > 1 else "single"},
            "gpu_launches": info.kernels_per_step * args.steps, "clocks": clk, "e2e": e2e, "roofline": roof,
            "gather_roofline": gather_roof,
            "stages_ms": {"pair_setup": float(st_avg[0]), "edge_with_exact_path": float(st_avg[1]),
                          "poses": float(st_avg[2])},
            "exact_fixup_samples": queued, "exact_fixup_overflow": overflow, "valid_evals": valid_evals,
            "wall_ms_per_step": 1e3 * t_wall / args.steps}
    del st_
    if args.no_legs:
        pass
    elif wl.key == "walk200":
        line["autograd"] = autograd_leg(epo, torch, s, T_init, evals, args, flush_l2, stream)
    elif wl.key == "batch64":
        leg = plain_per_scene_leg(epo, torch, wl, s, parts, (rd, md), lr, evals, args, flush_l2, stream)
        leg["speedup_of_batched_graph_step"] = leg["ms_per_step"] / (tot_ms / args.steps)
        line["plain_per_scene"] = leg
    elif wl.key == "ring500":
        line["fp32_form"] = fp32_form_leg(epo, torch, wl, s, scene, lr, evals, args, flush_l2, stream)
    elif wl.key == "ring32":
        line["refine"] = refine_leg(epo, torch, wl, parts, (rd, md), lr, evals, args, flush_l2, stream, sched)
        line["viewgraph"] = viewgraph_leg(epo, torch, wl)
        line["pose_mlp"] = pose_mlp_leg(epo, torch, wl, parts, (rd, md), lr, evals, args, flush_l2, stream,
                                        {k: v for k, v in sched.items()})
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def roofline_line(wl, info, evals, kern_ms, gr, traffic, hbm_peak, peak_src):
    """The edge kernel against its roofline t_roof = max(t_hbm, t_gather) (gather_roofline).
    The bound is the larger term: "gather" when serving one 2x2 footprint per evaluation at the
    best rate this GPU's gather probe measured takes longer than moving the compulsory bytes
    (records and maps once) at the measured HBM bandwidth, else "hbm".  achieved and peak are
    the gather term's tap bytes (4 s_map per evaluation) per second: the kernel's, and the
    probe's; frac = t_roof / kernel time.  The HBM side is reported beside it: the compulsory
    bytes, their time at the measured peak, and the DRAM bytes ncu counted for the kernel."""
    s_map = 2 if wl.mixed else 4
    tap = 4 * s_map
    probe = max(gr["gather_footprints_per_s"].values())
    bound = "gather" if gr["t_gather_ms"] >= gr["t_hbm_ms"] else "hbm"
    if bound == "gather":
        achieved, peak, unit = evals * tap / (kern_ms * 1e-3) / 1e9, probe * tap / 1e9, "GB/s"
        psrc = (f"measured in this run: best 2x2-footprint rate of epo_gather_probe "
                f"({probe / 1e9:.1f} G footprints/s x {tap} B of taps)")
    else:
        achieved, peak, unit = gr["hbm_compulsory_bytes"] / (kern_ms * 1e-3) / 1e9, hbm_peak, "GB/s"
        psrc = f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": gr["t_roof_ms"] / kern_ms,
            "traffic": traffic, "peak_source": psrc, "kernel": "k_edge (fused loss + gradient)",
            "kernel_ms": kern_ms, "t_roof_ms": gr["t_roof_ms"], "tap_bytes_per_eval": tap,
            "hbm": {"compulsory_bytes": gr["hbm_compulsory_bytes"], "t_ms": gr["t_hbm_ms"],
                    "peak_gbs": hbm_peak, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                    "compulsory_frac_of_kernel_time": gr["t_hbm_ms"] / kern_ms,
                    "dram_gbs_of_traffic": None if traffic is None else traffic / (kern_ms * 1e-3) / 1e9,
                    "dram_frac": None if traffic is None else traffic / (kern_ms * 1e-3) / 1e9 / hbm_peak,
                    "traffic_over_compulsory": None if traffic is None else traffic / gr["hbm_compulsory_bytes"]}}


def gather_roofline(epo, wl, info, evals, kern_ms, hbm_peak):
    """The edge kernel against max(compulsory HBM time, gather time): the first term moves
    every record and map once at the measured HBM bandwidth; the second serves one 2x2
    footprint per evaluation at the best rate of the library's gather probe (both fetch
    forms, scattered and warp-coherent positions, on an L2-resident set of maps of the
    workload's size and type)."""
    sc = wl.scenes[0]
    W, H = int(sc.W[0]), int(sc.H[0])
    s_map = 2 if wl.mixed else 4
    n_maps = int(max(1, min(sc.n_views, (48 << 20) // (W * H * s_map))))
    rates = {}
    for g, gname in ((epo.EPO_GATHER_LDG, "ldg"), (epo.EPO_GATHER_TEX, "tex")):
        for pat, pname in ((0, "scattered"), (1, "warp_coherent")):
            rates[f"{gname}_{pname}"] = epo._binding.epo_gather_probe(
                n_maps, W, H, epo.EPO_BF16 if wl.mixed else epo.EPO_F32, g, pat, 1 << 26, 7)
    best = max(rates.values())
    hbm_bytes = info.record_bytes + info.map_bytes
    t_hbm = hbm_bytes / (hbm_peak * 1e9) * 1e3
    t_gather = evals / best * 1e3
    t_roof = max(t_hbm, t_gather)
    return {"t_roof_ms": t_roof, "kernel_ms": kern_ms, "frac": t_roof / kern_ms,
            "t_hbm_ms": t_hbm, "hbm_compulsory_bytes": int(hbm_bytes), "t_gather_ms": t_gather,
            "gather_footprints_per_s": rates, "probe": f"{n_maps} maps of {W}x{H} "
            f"{'bf16' if wl.mixed else 'f32'}, 2^26 footprints per launch, median of 7"}


ACC_STEPS = 100  # optimisation steps behind the final-accuracy comparisons


def viewgraph_leg(epo, torch, wl, stride=4):
    """Viewgraph estimation (Section 3, Eq. 2): every ordered pair's round-trip fraction over
    a grid of source pixels, on the GPU in FP64, at the initial poses and depths."""
    sc = wl.scenes[0]
    depth = torch.cat([torch.from_numpy(d).reshape(-1) for d in sc.depth]).cuda()
    run = lambda: epo.build_viewgraph(sc.W, sc.H, sc.K, sc.T_init, depth, stride=stride, tau=3.0, min_frac=0.125)
    run()
    n = 5
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n):
        frac, pairs = run()
    ms = 1e3 * (time.perf_counter() - t0) / n
    grid = sum(((int(w) + stride - 1) // stride) * ((int(h) + stride - 1) // stride) for w, h in zip(sc.W, sc.H))
    trips = grid * (sc.n_views - 1)
    return {"ms": ms, "round_trips": trips, "round_trips_per_s": trips / (ms * 1e-3), "grid_stride": stride,
            "tau_px": 3.0, "min_frac": 0.125, "pairs_kept": int(len(pairs)),
            "pairs_candidate": sc.n_views * (sc.n_views - 1),
            "note": "wall time of epo_build_viewgraph (FP64 round trips, host copy of the fraction matrix)"}


def refine_leg(epo, torch, wl, parts, dtypes, lr, evals, args, flush_l2, stream, sched):
    """Focal and per-pixel depth refinement (Eqs. 4-5): the objective with its gradient for
    the poses, the focal scales and every edge pixel's depth parameters, through the public
    call (one fused pass storing every sample's d(rho)/dz, then the depth kernel; host outputs),
    at a random small refinement; and the full refinement step (Algorithm 2 with the camera and
    depth modules) as graph steps."""
    def refined(**o):
        h = epo.Scene(parts, record_dtype=dtypes[0], map_dtype=dtypes[1],
                      options=epo.default_options(refine=1, **lr, **o), on_device=True)
        h.set_poses(wl.T_init)
        info = h.info()
        rng = np.random.default_rng(0)
        epo._binding.epo_set_refinement(h.handle, rng.normal(0, 0.005, info.n_views),
                                        1.0 + rng.normal(0, 0.005, info.n_records).astype(np.float32),
                                        rng.normal(0, 0.02, info.n_records).astype(np.float32))
        return h, info

    sched = {k: v for k, v in sched.items() if k != "records_per_thread"}
    hs, info_s = refined(lr_focal=1e-3, lr_depth=1e-3, **sched)
    for _ in range(3):
        hs.step_async(1)
    torch.cuda.synchronize()
    n = max(5, min(args.steps, 50))
    step_ms = float(np.mean(time_steps(hs, n, flush_l2, stream, torch)))
    step = {"value": evals / (step_ms * 1e-3), "unit": UNIT, "ms_per_step": step_ms, "iterations": n,
            "kernels_per_step": int(info_s.kernels_per_step),
            "note": "graph steps with lr_focal = lr_depth = 1e-3 and no schedule (the depth module steps "
                    "every step): fused pass with per-sample d(rho)/dz, pose + focal Adam, depth kernel (Adam)"}
    del hs
    h, info = refined()
    call = lambda: epo._binding.epo_refine_loss_and_grad(h.handle, info.n_scenes, info.n_views, info.n_records)
    for _ in range(3):
        call()
    n = max(5, min(args.steps, 50))
    tot = 0.0
    for k in range(n):
        flush_l2(k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        call()
        tot += time.perf_counter() - t0
    ms = 1e3 * tot / n
    return {"value": evals / (ms * 1e-3), "unit": UNIT, "ms_per_evaluation": ms, "iterations": n,
            "passes_per_evaluation": 1, "kernels_per_evaluation": 5,
            "d2h_bytes_per_evaluation": int(8 * info.n_scenes + 56 * info.n_views + 8 * info.n_records),
            "note": "wall time of epo_refine_loss_and_grad (fused pass, depth kernel, host copies of all gradients)",
            "step": step}


def pose_mlp_leg(epo, torch, wl, parts, dtypes, lr, evals, args, flush_l2, stream, sched):
    """The paper's pose parameterisation (Eq. 3: one MLP per scene, Gram-Schmidt, translation
    offsets, AdamW with warm-up and cosine decay) as graph steps: the fused pass, the pose
    kernel's gradient, the MLP's backward, AdamW and forward."""
    import synth
    B = epo._binding
    h = epo.Scene(parts, record_dtype=dtypes[0], map_dtype=dtypes[1], on_device=True,
                  options=epo.default_options(pose_param=B.EPO_POSE_MLP, **lr, **sched))
    h.set_poses(wl.T_init)
    B.epo_set_pose_mlp(h.handle, np.concatenate([synth.pose_mlp_init(20260100 + k) for k in range(h.info().n_scenes)]))
    for _ in range(3):
        h.step_async(1)
    torch.cuda.synchronize()
    n = max(5, min(args.steps, 50))
    ms = float(np.mean(time_steps(h, n, flush_l2, stream, torch)))
    return {"value": evals / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "iterations": n,
            "kernels_per_step": int(h.info().kernels_per_step),
            "note": "graph steps of the MLP parameterisation (per-scene MLP 12-128x5-12 in FP32, "
                    "Gram-Schmidt and poses in FP64), Kaiming-initialised, inside the warm-up"}


def autograd_leg(epo, torch, s, T_init, evals, args, flush_l2, stream):
    """Forward + adjoint through the autograd function at the current poses (two passes over
    the samples: the adjoint recomputes every projection instead of storing per-sample
    Jacobians), and the device memory this takes against a stored-Jacobian variant."""
    s.set_poses(T_init)
    xi = torch.zeros((s.n_views, 6), dtype=torch.float64, device="cuda", requires_grad=True)
    for _ in range(3):
        epo.EdgeLoss.apply(xi, s).sum().backward()
    xi.grad = None
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    n = max(5, min(args.steps, 50))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for k in range(n):
        flush_l2(k)
        ev[k][0].record(stream)
        epo.EdgeLoss.apply(xi, s).sum().backward()
        ev[k][1].record(stream)
        xi.grad = None
    torch.cuda.synchronize()
    ms = float(np.mean([x.elapsed_time(y) for x, y in ev]))
    info = s.info()
    return {"value": evals / (ms * 1e-3), "unit": UNIT, "ms_per_forward_backward": ms, "iterations": n,
            "torch_peak_bytes_above_inputs": int(torch.cuda.max_memory_allocated() - base),
            "library_device_bytes": int(info.device_bytes),
            "inputs_bytes": int(info.record_bytes + info.map_bytes),
            "stored_jacobian_bytes": int(evals * 14 * 4),
            "note": "stored-Jacobian variant: per evaluation d(rho)/d(xi_i), d(rho)/d(xi_j) (2 x 6 FP32), "
                    "rho and the validity flag, on top of the same inputs"}


def plain_per_scene_leg(epo, torch, wl, s, parts, dtypes, lr, evals, args, flush_l2, stream):
    """The per-scene plain form: one handle per scene with the default schedule, the same
    kernels launched one by one from the host each step (host-side synchronisation per
    scene), against the batched graph step; then both forms run ACC_STEPS steps from the
    initial poses and their final pose errors are compared."""
    hs = [epo.Scene([p], record_dtype=dtypes[0], map_dtype=dtypes[1],
                    options=epo.default_options(**lr), on_device=True) for p in parts]
    for h, sc in zip(hs, wl.scenes):
        h.set_poses(sc.T_init)
        h.step_plain(1)
    n = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for k in range(n):
        flush_l2(k)
        e0.record(stream)
        for h in hs:
            h.step_plain(1)
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    plain_ms = tot / n
    # equal final accuracy: both forms from the initial poses, ACC_STEPS steps
    s.set_poses(wl.T_init)
    s.set_state(0)
    s.step(ACC_STEPS)
    Tb = s.get_poses()
    Tp = []
    for h, sc in zip(hs, wl.scenes):
        h.set_poses(sc.T_init)
        h.set_state(0)
        h.step_plain(ACC_STEPS)
        Tp.append(h.get_poses())
    Tp = np.concatenate(Tp)
    del hs
    r0, t0 = pose_errors(wl.T_init, wl.scenes)
    rb, tb = pose_errors(Tb, wl.scenes)
    rp, tp = pose_errors(Tp, wl.scenes)
    return {"value": evals / (plain_ms * 1e-3), "unit": UNIT, "ms_per_step": plain_ms, "steps": n,
            "schedule": "library default (block 256, 2 records per thread, plain loads), no autotuning",
            "speedup_of_batched_graph_step": None,
            "final_accuracy": {"steps": ACC_STEPS, "initial_rot_deg": r0, "initial_trans_frac": t0,
                               "batched_graph_rot_deg": rb, "batched_graph_trans_frac": tb,
                               "plain_per_scene_rot_deg": rp, "plain_per_scene_trans_frac": tp,
                               "max_abs_pose_difference": float(np.abs(Tb - Tp).max())}}


def fp32_form_leg(epo, torch, wl, s, scene, lr, evals, args, flush_l2, stream):
    """The same scene with FP32 maps and records (autotuned the same way): its step
    throughput, and both forms' final pose errors after ACC_STEPS steps."""
    parts32 = wl.parts(epo, torch, mixed=False)
    s32 = scene(epo.default_options(autotune=2, **lr), prts=parts32, dt=wl.dtypes(epo, mixed=False))
    s32.set_poses(wl.T_init)
    s32.autotune()
    for _ in range(3):
        s32.step_async(1)
    s32.set_poses(wl.T_init)
    s32.set_state(0)
    ms32 = float(np.mean(time_steps(s32, max(5, min(args.steps, 50)), flush_l2, stream, torch)))
    res = {}
    for name, h in (("bf16_f16", s), ("fp32", s32)):
        h.set_poses(wl.T_init)
        h.set_state(0)
        h.step(ACC_STEPS)
        res[name] = h.get_poses()
    r0, t0 = pose_errors(wl.T_init, wl.scenes)
    ra, ta = pose_errors(res["bf16_f16"], wl.scenes)
    rf, tf = pose_errors(res["fp32"], wl.scenes)
    sc = wl.scenes[0]
    Ta, Tf = res["bf16_f16"].reshape(-1, 3, 4), res["fp32"].reshape(-1, 3, 4)
    dR = [np.degrees(np.arccos(np.clip((np.trace(a[:, :3] @ f[:, :3].T) - 1) / 2, -1, 1))) for a, f in zip(Ta, Tf)]
    dC = [np.linalg.norm(-a[:, :3].T @ a[:, 3] + f[:, :3].T @ f[:, 3]) / sc.scale for a, f in zip(Ta, Tf)]
    return {"value": evals / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32,
            "final_accuracy": {"steps": ACC_STEPS, "initial_rot_deg": r0, "initial_trans_frac": t0,
                               "bf16_f16_rot_deg": ra, "bf16_f16_trans_frac": ta,
                               "fp32_rot_deg": rf, "fp32_trans_frac": tf,
                               "max_rot_deg_between_forms": float(np.max(dR)),
                               "max_trans_frac_between_forms": float(np.max(dC))}}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
