"""Benchmark: INR-CT stochastic gradient steps per second on one GB300 (or N replicas).

One step is Algorithm 1 of the paper followed by an Adam update, through the
library's grad_step: grid evaluation of the INR (tcgen05 BF16 MLP), Joseph
projection with the LS loss epilogue, exact adjoint backprojection, the fused
residual-weighted VJP at |I| sampled points, weight-gradient GEMM, FP64
reduction, Adam.  Workload (default, the largest single-GPU configuration): 501^3 cone
beam, 60 views over 360 deg, 768 x 768 flat panel, SOD/SDD 1000/1500, Fourier features 512
(sigma 8) + 5 x 256 ReLU, |I| = 2^22, synthetic 40-ellipsoid phantom with 1 % noise.  The same
line carries, under "fan2d_512_siren256", the figures of the 512^2 fan beam workload (90 views,
729 curved bins, SIREN 5 x 256, |I| = n/4).

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead.
Under torchrun every rank runs an independent replica (weak scaling, no
data-path collective); the timed region is bracketed by a barrier and the
slowest rank's time is reported.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "INR-CT grad steps/s, proj+backproj GRays/s; BF16 vs FP32 at <=1e-2 grad err"
L2_BYTES = 129 * 1024 * 1024
BATCHED = "batched16_siren128"
HEADLINE = "cone3d_501_ffn512"       # the default workload: the largest single-GPU configuration
SECONDARY = "fan2d_512_siren256"     # carried in the default line as an extra key
VJP_CHUNK = 1 << 20          # points per VJP chunk (the library's scratch unit)
# FP32 FMA peak of the SIMT path: 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x 2.07 GHz
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=HEADLINE)
    p.add_argument("--no-secondary", action="store_true",
                   help=f"default workload only: skip the {SECONDARY} figures carried in the line")
    p.add_argument("--secondary-steps", type=int, default=1000, help=f"timed steps of {SECONDARY}")
    p.add_argument("--only", choices=["projector", "eval", "vjp"], default=None,
                   help="time one stage alone on the workload (P and P^T; the grid evaluation; the VJP "
                        "at |I| points), e.g. for a profiler")
    p.add_argument("--grid-n", type=int, default=None,
                   help="with --only eval/vjp: a grid of this side instead of the workload's (same network)")
    p.add_argument("--prec", default="bf16", choices=["bf16", "fp32"])
    p.add_argument("--frac", type=float, default=None, help="|I|/n (default: the workload's)")
    p.add_argument("--loss", default="ls", choices=["ls", "fls"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=200)
    p.add_argument("--no-fp32", action="store_true", help="skip the FP32 path and the BF16/FP32 gradient check")
    p.add_argument("--fp32-steps", type=int, default=10)
    p.add_argument("--no-fractions", action="store_true", help="skip the |I|/n = 1.0 and 0.05 step rates")
    p.add_argument("--ref-seconds", type=float, default=120.0,
                   help="--impl reference: host seconds the timed oracle samples take in total")
    p.add_argument("--subsets", type=int, default=1,
                   help="ordered subsets: step t uses interleaved view subset t mod S (Sec. 3)")
    p.add_argument("--plan", default=None, metavar="SEG,BP_SPLITS,ZC",
                   help="pin this projector launch plan instead of running the autotuner")
    return p.parse_args()


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# oracle timing (cpu_baseline and the reference arm)
# ----------------------------------------------------------------------------
def oracle_sample(w, frac: float, seed: int = 0) -> float:
    """Extrapolated seconds of one full oracle step, from one sample covering about
    `frac` of it: the forward on frac*n grid points, P and P^T on max(1, frac*V)
    views, the estimator on frac*|I| points, and Adam on all of theta.  Each part
    scales linearly in what it covers, so each is divided by its own fraction."""
    import oracle as O
    from paper_2604_09884_gb300 import synth
    g, a = w.geom, w.arch
    Vs = max(1, int(round(g.V * frac)))
    og = O.Geometry(g.kind, g.N, Vs, g.A, g.B, g.du, g.dv, g.sod, g.sdd, g.angle0,
                    g.span * Vs / g.V)
    B = synth.fourier_matrix(a.n_feat, a.d, a.sigma, seed) if a.kind == "ffn" else None
    oa = O.Arch(a.kind, a.d, a.width, a.n_hidden, a.n_feat, B, a.omega0, hash_levels=a.hash_levels,
                hash_feats=a.hash_feats, hash_log2_T=a.hash_log2_T, hash_base=a.hash_base,
                hash_growth=a.hash_growth)
    theta = synth.init_theta(a, seed)
    n_pts = max(1, int(g.n * frac))
    n_I = max(1, int(w.batch * frac))
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    f = O.forward(oa, theta, O.grid_coords(g.d, g.N, np.arange(n_pts)), N=g.N)
    t1 = time.perf_counter()
    img = np.zeros(g.n)
    img[:n_pts] = f
    z = O.project(og, img)
    L, r = O.ls_loss(z, np.zeros_like(z))
    v = O.backproject(og, r)
    t2 = time.perf_counter()
    I = rng.choice(g.n, n_I, replace=False)
    ghat = O.vjp(oa, theta, O.grid_coords(g.d, g.N, I), (g.n / w.batch) * v[I], N=g.N)
    t3 = time.perf_counter()
    st = O.AdamState(np.zeros_like(theta), np.zeros_like(theta))
    O.adam_step(theta, ghat, st, lr=w.lr)
    t4 = time.perf_counter()
    return ((t1 - t0) * g.n / n_pts + (t2 - t1) * g.V / Vs + (t3 - t2) * w.batch / n_I + (t4 - t3))


def oracle_sample_any(w, frac: float, seed: int = 0) -> float:
    """oracle_sample for one workload, or summed over a batch of problems (a list)."""
    if isinstance(w, list):
        return sum(oracle_sample(q, frac, seed) for q in w)
    return oracle_sample(w, frac, seed)


def oracle_frac(w, budget_s: float, frac_max: float) -> float:
    """A sample fraction for which one oracle sample takes about budget_s / 4 seconds,
    found from a tiny first sample (which also builds and warms the C projector)."""
    q = w[0] if isinstance(w, list) else w
    f0 = min(frac_max, max(1.0 / 65536, 2048.0 / q.geom.n))
    t = time.perf_counter()
    oracle_sample_any(w, f0)
    dt = max(time.perf_counter() - t, 1e-3)
    return min(frac_max, max(f0, f0 * (budget_s / 4) / dt))


def oracle_rate(w, budget_s: float, frac_max: float):
    """(steps/s, samples timed, fraction per sample) of the oracle within about budget_s seconds."""
    frac = oracle_frac(w, budget_s, frac_max)
    total, k, t0 = 0.0, 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s or k == 0:
        total += oracle_sample_any(w, frac, seed=k)
        k += 1
    return k / total, k, frac


# ----------------------------------------------------------------------------
def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of every rank's x (the slowest rank's time); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, seconds: float, world: int, device):
    """Whole-job throughput: every rank's units over the slowest rank's time.
    Returns (rate, slowest seconds)."""
    slowest = max_over_ranks(seconds, world, device)
    return world * units_per_rank / slowest, slowest


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    # each step is one oracle sample of a fraction of the step (extrapolated to the whole
    # step part by part), sized so that the whole --steps run takes about two minutes
    steps = max(1, args.steps)
    frac = oracle_frac(w, 4.0 * args.ref_seconds / (steps + 2), 1 / 16)
    for _ in range(max(1, min(args.warmup, 2))):
        oracle_sample_any(w, frac)
    total = 0.0
    for k in range(steps):
        total += oracle_sample_any(w, frac, seed=k)
    value = steps / total
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": ({"workload": BATCHED, "problems": len(w)} if isinstance(w, list)
                       else {"workload": w.name, "note": w.note, "batch": w.batch}),
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{steps} samples of about {frac:.4g} of a step each (forward "
                                       "on that fraction of the grid, P/P^T on that fraction of "
                                       "the views (at least one), VJP on that fraction of |I|), each "
                                       "part extrapolated linearly to the full step"},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def recorded_traffic(kernel_key: str, workload: str):
    """DRAM bytes per launch of a kernel from the committed ncu record, or None when
    there is none or the kernel's source file changed since it was captured."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(f"{kernel_key}@{workload}")
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["source_sha256"]:
        return None
    return rec["dram_bytes_per_launch"]


def mlp_flops(a, pts, vjp):
    """Tensor-core FLOPs of the MMA stages for `pts` points."""
    shapes = a.layer_shapes()
    first = 1 if a.kind == "siren" else 0
    fwd = sum(o * i for o, i in shapes[first:-1])
    if not vjp:
        return 2.0 * pts * fwd
    bwd = sum(o * i for o, i in shapes[1:-1])
    return 2.0 * pts * (fwd + bwd)


def dw_flops(a, pts):
    shapes = a.layer_shapes()
    return 2.0 * pts * sum(o * i for o, i in shapes[:-1] if i >= 64)


def run_batched(args, probs, rank, world, local, dev):
    """The batched workload: 16 uneven 2-D problems stepped together by one graph launch."""
    import torch

    from paper_2604_09884_gb300 import inrct, synth
    arch = probs[0].arch
    mlp = inrct.mlp_desc(arch, inrct.BF16, device=dev)
    n_sets = 4
    state, idx_host, idx_dev = [], [], []
    for k, w in enumerate(probs):
        g = w.geom
        seed = w.seed + 1000 * rank
        x_true = torch.tensor(synth.phantom(g.d, g.N, w.n_shapes, seed).reshape(-1), dtype=torch.float32,
                              device=dev)
        y = torch.tensor(synth.noisy(inrct.project(g, x_true).cpu().numpy(), w.noise, seed + 1), device=dev)
        theta = torch.tensor(synth.init_theta(arch, seed + 3), dtype=torch.float32, device=dev)
        n_idx = w.batch
        state.append({"geom": g, "theta": theta, "y": y, "idx": torch.empty(n_idx, dtype=torch.int32, device=dev),
                      "scale": g.n / n_idx, "m": torch.zeros_like(theta), "s": torch.zeros_like(theta),
                      "loss": torch.zeros(1, dtype=torch.float64, device=dev)})
        hs = [torch.from_numpy(synth.index_set(g.n, n_idx, seed + 10 + j)).pin_memory() for j in range(n_sets)]
        idx_host.append(hs)
        idx_dev.append([h.to(dev) for h in hs])
    batch = inrct.Batch(mlp, state, inrct.adam(lr=probs[0].lr), device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def set_idx(t):
        for k, q in enumerate(state):
            q["idx"].copy_(idx_dev[k][t % n_sets], non_blocking=True)

    t = 0
    for _ in range(args.warmup):
        t += 1
        set_idx(t)
        batch.step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    l0 = inrct.launch_count()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            t += 1
            starts[k].record(stream)
            set_idx(t)                      # a new index set per problem and step (device copies)
            batch.step()
            ends[k].record(stream)
        torch.cuda.synchronize()
    launches = inrct.launch_count() - l0
    value, total_s = job_rate(args.steps, sum(st.elapsed_time(en) for st, en in zip(starts, ends)) / 1000.0,
                              world, dev)
    ms_per_step = 1000.0 * total_s / args.steps

    # end to end: index sets from pinned host memory, losses back to the host
    loss_host = torch.zeros(len(state), dtype=torch.float64).pin_memory()
    loss_dev = torch.zeros(len(state), dtype=torch.float64, device=dev)
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        t += 1
        for k, q in enumerate(state):
            q["idx"].copy_(idx_host[k][t % n_sets], non_blocking=True)
        batch.step()
        for k, q in enumerate(state):
            loss_dev[k:k + 1].copy_(q["loss"])
        loss_host.copy_(loss_dev, non_blocking=True)
    torch.cuda.synchronize()
    e2e_value = world * e2e_steps / (time.perf_counter() - t0)
    peak_mem = torch.cuda.max_memory_allocated(dev)

    # dominant kernel: the same problems stepped one by one with the stage profile on
    prof = 4
    ws = [torch.empty(inrct.step_ws_bytes(q["geom"], mlp, q["idx"].numel()), dtype=torch.uint8, device=dev)
          for q in state]
    th = [q["theta"].clone() for q in state]
    mm = [q["m"].clone() for q in state]
    ss = [q["s"].clone() for q in state]
    inrct.profile_begin(prof * len(state))
    for r in range(prof):
        for k, q in enumerate(state):
            inrct.grad_step(q["geom"], mlp, th[k], q["y"], q["idx"], q["scale"],
                            inrct.adam(lr=probs[0].lr, t=t + 1 + r), mm[k], ss[k], None, None, ws[k])
    stages, nprof = inrct.profile_end()
    per_batch = {k: v / prof for k, v in stages.items()}   # ms per batched step, summed over problems
    n_eval = sum(q["geom"].n for q in state)
    n_vjp = sum(q["idx"].numel() for q in state)
    f_eval = mlp_flops(arch, n_eval, vjp=False)
    f_vjp = mlp_flops(arch, n_vjp, vjp=True)
    dominant = max(("eval_mlp_kernel", "vjp_mlp_kernel"), key=lambda k: per_batch[k])
    flops = f_eval if dominant == "eval_mlp_kernel" else f_vjp
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    achieved = flops / per_batch[dominant] / 1e9
    roofline = {"kernel": "mlp_tile_kernel (" + ("grid evaluation" if dominant == "eval_mlp_kernel" else "VJP")
                + "), summed over the 16 problems, timed with the problems stepped one by one",
                "bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                "frac": achieved / bf16_peak,
                "peak_source": ("measured" if peaks else "fallback") + " (bf16 burst)", "traffic": None}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, k, fr = oracle_rate(probs, budget_s=20.0, frac_max=1 / 32)
        cpu = {"value": rate, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{k} samples of about {fr:.3g} of every problem's step (forward, P/P^T on at "
                         "least one view, VJP), each part extrapolated linearly, summed over the 16 "
                         "problems"}
    if rank == 0:
        sizes = sorted(q["geom"].N for q in state)
        line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                "data": "synthetic",
                "config": {"workload": BATCHED, "problems": len(state), "grid_sizes": sizes,
                           "pixels_total": n_eval, "batch_total": n_vjp,
                           "note": "16 independent 2-D par/fan problems, SIREN 3x128 each, |I| = n/4; "
                                   "one CUDA graph launch per step (a branch per problem)",
                           "l2": "flushed between timed steps (untimed 258 MB write)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "problem_steps_per_s": value * len(state),
                "stage_ms_sequential": per_batch, "roofline": roofline,
                "e2e": {"value": e2e_value, "unit": "steps/s",
                        "h2d_bytes_per_step": int(sum(q["idx"].numel() * 4 for q in state)),
                        "d2h_bytes_per_step": 8 * len(state)},
                "gpu_launches": int(launches), "clocks": clk.summary(), "cpu_baseline": cpu,
                "peak_mem_bytes": int(peak_mem),
                "loss_last": [float(x) for x in loss_host.tolist()]}
        print(json.dumps(line), flush=True)
    batch.close()


def projector_roofline(g, m_step, per, hbm_peak, peak_src, name, zc=None, seg=None):
    """Rates of P and P^T from the stage profile against the measured HBM bandwidth, under both
    byte models: compulsory bytes (P: image in, sinogram, residual out and y in: 4n + 12m;
    P^T: sinogram in, image out: 4n + 4m) and the per-view streaming model (the image read once
    per view, 4nV + 4m, and 12m / 4m of sinogram traffic), with the DRAM bytes per launch of the
    committed ncu record where one matches the current source (the cone record is that of the
    kernel the plan runs: seg = 1 the row-patch projector, zc = 0 the column adjoint)."""
    out = {}
    V = g.V
    for key, stage, sino_bytes, traffic_key in (("project", "project_loss", 12.0, ("project3d_rows_kernel" if seg == 1
                                                  else "project3d_kernel") if g.d == 3 else "project2d_kernel"),
                                                ("backproject", "backproject", 4.0,
                                                 ("backproject3d_col_kernel" if zc == 0 else "backproject3d_kernel")
                                                 if g.d == 3 else "backproject2d_tile_kernel")):
        ms = per[stage]
        if ms <= 0:
            continue
        comp = 4.0 * g.n + sino_bytes * m_step
        stream = 4.0 * g.n * V + sino_bytes * m_step
        out[key] = {"ms": ms, "GRays/s": m_step / ms / 1e6,
                    "compulsory_bytes": comp, "streaming_bytes": stream,
                    "achieved_GB/s_compulsory": comp / ms / 1e6, "achieved_GB/s_streaming": stream / ms / 1e6,
                    "frac_compulsory": comp / ms / 1e6 / hbm_peak, "frac_streaming": stream / ms / 1e6 / hbm_peak,
                    "peak": hbm_peak, "peak_source": f"{peak_src} (HBM copy)",
                    "traffic": recorded_traffic(traffic_key, name)}
    return out


def build_problem(w, rank, dev, prec_name):
    """The workload's synthetic problem, resident on the device: phantom, noisy data, network."""
    import torch

    from paper_2604_09884_gb300 import inrct, synth
    g, a = w.geom, w.arch
    seed = w.seed + 1000 * rank                      # every replica its own problem
    x_true = torch.tensor(synth.phantom(g.d, g.N, w.n_shapes, seed).reshape(-1), dtype=torch.float32,
                          device=dev)
    y_clean = inrct.project(g, x_true)
    y = torch.tensor(synth.noisy(y_clean.cpu().numpy(), w.noise, seed + 1), device=dev)
    del y_clean
    B = synth.fourier_matrix(a.n_feat, a.d, a.sigma, seed + 2) if a.kind == "ffn" else None
    prec = inrct.BF16 if prec_name == "bf16" else inrct.FP32
    mlp = inrct.mlp_desc(a, prec, B, device=dev)
    theta = torch.tensor(synth.init_theta(a, seed + 3), dtype=torch.float32, device=dev)
    return {"seed": seed, "x_true": x_true, "y": y, "B": B, "mlp": mlp, "theta": theta}


def run_stage_only(args, w, rank, world, local, dev):
    """One stage alone, CUDA-event timed per call with L2 flushed in between (used by the
    profiles): P and P^T on the workload's geometry (tuned plans, or --plan), or the grid
    evaluation / the VJP at |I| = the workload's batch (scaled to --grid-n) with the workload's
    network in its precision."""
    import torch

    from paper_2604_09884_gb300 import inrct, synth
    g = w.geom
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    info = {}
    if args.only == "projector":
        x = torch.tensor(synth.phantom(g.d, g.N, w.n_shapes, w.seed).reshape(-1), dtype=torch.float32, device=dev)
        if args.plan:
            inrct.tune_set(g, *(int(q) for q in args.plan.split(",")))
            info["plan"] = inrct.tune_plan(g)
        else:
            info["plan"] = inrct.tune(g, device=dev)
        y = inrct.project(g, x)
        fns = (("project", lambda: inrct.project(g, x, y)), ("backproject", lambda: inrct.backproject(g, y)))
        units = g.m
        info.update(rays=g.m, voxels=g.n)
    else:
        a = w.arch
        N = args.grid_n or g.N
        n = N ** g.d
        B = synth.fourier_matrix(a.n_feat, a.d, a.sigma, w.seed + 2) if a.kind == "ffn" else None
        mlp = inrct.mlp_desc(a, inrct.BF16 if args.prec == "bf16" else inrct.FP32, B, device=dev)
        theta = torch.tensor(synth.init_theta(a, w.seed + 3), dtype=torch.float32, device=dev)
        if args.only == "eval":
            fns = (("eval", lambda: inrct.inr_eval_grid(mlp, theta, N)),)
            units = n
            info.update(points=n, flops=mlp_flops(a, n, vjp=False))
        else:
            nI = max(1, min(n, int(round(w.batch * n / g.n))))
            idx = torch.from_numpy(synth.index_set(n, nI, w.seed + 10)).to(dev)
            v = torch.tensor(synth.uniform(n, w.seed + 11), dtype=torch.float32, device=dev)
            fns = (("vjp", lambda: inrct.inr_weighted_vjp(mlp, theta, N, idx, v, n / nI)),)
            units = nI
            info.update(points=nI, flops=mlp_flops(a, nI, vjp=True) + dw_flops(a, nI))
        info.update(grid_n=N, precision=args.prec)
    res = {}
    for name, fn in fns:
        for _ in range(max(1, args.warmup)):
            fn()
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        med = statistics.median(ts)
        res[name] = {"ms_median": med, "ms_min": min(ts), "units_per_s": units / med * 1e3}
        if "flops" in info:
            res[name]["TFLOP/s"] = info["flops"] / med / 1e9
    inrct.device_status()
    if rank == 0:
        print(json.dumps({"mode": f"only {args.only}", "workload": w.name, **info, "calls": args.steps,
                          "timing": res, "note": "each call is the library entry point (workspace set-up "
                                                 "included); L2 flushed between calls"}), flush=True)


def run_single(args, w, rank, world, local, dev, steps, warmup, e2e_steps, cpu_budget, headline):
    """One workload: timed steps, end-to-end steps, and the figures of the line (rank 0 gets the
    line as a dict; other ranks None).  Large workloads (n > 2^24) compare against one FP32
    full gradient instead of timed FP32 steps and skip the |I|/n sweep."""
    import torch

    from paper_2604_09884_gb300 import inrct, synth
    g, a = w.geom, w.arch
    big = g.n > (1 << 24)
    torch.cuda.reset_peak_memory_stats(dev)          # the peak of this workload alone
    pb = build_problem(w, rank, dev, args.prec)
    x_true, y, B, mlp, theta = pb["x_true"], pb["y"], pb["B"], pb["mlp"], pb["theta"]
    seed = pb["seed"]
    m = torch.zeros_like(theta)
    s = torch.zeros_like(theta)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    n_idx = w.batch
    scale = g.n / n_idx
    ws = torch.empty(inrct.step_ws_bytes(g, mlp, n_idx), dtype=torch.uint8, device=dev)
    loss_kind = inrct.LOSS_FLS if args.loss == "fls" else inrct.LOSS_LS
    # index sets: a fresh uniform subset per step (drawn on the host, staged in HBM)
    n_sets = 4 if big else 16
    idx_host = [torch.from_numpy(synth.index_set(g.n, n_idx, seed + 10 + k)).pin_memory()
                for k in range(n_sets)]
    idx_dev = [t.to(dev) for t in idx_host]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    S = max(1, args.subsets)
    sub_g = [inrct.view_subset(g, S, k) for k in range(S)] if S > 1 else [g]
    sub_y = [inrct.view_subset_rows(g, y, S, k) for k in range(S)] if S > 1 else [y]
    sub_ws = [ws] if S == 1 else [torch.empty(inrct.step_ws_bytes(q, mlp, n_idx), dtype=torch.uint8, device=dev)
                                  for q in sub_g]
    # projector launch shapes: the library's autotuner, once per geometry, before any timing
    # (or a plan pinned on the command line, e.g. to reproduce a measurement's launch shapes)
    if args.plan:
        seg, bp, zc = (int(x) for x in args.plan.split(","))
        for q in sub_g:
            inrct.tune_set(q, seg, bp, zc)
        plans = [inrct.tune_plan(q) for q in sub_g]
    else:
        plans = [inrct.tune(q, device=dev) for q in sub_g]

    def step(t, idx):
        k = t % S
        inrct.grad_step(sub_g[k], mlp, theta, sub_y[k], idx, scale, inrct.adam(lr=w.lr, t=t), m, s, loss,
                        None, sub_ws[k], loss_kind)

    t = 0
    for _ in range(warmup):
        t += 1
        step(t, idx_dev[t % n_sets])
    torch.cuda.synchronize()
    inrct.device_status()

    # ---- timed region (device): inputs resident, L2 flushed between steps (untimed) ----
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    prof_steps = min(steps, 256)
    inrct.profile_begin(prof_steps)
    l0 = inrct.launch_count()
    with ClockSampler(local) as clk:
        for k in range(steps):
            flush.zero_()
            t += 1
            starts[k].record(stream)
            step(t, idx_dev[t % n_sets])
            ends[k].record(stream)
        torch.cuda.synchronize()
    launches = inrct.launch_count() - l0
    stages, nprof = inrct.profile_end()
    inrct.device_status()                            # no bounded wait gave up in the timed steps
    if world > 1:
        torch.distributed.barrier()
    step_ms = [st.elapsed_time(en) for st, en in zip(starts, ends)]
    value, total_s = job_rate(steps, sum(step_ms) / 1000.0, world, dev)
    ms_per_step = 1000.0 * total_s / steps

    # ---- end to end through the public API, host buffers, copies inside the timed region ----
    loss_host = torch.zeros(1, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(e2e_steps, steps))
    idx_stage = torch.empty_like(idx_dev[0])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        t += 1
        idx_stage.copy_(idx_host[t % n_sets], non_blocking=True)
        step(t, idx_stage)
        loss_host.copy_(loss, non_blocking=True)
    torch.cuda.synchronize()
    e2e_value, e2e_s = job_rate(e2e_steps, time.perf_counter() - t0, world, dev)
    peak_mem = torch.cuda.max_memory_allocated(dev)
    del idx_stage

    # ---- reconstruction error of the trained INR, and other subsampling fractions ----
    with torch.no_grad():
        img = inrct.inr_eval_grid(mlp, theta, g.N)
        mse = float(((img - x_true) ** 2).mean())
        del img
    fractions = {f"{n_idx / g.n:.4g}": {"steps_per_s": value / world, "batch": n_idx}}
    if not args.no_fractions and not big:
        for f in (1.0, 0.05):
            nI = max(1, int(round(f * g.n)))
            wsf = torch.empty(inrct.step_ws_bytes(g, mlp, nI), dtype=torch.uint8, device=dev)
            idxf = torch.from_numpy(synth.index_set(g.n, nI, seed + 99)).to(dev)
            thf, mf, sf = theta.clone(), torch.zeros_like(theta), torch.zeros_like(theta)
            kf = 20
            for tf in range(1, 3 + kf):
                if tf == 3:
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                inrct.grad_step(g, mlp, thf, y, idxf, g.n / nI, inrct.adam(lr=w.lr, t=tf), mf, sf, None, None,
                                wsf, loss_kind)
            e1 = torch.cuda.Event(enable_timing=True)
            e1.record(stream)
            torch.cuda.synchronize()
            fractions[f"{f:.4g}"] = {"steps_per_s": 1000.0 * kf / e0.elapsed_time(e1), "batch": nI,
                                     "timing": f"{kf} steps back to back, L2 not flushed"}
            del wsf

    # ---- the plain FP32 path and the BF16 / FP32 gradient agreement ----
    fp32 = None
    if args.prec == "bf16" and not args.no_fp32:
        mlp32 = inrct.mlp_desc(a, inrct.FP32, B, device=dev)

        def agree(ga, gb):
            return {"rel_l2": float(torch.linalg.norm(ga - gb) / torch.linalg.norm(gb)),
                    "cosine": float(torch.dot(ga, gb) / (torch.linalg.norm(ga) * torch.linalg.norm(gb)))}

        # one estimator at the current theta: v = P^T r of the FP32 image, the same index set
        img = inrct.inr_eval_grid(mlp32, theta, g.N)
        _, r, _ = inrct.project(g, img, y)
        del img
        vfull = inrct.backproject(g, r)
        del r
        g16 = inrct.inr_weighted_vjp(mlp, theta, g.N, idx_dev[0], vfull, scale)
        g32 = inrct.inr_weighted_vjp(mlp32, theta, g.N, idx_dev[0], vfull, scale)
        same_I = dict(agree(g16, g32), batch=n_idx, v="P^T (P f_theta - y) at the current theta")
        del g32
        torch.cuda.reset_peak_memory_stats(dev)
        idx_all = torch.arange(g.n, dtype=torch.int32, device=dev)
        ws32 = torch.empty(inrct.step_ws_bytes(g, mlp32, g.n), dtype=torch.uint8, device=dev)
        th32 = theta.clone()
        loss32 = torch.zeros(1, dtype=torch.float64, device=dev)
        if big:
            # the plain FP32 form once: the full gradient (|I| = n) at the current theta, timed
            gfull = torch.empty(a.p, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inrct.grad_step(g, mlp32, th32, y, idx_all, 1.0, None, None, None, loss32, gfull, ws32, loss_kind)
            e1.record(stream)
            torch.cuda.synchronize()
            k32, ms32 = 1, e0.elapsed_time(e1)
            full = dict(agree(g16, gfull), note="the BF16 estimator (|I| = batch, the same theta and v) against "
                                                "the FP32 full gradient (|I| = n): subsampling and precision")
            del gfull
        else:
            m32, s32 = torch.zeros_like(theta), torch.zeros_like(theta)
            for t32 in range(1, 3):
                inrct.grad_step(g, mlp32, th32, y, idx_all, 1.0, inrct.adam(lr=w.lr, t=t32), m32, s32, loss32,
                                None, ws32, loss_kind)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k32 = max(1, args.fp32_steps)
            e0.record(stream)
            for t32 in range(3, 3 + k32):
                inrct.grad_step(g, mlp32, th32, y, idx_all, 1.0, inrct.adam(lr=w.lr, t=t32), m32, s32, loss32,
                                None, ws32, loss_kind)
            e1.record(stream)
            torch.cuda.synchronize()
            ms32 = e0.elapsed_time(e1) / k32
            full = None
        inrct.device_status()
        fp32 = {"steps_per_s": 1000.0 / ms32, "ms_per_step": ms32, "batch": g.n, "steps": k32,
                "step_ws_bytes": int(ws32.numel()),
                "peak_mem_bytes": int(torch.cuda.max_memory_allocated(dev)),
                "peak_mem_note": "device peak during the FP32 steps, the BF16 run's buffers still allocated",
                "grad_bf16_vs_fp32": same_I}
        if full is not None:
            fp32["grad_bf16_estimator_vs_fp32_full"] = full
        del ws32, idx_all, th32, g16, vfull

    # ---- kernel rates from the stage profile (live, inside the timed steps) ----
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    peak_src = "measured" if peaks else "fallback"
    per = {k: v / max(nprof, 1) for k, v in stages.items()}
    kernels = {}
    f_eval = mlp_flops(a, g.n, vjp=False)
    # the VJP runs in chunks of at most VJP_CHUNK points; the profile marks bracket the
    # first chunk's tile kernel, everything after it (further chunks, all GEMMs) is the
    # "rest" stage
    first = min(n_idx, VJP_CHUNK)
    f_vjp = mlp_flops(a, first, vjp=True)
    f_dw = dw_flops(a, n_idx) + mlp_flops(a, n_idx - first, vjp=True)
    if per["eval_mlp_kernel"] > 0:
        kernels["eval_mlp_kernel"] = {"ms": per["eval_mlp_kernel"],
                                      "TFLOP/s": f_eval / per["eval_mlp_kernel"] / 1e9}
    if per["vjp_mlp_kernel"] > 0:
        kernels["vjp_mlp_kernel"] = {"ms": per["vjp_mlp_kernel"],
                                     "TFLOP/s": f_vjp / per["vjp_mlp_kernel"] / 1e9,
                                     "note": "algorithmic FLOPs; the ReLU networks' forward stages run "
                                             "three MMAs per product (split operands)" if a.kind == "ffn" else ""}
    if per["vjp_dw_gemm_reduce"] > 0:
        key = "vjp_dw_gemm_reduce" if n_idx <= VJP_CHUNK else "vjp_rest (further chunks + dW GEMMs)"
        kernels[key] = {"ms": per["vjp_dw_gemm_reduce"], "TFLOP/s": f_dw / per["vjp_dw_gemm_reduce"] / 1e9}
    m_step = g.m // S                                # rays per step (a view subset when S > 1)
    roof_proj = projector_roofline(g, m_step, per, hbm_peak, peak_src, w.name, plans[0]["zc"],
                                   plans[0]["seg"])
    pair_ms = per["project_loss"] + per["backproject"]
    dominant = max(("eval_mlp_kernel", "vjp_mlp_kernel"), key=lambda k: per[k])
    flops = f_eval if dominant == "eval_mlp_kernel" else f_vjp
    achieved = flops / per[dominant] / 1e9
    roofline = {"kernel": "mlp_tile_kernel (" + ("grid evaluation" if dominant == "eval_mlp_kernel"
                                                 else "VJP") + ")",
                "bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                "frac": achieved / bf16_peak, "peak_source": f"{peak_src} (bf16 burst)",
                "traffic": recorded_traffic("mlp_tile_kernel_" + ("eval" if dominant == "eval_mlp_kernel"
                                                                  else "vjp"), w.name)}
    if args.prec != "bf16":
        # FP32 SIMT path: FMA-bound at best (nominal peak from unit counts and the maximum clock)
        roofline = {"kernel": "simt_fwd_kernel + simt_bwd_kernel (" +
                              ("grid evaluation" if dominant == "eval_mlp_kernel" else "VJP") + ")",
                    "bound": "alu", "achieved": achieved, "peak": FP32_SIMT_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_SIMT_TFLOPS,
                    "peak_source": "nominal FP32 FMA rate (152 SMs x 128 lanes x 2 x 2.07 GHz)",
                    "traffic": recorded_traffic("simt_" + ("eval" if dominant == "eval_mlp_kernel" else "vjp"),
                                                w.name)}

    cpu = None
    if rank == 0 and world == 1 and cpu_budget > 0:
        rate, k, fr = oracle_rate(w, budget_s=cpu_budget, frac_max=1 / 16)
        cpu = {"value": rate, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{k} samples of about {fr:.3g} of a step each (forward on that fraction of "
                         "the grid, P/P^T on that fraction of the views (at least one), VJP on that "
                         "fraction of |I|), each part extrapolated linearly to the full step"}
    if rank != 0:
        return None
    return {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": steps, "warmup": warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if args.prec == "bf16" else "f32", "data": "synthetic",
            "config": {"workload": w.name, "note": w.note, "batch": n_idx,
                       "loss": args.loss, "precision": args.prec, "view_subsets": S,
                       "projector_plan": {k: plans[0][k] for k in ("seg", "bp_splits", "zc")},
                       "l2": "flushed between timed steps (untimed 258 MB write)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "gray_s_proj_backproj": m_step / pair_ms / 1e6 if pair_ms > 0 else None,
            "stage_ms": per, "kernels": kernels, "roofline": roofline, "roofline_projector": roof_proj,
            "e2e": {"value": e2e_value, "unit": "steps/s",
                    "h2d_bytes_per_step": int(idx_host[0].numel() * 4), "d2h_bytes_per_step": 8},
            "gpu_launches": int(launches), "clocks": clk.summary(), "cpu_baseline": cpu,
            "peak_mem_bytes": int(peak_mem), "step_ws_bytes": int(ws.numel()),
            "fp32_path": fp32, "fractions": fractions,
            "mse_vs_x_true": mse,
            "loss_last": float(loss_host.item())}


def main():
    args = parse()
    import torch

    from paper_2604_09884_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = synth.workloads()
    if args.workload == BATCHED:
        w = synth.batched_problems()
    elif args.workload not in wl:
        raise SystemExit(f"unknown workload {args.workload}; choose from {sorted(wl) + [BATCHED]}")
    else:
        w = wl[args.workload]
    if not isinstance(w, list) and w.arch.kind == "hash":
        args.prec = "fp32"                       # the hash-encoded INR has the FP32 path only
    if args.frac is not None and not isinstance(w, list):
        w.batch = max(1, int(round(args.frac * w.geom.n)))

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if isinstance(w, list):
        run_batched(args, w, rank, world, local, dev)
    elif args.only:
        run_stage_only(args, w, rank, world, local, dev)
    else:
        cpu_s = 0.0 if args.no_cpu_baseline else 15.0
        line = run_single(args, w, rank, world, local, dev, args.steps, args.warmup, args.e2e_steps, cpu_s,
                          headline=True)
        if w.name == HEADLINE and args.frac is None and not args.no_secondary and args.subsets == 1:
            # the 512^2 fan workload's figures, carried in the same line
            torch.cuda.empty_cache()
            sec = run_single(args, wl[SECONDARY], rank, world, local, dev, max(1, args.secondary_steps),
                             max(args.warmup, 20), 200, 0.0 if args.no_cpu_baseline else 10.0, headline=False)
            if rank == 0:
                line[SECONDARY] = {k: sec[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "config",
                                                       "roofline", "roofline_projector", "kernels", "stage_ms",
                                                       "e2e", "gpu_launches", "clocks", "cpu_baseline",
                                                       "peak_mem_bytes", "step_ws_bytes", "fp32_path",
                                                       "fractions", "mse_vs_x_true")}
        if rank == 0:
            print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
