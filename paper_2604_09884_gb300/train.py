"""Training driver: Algorithm 1 with Adam over many steps, metrics and checkpoints.

Every step is one call of the library's ``grad_step`` (grid evaluation, projection, loss,
backprojection, the estimator of Eq. 2 at a fresh index set, Adam).  This module only chooses
the index sets, keeps the Adam state, and reports:

- a JSON line per logged step: the loss at the incoming theta, the MSE of the INR image against
  the phantom (when one is given), the norm of the estimated gradient and the step's wall time;
- checkpoints holding theta, the Adam moments, the step index, the seed and the projector's launch
  plans.  Index set t is drawn from (seed, t) alone and loading a checkpoint pins its plan, so a
  run resumed from a checkpoint takes exactly the steps an uninterrupted run takes (bit for bit:
  every kernel of the step is deterministic, except the FP64 atomics of the hash-encoded INR's
  table gradient).

Usage (the 512^2 fan workload's comparison of the BF16 estimator at three subsampling fractions
with the plain FP32 form)::

    python -m paper_2604_09884_gb300.train --workload fan2d_512_siren256 --steps 500 \\
        --fracs 1.0,0.25,0.05 --fp32 --log-every 10 --out runs/fan512

The MSE and the norm are reporting only; they are computed with PyTorch on the library's outputs
and take no part in the step.
"""
from __future__ import annotations

import argparse
import json
import os
import time
from dataclasses import dataclass

import torch

from . import inrct, synth


@dataclass
class Problem:
    """A reconstruction problem on the device: geometry, data, and (optionally) the phantom."""
    geom: synth.GeomSpec
    y: torch.Tensor
    x_true: torch.Tensor | None = None


def make_problem(w: synth.Workload, device="cuda", seed: int | None = None) -> Problem:
    """The workload's synthetic problem: seeded phantom, y = P x_true plus the workload's noise."""
    g = w.geom
    s = w.seed if seed is None else seed
    x_true = torch.tensor(synth.phantom(g.d, g.N, w.n_shapes, s).reshape(-1), dtype=torch.float32, device=device)
    y_clean = inrct.project(g, x_true)
    y = torch.tensor(synth.noisy(y_clean.cpu().numpy(), w.noise, s + 1), device=device)
    return Problem(g, y, x_true)


class Trainer:
    """Algorithm 1 + Adam on one problem, with a fixed |I| per step.

    mlp: an ``inrct.MlpHandle`` (its precision selects the BF16 or the FP32 path); theta: the
    initial parameters (copied); n_idx: |I| (g.n for the plain full-gradient form); seed: the
    seed of the index sets.  Index set t is drawn on the device: the first |I| entries of a
    permutation of [0, n) from a generator seeded with seed * 1000003 + t, sorted.  subsets: S > 1
    takes the ordered-subsets form of Sec. 3, step t fitting interleaved view subset (t - 1) mod S
    (``inrct.view_subset``) with that subset's rows of the data; each subset keeps its own
    workspace, so its ray tables are built once.
    """

    def __init__(self, problem: Problem, mlp: inrct.MlpHandle, theta: torch.Tensor, n_idx: int, lr: float,
                 seed: int = 0, loss_kind: int = inrct.LOSS_LS, subsets: int = 1):
        g = problem.geom
        if not 1 <= n_idx <= g.n:
            raise ValueError(f"|I| = {n_idx} outside [1, {g.n}]")
        self.problem, self.mlp, self.n_idx, self.lr, self.seed = problem, mlp, int(n_idx), float(lr), int(seed)
        self.loss_kind = loss_kind
        self.subsets = S = int(subsets)
        self.sub_g = [inrct.view_subset(g, S, k) for k in range(S)] if S > 1 else [g]
        self.sub_y = [inrct.view_subset_rows(g, problem.y, S, k) for k in range(S)] if S > 1 else [problem.y]
        dev = theta.device
        self.theta = theta.detach().clone().contiguous()
        self.m = torch.zeros_like(self.theta)
        self.s = torch.zeros_like(self.theta)
        self.t = 0                                        # steps taken
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.grad = torch.zeros(mlp.p, dtype=torch.float64, device=dev)
        self.ws = [torch.empty(inrct.step_ws_bytes(q, mlp, self.n_idx), dtype=torch.uint8, device=dev)
                   for q in self.sub_g]

    def index_set(self, t: int) -> torch.Tensor:
        n, dev = self.problem.geom.n, self.theta.device
        if self.n_idx == n:
            return torch.arange(n, dtype=torch.int32, device=dev)
        gen = torch.Generator(device=dev)
        gen.manual_seed(self.seed * 1000003 + t)
        pick = torch.randperm(n, generator=gen, device=dev)[:self.n_idx]
        return torch.sort(pick).values.to(torch.int32)

    def step(self) -> None:
        """One step of Algorithm 1 followed by Adam (step index t + 1)."""
        k = self.t % self.subsets
        idx = self.index_set(self.t + 1)
        inrct.grad_step(self.sub_g[k], self.mlp, self.theta, self.sub_y[k], idx, self.problem.geom.n / self.n_idx,
                        inrct.adam(lr=self.lr, t=self.t + 1), self.m, self.s, self.loss, self.grad, self.ws[k],
                        self.loss_kind)
        self.t += 1

    def metrics(self) -> dict:
        """The last step's loss (at its incoming theta) and gradient norm (None before the first
        step), and the MSE of the current INR image against the phantom (None without one)."""
        mse = None
        if self.problem.x_true is not None:
            img = inrct.inr_eval_grid(self.mlp, self.theta, self.problem.geom.N)
            mse = float(((img - self.problem.x_true) ** 2).mean())
        stepped = self.t > 0
        return {"step": self.t, "loss": float(self.loss.item()) if stepped else None,
                "grad_norm": float(torch.linalg.norm(self.grad)) if stepped else None, "mse_vs_x_true": mse}

    # ---- checkpoints ----
    def state(self) -> dict:
        plans = [inrct.tune_plan(q) for q in self.sub_g]
        return {"theta": self.theta.clone(), "m": self.m.clone(), "s": self.s.clone(), "t": self.t,
                "seed": self.seed, "n_idx": self.n_idx, "lr": self.lr, "subsets": self.subsets,
                "plans": [(p["seg"], p["bp_splits"], p["zc"]) for p in plans]}

    def save(self, path: str) -> None:
        torch.save(self.state(), path)

    def load(self, path: str) -> None:
        st = torch.load(path, map_location=self.theta.device)
        if st["n_idx"] != self.n_idx or st["seed"] != self.seed or st["subsets"] != self.subsets:
            raise ValueError("checkpoint of another run (|I|, seed or view subsets differ)")
        self.theta.copy_(st["theta"])
        self.m.copy_(st["m"])
        self.s.copy_(st["s"])
        self.t = int(st["t"])
        self.lr = float(st["lr"])
        for q, plan in zip(self.sub_g, st["plans"]):
            inrct.tune_set(q, *plan)  # the summation order of P and P^T


def run(tr: Trainer, steps: int, log_every: int = 1, log=None, checkpoint: str | None = None,
        checkpoint_every: int = 0) -> list[dict]:
    """Take steps until tr.t == steps; return the logged metrics (also written to ``log``, a
    text file, one JSON object per line).  Wall time per step is measured over each logging
    interval on the host, with the device synchronised at its ends."""
    out = []
    if tr.t == 0:                                     # the starting point of the curve
        rec = {**tr.metrics(), "step_ms": None}
        out.append(rec)
        if log is not None:
            log.write(json.dumps(rec) + "\n")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    since = 0
    while tr.t < steps:
        tr.step()
        since += 1
        if tr.t % log_every == 0 or tr.t == steps:
            torch.cuda.synchronize()
            rec = tr.metrics()
            rec["step_ms"] = 1000.0 * (time.perf_counter() - t0) / since
            out.append(rec)
            if log is not None:
                log.write(json.dumps(rec) + "\n")
                log.flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            since = 0
        if checkpoint and checkpoint_every and tr.t % checkpoint_every == 0:
            tr.save(checkpoint)
    return out


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--workload", default="fan2d_512_siren256")
    p.add_argument("--steps", type=int, default=500)
    p.add_argument("--fracs", default="0.25", help="|I|/n of the BF16 runs, comma separated")
    p.add_argument("--fp32", action="store_true", help="also the plain FP32 form (|I| = n)")
    p.add_argument("--lr", type=float, default=None)
    p.add_argument("--log-every", type=int, default=10)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--subsets", type=int, default=1, help="ordered subsets of the views (Sec. 3)")
    p.add_argument("--out", default="runs", help="directory of the JSONL logs and checkpoints")
    a = p.parse_args(argv)
    w = synth.workloads()[a.workload]
    arch, g = w.arch, w.geom
    os.makedirs(a.out, exist_ok=True)
    prob = make_problem(w)
    B = synth.fourier_matrix(arch.n_feat, arch.d, arch.sigma, w.seed + 2) if arch.kind == "ffn" else None
    theta0 = torch.tensor(synth.init_theta(arch, w.seed + 3), dtype=torch.float32, device="cuda")
    runs = [(f"bf16_frac{f}", inrct.BF16, max(1, int(round(float(f) * g.n)))) for f in a.fracs.split(",")]
    if a.fp32:
        runs.append(("fp32_full", inrct.FP32, g.n))
    summary = {}
    for name, prec, n_idx in runs:
        mlp = inrct.mlp_desc(arch, prec if arch.kind != "hash" else inrct.FP32, B)
        tr = Trainer(prob, mlp, theta0, n_idx, a.lr if a.lr is not None else w.lr, seed=a.seed, subsets=a.subsets)
        with open(os.path.join(a.out, f"{name}.jsonl"), "w") as log:
            recs = run(tr, a.steps, a.log_every, log, os.path.join(a.out, f"{name}.pt"), a.steps)
        timed = [r["step_ms"] for r in recs if r["step_ms"] is not None]
        summary[name] = {"initial_mse": recs[0]["mse_vs_x_true"], "final": recs[-1], "batch": n_idx,
                         "mean_step_ms": sum(timed) / len(timed)}
        print(json.dumps({"run": name, **summary[name]}), flush=True)
    with open(os.path.join(a.out, "summary.json"), "w") as f:
        json.dump(summary, f, indent=1)


if __name__ == "__main__":
    main()
