"""grad_step_batched: one recorded CUDA graph over independent problems.

Every branch of the graph runs the same kernels with the same inputs as a
grad_step call on that problem alone, so after each launch the parameters, Adam
moments and losses must equal those of sequential grad_step calls bit for bit
(grad_step itself is checked against the oracle in test_gpu_mlp_*.py and
test_gpu_projector.py).  The Adam step index comes from the batch's device
counter; the sequential calls pass the same t on the host.  The index sets are
rewritten between launches, as a training loop does, to check that the graph
reads the buffers' current contents.
"""
import math

import numpy as np
import pytest
import torch

from paper_2604_09884_gb300 import inrct, synth

pytestmark = pytest.mark.gpu


def _problems():
    two_pi = 2 * math.pi
    return [synth.GeomSpec("par2d", 64, 30, 91),
            synth.GeomSpec("fan2d", 96, 45, 137, sod=384.0, sdd=576.0, span=two_pi),
            synth.GeomSpec("par2d", 128, 60, 182),
            synth.GeomSpec("fan2d", 80, 36, 114, sod=320.0, sdd=480.0, span=two_pi)]


def _state(geoms, arch, dev, seed):
    out = []
    for k, g in enumerate(geoms):
        x = torch.tensor(synth.phantom(2, g.N, 6, seed + k).reshape(-1), dtype=torch.float32, device=dev)
        y = inrct.project(g, x)
        theta = torch.tensor(synth.init_theta(arch, seed + 10 + k), dtype=torch.float32, device=dev)
        n_idx = g.n // 4
        out.append({"geom": g, "theta": theta, "y": y.contiguous(),
                    "idx": torch.empty(n_idx, dtype=torch.int32, device=dev), "scale": g.n / n_idx,
                    "m": torch.zeros_like(theta), "s": torch.zeros_like(theta),
                    "loss": torch.zeros(1, dtype=torch.float64, device=dev)})
    return out


def _fill_idx(probs, step):
    for k, q in enumerate(probs):
        g = q["geom"]
        q["idx"].copy_(torch.from_numpy(synth.index_set(g.n, q["idx"].numel(), 500 + 31 * step + k)))


@pytest.mark.parametrize("prec", [inrct.BF16, inrct.FP32], ids=["bf16", "fp32"])
def test_batched_graph_matches_sequential_grad_steps(prec):
    dev = torch.device("cuda")
    arch = synth.ArchSpec("siren", 2, 128, 3, omega0=30.0)
    mlp = inrct.mlp_desc(arch, prec)
    geoms = _problems()
    batched = _state(geoms, arch, dev, 7)
    seq = _state(geoms, arch, dev, 7)
    opt = inrct.adam(lr=1e-3)
    batch = inrct.Batch(mlp, batched, opt)
    for step in range(1, 3):
        _fill_idx(batched, step)
        _fill_idx(seq, step)
        batch.step()
        for q in seq:
            inrct.grad_step(q["geom"], mlp, q["theta"], q["y"], q["idx"], q["scale"],
                            inrct.adam(lr=1e-3, t=step), q["m"], q["s"], q["loss"])
        torch.cuda.synchronize()
        assert int(batch.counter.item()) == step
        for k, (a, b) in enumerate(zip(batched, seq)):
            for key in ("theta", "m", "s", "loss"):
                assert torch.equal(a[key], b[key]), (step, k, key)
            assert np.isfinite(a["loss"].item())
    # the parameters did move
    theta0 = torch.tensor(synth.init_theta(arch, 17), dtype=torch.float32, device=dev)
    assert not torch.equal(batched[0]["theta"], theta0)
    batch.close()


def test_batched_launches_are_counted():
    dev = torch.device("cuda")
    arch = synth.ArchSpec("siren", 2, 128, 3, omega0=30.0)
    mlp = inrct.mlp_desc(arch, inrct.BF16)
    probs = _state(_problems()[:2], arch, dev, 3)
    _fill_idx(probs, 0)
    batch = inrct.Batch(mlp, probs, inrct.adam(lr=1e-3))
    c0 = inrct.launch_count()
    batch.step()
    batch.step()
    torch.cuda.synchronize()
    per = (inrct.launch_count() - c0) / 2
    # at least the step counter plus, per problem, evaluation, projection, backprojection,
    # the VJP tile kernel, its weight-gradient GEMM and Adam
    assert per >= 1 + 2 * 6
    batch.close()
