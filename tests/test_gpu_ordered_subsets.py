"""Ordered subsets of views (Sec. 3): Algorithm 1 evaluated on a subset of the views.

Interleaved subset s of S is the same scan with V/S views (inrct.view_subset) and
the matching sinogram rows.  The subsets partition the rays, so the LS loss and the
residual backprojection split into per-subset sums, and the estimator of Eq. 2 is
linear in v: with one index set, the gradients of the S subset steps add up to the
gradient of the full step (FP32 path; the oracle side of the identity is pinned in
test_oracle_projector.py)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_09884_gb300 import inrct, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("g", [
    synth.GeomSpec("fan2d", 64, 36, 91, sod=256.0, sdd=384.0, span=2 * math.pi),
    synth.GeomSpec("par2d", 48, 30, 69, angle0=0.1),
    synth.GeomSpec("cone3d", 24, 12, 37, 33, sod=96.0, sdd=144.0, span=2 * math.pi),
], ids=["fan64", "par48", "cone24"])
def test_subset_gradients_sum_to_the_full_gradient(g):
    S = 3
    dev = torch.device("cuda")
    arch = synth.ArchSpec("siren", g.d, 128, 2, omega0=30.0)
    mlp = inrct.mlp_desc(arch, inrct.FP32)
    theta = torch.tensor(synth.init_theta(arch, 5), dtype=torch.float32, device=dev)
    y = torch.tensor(synth.uniform(g.m, seed=6, lo=0.0, hi=1.0), dtype=torch.float32, device=dev)
    idx = torch.from_numpy(synth.index_set(g.n, g.n // 2, 7)).to(dev)
    scale = g.n / idx.numel()

    def grad(geom, yy):
        gout = torch.empty(arch.p, dtype=torch.float64, device=dev)
        loss = torch.empty(1, dtype=torch.float64, device=dev)
        inrct.grad_step(geom, mlp, theta, yy, idx, scale, None, None, None, loss, gout)
        return gout, loss

    g_full, l_full = grad(g, y)
    g_sum = torch.zeros_like(g_full)
    l_sum = 0.0
    for s in range(S):
        gs = inrct.view_subset(g, S, s)
        # the subset geometry matches the oracle's own construction of that scan
        og = O.Geometry(gs.kind, gs.N, gs.V, gs.A, gs.B, gs.du, gs.dv, gs.sod, gs.sdd,
                        g.angle0 + g.span * s / g.V, g.span)
        assert og.angle0 == gs.angle0 and gs.V * S == g.V
        gr, lo = grad(gs, inrct.view_subset_rows(g, y, S, s))
        g_sum += gr
        l_sum += lo.item()
    torch.cuda.synchronize()
    assert abs(l_sum - l_full.item()) <= 1e-5 * abs(l_full.item())
    rel = (torch.linalg.norm(g_sum - g_full) / torch.linalg.norm(g_full)).item()
    assert rel <= 1e-4, rel

