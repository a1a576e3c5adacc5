"""Ordered subsets of views (Sec. 3): Algorithm 1 evaluated on a subset of the views.

Interleaved subset s of S is the same scan with V/S views (inrct.view_subset) and
the matching sinogram rows.  The subsets partition the rays, so the LS loss and the
residual backprojection split into per-subset sums, and the estimator of Eq. 2 is
linear in v: with one index set, the gradients of the S subset steps add up to the
gradient of the full step (FP32 path; the oracle side of the identity is pinned in
test_oracle_projector.py).  Each subset step's gradient and loss are also compared with the
oracle's Algorithm 1 run on the subset scan itself (its own geometry, the subset's rows of y)."""
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


@pytest.mark.parametrize("g", [
    synth.GeomSpec("fan2d", 64, 36, 91, sod=256.0, sdd=384.0, span=2 * math.pi),
    synth.GeomSpec("par2d", 48, 30, 69, angle0=0.1),
    synth.GeomSpec("cone3d", 24, 12, 37, 33, sod=96.0, sdd=144.0, span=2 * math.pi),
], ids=["fan64", "par48", "cone24"])
@pytest.mark.parametrize("kind", ["siren", "ffn"])
def test_subset_step_matches_the_oracle_on_the_subset_scan(g, kind):
    """One subset step's loss and gradient (Eq. 2 with v = P_s^T (P_s E{f} - y_s)) against the
    oracle's estimator on the subset geometry, FP32 path, bar 1e-4 relative L2."""
    S = 3
    dev = torch.device("cuda")
    if kind == "siren":
        arch = synth.ArchSpec("siren", g.d, 128, 2, omega0=30.0)
        B32 = None
    else:
        arch = synth.ArchSpec("ffn", g.d, 128, 2, n_feat=32, sigma=3.0)
        B32 = synth.fourier_matrix(arch.n_feat, g.d, arch.sigma, 8).astype(np.float32)
    oa = O.Arch(arch.kind, g.d, arch.width, arch.n_hidden, arch.n_feat,
                B32.astype(np.float64) if B32 is not None else None, arch.omega0)
    mlp = inrct.mlp_desc(arch, inrct.FP32, B32)
    theta32 = synth.init_theta(arch, 5).astype(np.float32)
    theta = torch.tensor(theta32, device=dev)
    y32 = synth.uniform(g.m, seed=6, lo=0.0, hi=1.0).astype(np.float32)
    y = torch.tensor(y32, device=dev)
    I = synth.index_set(g.n, g.n // 2, 7)
    if kind == "ffn":
        # the ReLU masks must be unique: points within rounding of a kink get no weight
        _, _, zs, _ = O.forward(oa, theta32.astype(np.float64), O.grid_coords(g.d, g.N, I), keep=True)
        ok = np.ones(I.size, bool)
        for z in zs[:-1]:
            ok &= (np.abs(z) >= 1e-6 * np.sqrt((z ** 2).mean())).all(axis=1)
        I = I[ok]
    idx = torch.from_numpy(I.astype(np.int32)).to(dev)
    scale = g.n / idx.numel()
    y_rows = y32.reshape(g.V, -1)
    for s in range(S):
        gs = inrct.view_subset(g, S, s)
        og = O.Geometry(gs.kind, gs.N, gs.V, gs.A, gs.B, gs.du, gs.dv, gs.sod, gs.sdd, gs.angle0, gs.span)
        ys = y_rows[s::S].reshape(-1)
        L_want, _, _, v = O.backprojected_residual(oa, theta32.astype(np.float64), og, ys)
        g_want = O.estimator(oa, theta32.astype(np.float64), og, v, I, scale)
        gout = torch.empty(arch.p, dtype=torch.float64, device=dev)
        loss = torch.empty(1, dtype=torch.float64, device=dev)
        inrct.grad_step(gs, mlp, theta, inrct.view_subset_rows(g, y, S, s), idx, scale, None, None, None,
                        loss, gout)
        torch.cuda.synchronize()
        got = gout.cpu().numpy()
        assert abs(loss.item() - L_want) <= 1e-5 * abs(L_want), (s, loss.item(), L_want)
        err = float(np.linalg.norm(got - g_want) / np.linalg.norm(g_want))
        assert err <= 1e-4, (s, err)
