"""The field of view (inrct_grid.fov = 1: the inscribed disk, Sec. 3 samples the INR inside
a FOV mask) on the GPU against the oracle: E{f} is zero outside the mask, listed points
outside it contribute nothing to the VJP, and grad_step on a masked problem matches the
oracle's loss and gradient (FP32 bar 1e-4, BF16 1e-2 with cosine >= 0.999)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_09884_gb300 import inrct, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def pair(spec, seed=1):
    B32 = synth.fourier_matrix(spec.n_feat, spec.d, spec.sigma, seed).astype(np.float32) if spec.kind == "ffn" else None
    oa = O.Arch(spec.kind, spec.d, spec.width, spec.n_hidden, spec.n_feat,
                B32.astype(np.float64) if B32 is not None else None, spec.omega0, hash_levels=spec.hash_levels,
                hash_feats=spec.hash_feats, hash_log2_T=spec.hash_log2_T, hash_base=spec.hash_base,
                hash_growth=spec.hash_growth)
    theta = synth.init_theta(spec, seed + 1, **({"table_scale": 0.5} if spec.kind == "hash" else {}))
    return oa, B32, theta.astype(np.float32)


CASES = [(synth.ArchSpec("siren", 2, 256, 3, omega0=30.0), inrct.BF16),
         (synth.ArchSpec("ffn", 2, 64, 2, n_feat=32, sigma=4.0), inrct.FP32),
         (synth.ArchSpec("hash", 2, 64, 2, hash_levels=6, hash_feats=2, hash_log2_T=10, hash_base=4,
                         hash_growth=1.7), inrct.FP32)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0].kind}_{'bf16' if c[1] else 'fp32'}")
def test_evaluation_is_zero_outside_the_field_of_view(case):
    spec, prec = case
    N = 70
    oa, B32, theta = pair(spec)
    img = inrct.inr_eval_grid(inrct.mlp_desc(spec, prec, B32), cuda(theta), N, fov=1).cpu().numpy()
    m = O.fov_mask(2, N)
    assert np.all(img[~m] == 0.0) and 0 < m.sum() < N * N
    want = O.forward(oa, theta.astype(np.float64), O.grid_coords(2, N), N=N)
    assert rel(img[m], want[m]) <= (2e-2 if prec == inrct.BF16 else 1e-5)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0].kind}_{'bf16' if c[1] else 'fp32'}")
def test_points_outside_the_field_of_view_carry_no_weight(case):
    spec, prec = case
    N = 70
    n = N * N
    oa, B32, theta = pair(spec, 3)
    h = inrct.mlp_desc(spec, prec, B32)
    v = cuda(np.random.default_rng(4).normal(size=n))
    idx = synth.index_set(n, 1500, 5)
    inside = idx[O.fov_mask(2, N, idx)]
    assert 0 < inside.size < idx.size
    a = inrct.inr_weighted_vjp(h, cuda(theta), N, cuda(idx, torch.int32), v, 2.0, fov=1).cpu().numpy()
    b = inrct.inr_weighted_vjp(h, cuda(theta), N, cuda(inside, torch.int32), v, 2.0, fov=1).cpu().numpy()
    assert rel(a, b) <= 1e-6
    if spec.kind == "siren":
        g = O.Geometry("par2d", N, 8, 99, fov=1)
        want = O.estimator(oa, theta.astype(np.float64), g, v.cpu().numpy(), idx, scale=2.0)
        assert rel(a, want) <= (1e-2 if prec == inrct.BF16 else 1e-4)


@pytest.mark.parametrize("prec", [inrct.FP32, inrct.BF16], ids=["fp32", "bf16"])
def test_grad_step_on_a_masked_problem_matches_the_oracle(prec):
    g = synth.GeomSpec("fan2d", 64, 24, 97, sod=120.0, sdd=180.0, span=2 * math.pi, fov=1)
    og = O.Geometry(g.kind, g.N, g.V, g.A, g.B, g.du, g.dv, g.sod, g.sdd, g.angle0, g.span, fov=1)
    spec = synth.ArchSpec("siren", 2, 128, 3, omega0=30.0)
    oa, _, theta = pair(spec, 6)
    y = O.project(og, synth.phantom(2, g.N, 5, 7).reshape(-1) * O.fov_mask(2, g.N)).astype(np.float32)
    inside = O.fov_indices(og)
    I = np.sort(np.random.default_rng(8).choice(inside, inside.size // 4, replace=False))
    I = np.concatenate([I, np.arange(0, g.N, 7)]).astype(np.int32)  # plus first-row points, mostly outside
    scale = inside.size / (inside.size // 4)
    L0, _, _, v0 = O.backprojected_residual(oa, theta.astype(np.float64), og, y.astype(np.float64))
    want = O.estimator(oa, theta.astype(np.float64), og, v0, I, scale)
    h = inrct.mlp_desc(spec, prec)
    th = cuda(theta)
    m, s = torch.zeros_like(th), torch.zeros_like(th)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros(spec.p, dtype=torch.float64, device="cuda")
    inrct.grad_step(g, h, th, cuda(y), cuda(I, torch.int32), scale, inrct.adam(lr=1e-4, t=1), m, s, loss, grad)
    torch.cuda.synchronize()
    got = grad.cpu().numpy()
    if prec == inrct.FP32:
        assert abs(loss.item() - L0) <= 1e-5 * L0
        assert rel(got, want) <= 1e-4
    else:
        assert abs(loss.item() - L0) <= 2e-2 * L0
        assert rel(got, want) <= 1e-2 and float(got @ want / np.linalg.norm(got) / np.linalg.norm(want)) >= 0.999


def test_index_set_check_counts():
    N = 48
    n = N * N
    idx = synth.index_set(n, 700, 9).astype(np.int64)
    listed = np.concatenate([idx, idx[:5], idx[100:102], [-1, n, n + 5, -(1 << 30)]]).astype(np.int32)
    c0 = inrct.check_index_set(2, N, cuda(listed, torch.int32))
    assert c0 == {"out_of_range": 4, "outside_fov": 0, "repeats": 7}
    c1 = inrct.check_index_set(2, N, cuda(listed, torch.int32), fov=1)
    valid = listed[(listed >= 0) & (listed < n)].astype(np.int64)
    assert c1 == {"out_of_range": 4, "outside_fov": int((~O.fov_mask(2, N, valid)).sum()), "repeats": 7}
    assert inrct.check_index_set(3, 20, cuda(np.arange(8000), torch.int32)) == {"out_of_range": 0, "outside_fov": 0,
                                                                             "repeats": 0}


CASES3 = [(synth.ArchSpec("siren", 3, 128, 3, omega0=30.0), inrct.BF16),
          (synth.ArchSpec("ffn", 3, 128, 2, n_feat=32, sigma=3.0), inrct.BF16),
          (synth.ArchSpec("siren", 3, 64, 2, omega0=30.0), inrct.FP32),
          (synth.ArchSpec("hash", 3, 64, 2, hash_levels=4, hash_feats=2, hash_log2_T=12, hash_base=4,
                          hash_growth=1.6), inrct.FP32)]


@pytest.mark.parametrize("case", CASES3, ids=lambda c: f"{c[0].kind}3d_{'bf16' if c[1] else 'fp32'}")
def test_three_d_field_of_view_is_a_cylinder(case):
    """3-D grids: E{f} is zero outside the cylinder (the disk test on x, y of every z slice) and
    the oracle's inside it, and listed points outside it carry no weight in the VJP."""
    spec, prec = case
    N = 24
    n = N ** 3
    oa, B32, theta = pair(spec, 5)
    h = inrct.mlp_desc(spec, prec, B32)
    img = inrct.inr_eval_grid(h, cuda(theta), N, fov=1).cpu().numpy()
    m = O.fov_mask(3, N)
    assert np.all(img[~m] == 0.0) and 0 < m.sum() < n
    sel = np.flatnonzero(m)[::7]
    want = O.forward(oa, theta.astype(np.float64), O.grid_coords(3, N, sel), N=N)
    assert rel(img[sel], want) <= (2e-2 if prec == inrct.BF16 else 1e-5)
    v = cuda(np.random.default_rng(6).normal(size=n))
    idx = synth.index_set(n, 3000, 7)
    inside = idx[O.fov_mask(3, N, idx)]
    assert 0 < inside.size < idx.size
    a = inrct.inr_weighted_vjp(h, cuda(theta), N, cuda(idx, torch.int32), v, 1.5, fov=1).cpu().numpy()
    b = inrct.inr_weighted_vjp(h, cuda(theta), N, cuda(inside, torch.int32), v, 1.5, fov=1).cpu().numpy()
    assert rel(a, b) <= 1e-6
