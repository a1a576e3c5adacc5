"""GPU parity of the FP32 SIMT INR path (the plain comparator) against the FP64
oracle: the grid evaluation E{f} and the weighted VJP of Eq. (2) (bar: FP32
grad within 1e-4 relative L2), and grad_step on the 128^2 parallel workload."""
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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def arch_pair(spec: synth.ArchSpec, seed=0):
    B = synth.fourier_matrix(spec.n_feat, spec.d, spec.sigma, seed) if spec.kind == "ffn" else None
    B32 = B.astype(np.float32) if B is not None else None
    oa = O.Arch(spec.kind, spec.d, spec.width, spec.n_hidden, spec.n_feat,
                B32.astype(np.float64) if B32 is not None else None, spec.omega0)
    return oa, B32


def kink_free(oa, theta, X, tau=1e-6):
    """Points whose ReLU pre-activations all stay at least tau * rms away from 0.

    Where |z| is within rounding of the kink, FP32 and FP64 can take different
    (equally valid) mask decisions; ReLU parity cases keep only the points where
    the decision is unique."""
    if oa.kind != "ffn":
        return np.ones(len(X), bool)
    _, _, zs, _ = O.forward(oa, np.asarray(theta, np.float64), X, keep=True)
    ok = np.ones(len(X), bool)
    for z in zs[:-1]:
        ok &= (np.abs(z) >= tau * np.sqrt((z ** 2).mean())).all(axis=1)
    return ok


ARCHS = [
    synth.ArchSpec("ffn", 2, 64, 3, n_feat=64, sigma=10.0),
    synth.ArchSpec("siren", 2, 256, 5, omega0=30.0),
    synth.ArchSpec("ffn", 3, 256, 4, n_feat=256, sigma=8.0),
    synth.ArchSpec("siren", 2, 128, 3, omega0=30.0),
    synth.ArchSpec("ffn", 3, 128, 2, n_feat=7, sigma=3.0),
]


@pytest.mark.parametrize("spec", ARCHS, ids=lambda a: f"{a.kind}{a.d}d_{a.width}x{a.n_hidden}")
def test_eval_grid_fp32_matches_oracle(spec):
    N = 64 if spec.d == 2 else 20
    oa, B32 = arch_pair(spec, 1)
    theta = synth.init_theta(spec, 2).astype(np.float32)
    h = inrct.mlp_desc(spec, inrct.FP32, B32)
    img = inrct.inr_eval_grid(h, cuda(theta), N).cpu().numpy()
    want = O.forward(oa, theta.astype(np.float64), O.grid_coords(spec.d, N))
    assert rel(img, want) <= 1e-5


@pytest.mark.parametrize("spec", ARCHS, ids=lambda a: f"{a.kind}{a.d}d_{a.width}x{a.n_hidden}")
def test_weighted_vjp_fp32_matches_oracle(spec):
    N = 64 if spec.d == 2 else 20
    n = N ** spec.d
    oa, B32 = arch_pair(spec, 3)
    theta = synth.init_theta(spec, 4).astype(np.float32)
    rng = np.random.default_rng(5)
    v = rng.normal(size=n).astype(np.float32)
    idx = synth.index_set(n, 1037, 6)
    idx = idx[kink_free(oa, theta, O.grid_coords(spec.d, N, idx))]
    idx = np.concatenate([idx, idx[:5]]).astype(np.int32)      # repeats are allowed
    scale = n / idx.size
    h = inrct.mlp_desc(spec, inrct.FP32, B32)
    g64, g32 = inrct.inr_weighted_vjp(h, cuda(theta), N, cuda(idx, torch.int32), cuda(v), scale,
                                      want_f32=True)
    want = O.vjp(oa, theta.astype(np.float64), O.grid_coords(spec.d, N, idx),
                 scale * v.astype(np.float64)[idx])
    assert rel(g64.cpu().numpy(), want) <= 1e-4
    assert rel(g32.cpu().numpy(), want) <= 1e-4


def test_grad_step_fp32_full_grid_128():
    w = synth.workloads()["par2d_128_ffn64"]
    g, spec = w.geom, w.arch
    oa, B32 = arch_pair(spec, 7)
    og = O.Geometry(g.kind, g.N, g.V, g.A, g.B, g.du, g.dv, g.sod, g.sdd, g.angle0, g.span)
    theta = synth.init_theta(spec, 8).astype(np.float32)
    y = synth.noisy(O.project(og, synth.phantom(2, g.N, 10, 9)), 0.01, 10).astype(np.float32)
    # the whole grid except the points within rounding of a ReLU kink
    idx = np.arange(g.n, dtype=np.int32)
    idx = idx[kink_free(oa, theta, O.grid_coords(2, g.N))]
    assert idx.size > 0.8 * g.n
    L0, _, _, v0 = O.backprojected_residual(oa, theta.astype(np.float64), og, y.astype(np.float64))
    grad0 = O.estimator(oa, theta.astype(np.float64), og, v0, idx, scale=1.0)
    h = inrct.mlp_desc(spec, inrct.FP32, B32)
    th = cuda(theta)
    m = torch.zeros_like(th)
    s = torch.zeros_like(th)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros(spec.p, dtype=torch.float64, device="cuda")
    ad = inrct.adam(lr=1e-3, t=1)
    inrct.grad_step(g, h, th, cuda(y), cuda(idx, torch.int32), 1.0, ad, m, s, loss, grad)
    torch.cuda.synchronize()
    assert abs(loss.item() - L0) <= 1e-5 * L0
    gg = grad.cpu().numpy()
    assert rel(gg, grad0) <= 1e-4
    # first Adam step moves by -lr g / (|g| + eps) (computed from the GPU's own gradient)
    step = th.double().cpu().numpy() - theta.astype(np.float64)
    np.testing.assert_allclose(step, -1e-3 * gg / (np.abs(gg) + 1e-8), rtol=2e-5, atol=1e-9)


def test_grad_step_fls_fp32_matches_oracle():
    g = synth.GeomSpec("fan2d", 64, 24, 97, sod=120.0, sdd=180.0, span=2 * math.pi)
    spec = synth.ArchSpec("siren", 2, 64, 2, omega0=30.0)
    oa, _ = arch_pair(spec)
    og = O.Geometry(g.kind, g.N, g.V, g.A, g.B, g.du, g.dv, g.sod, g.sdd, g.angle0, g.span)
    theta = synth.init_theta(spec, 12).astype(np.float32)
    y = O.project(og, synth.phantom(2, g.N, 6, 13)).astype(np.float32)
    idx = synth.index_set(g.n, g.n // 4, 14)
    scale = g.n / idx.size
    th = cuda(theta)
    x = O.evaluate_image(oa, theta.astype(np.float64), og)
    Lf, Fd = O.fls_loss(og, O.project(og, x), y)
    v = O.backproject(og, Fd)
    want = O.estimator(oa, theta.astype(np.float64), og, v, idx, scale)
    h = inrct.mlp_desc(spec, inrct.FP32)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros(spec.p, dtype=torch.float64, device="cuda")
    inrct.grad_step(g, h, th, cuda(y), cuda(idx, torch.int32), scale, None, None, None, loss, grad,
                    loss_kind=inrct.LOSS_FLS)
    torch.cuda.synchronize()
    assert abs(loss.item() - Lf) <= 1e-4 * abs(Lf)
    assert rel(grad.cpu().numpy(), want) <= 1e-4
    np.testing.assert_array_equal(th.cpu().numpy(), theta)      # no Adam: theta untouched


def test_adam_state_over_three_steps_matches_the_oracle():
    """Adam inside grad_step over t = 1, 2, 3: after every step theta, m and s equal the oracle's
    bias-corrected FP64 Adam applied to the kernel's own gradient of that step (the moments
    accumulate and the bias correction changes with t; the first step alone cannot show either)."""
    w = synth.workloads()["par2d_128_ffn64"]
    g, spec = w.geom, w.arch
    oa, B32 = arch_pair(spec, 7)
    og = O.Geometry(g.kind, g.N, g.V, g.A, g.B, g.du, g.dv, g.sod, g.sdd, g.angle0, g.span)
    theta = synth.init_theta(spec, 8).astype(np.float32)
    y = synth.noisy(O.project(og, synth.phantom(2, g.N, 10, 9)), 0.01, 10).astype(np.float32)
    idx = synth.index_set(g.n, g.n // 4, 12)
    h = inrct.mlp_desc(spec, inrct.FP32, B32)
    th = cuda(theta)
    m = torch.zeros_like(th)
    s = torch.zeros_like(th)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros(spec.p, dtype=torch.float64, device="cuda")
    st = O.AdamState(np.zeros(spec.p), np.zeros(spec.p))
    for t in (1, 2, 3):
        before = th.double().cpu().numpy()
        inrct.grad_step(g, h, th, cuda(y), cuda(idx, torch.int32), g.n / idx.size, inrct.adam(lr=1e-3, t=t),
                        m, s, loss, grad)
        torch.cuda.synchronize()
        want = O.adam_step(before, grad.cpu().numpy(), st, lr=1e-3)
        # FP32 state against FP64: norm-wise (single entries lose relative accuracy where the
        # moment's two terms cancel); the kernel applies beta2 = 0.999 as an FP32 value, which
        # puts 1 - beta2 1.3e-5 (relative) off.  A wrong bias correction is off by a factor.
        assert rel(m.double().cpu().numpy(), st.m) <= 1e-6
        assert rel(s.double().cpu().numpy(), st.s) <= 5e-5
        step = th.double().cpu().numpy() - before
        assert rel(step, want - before) <= 5e-5
        # and entry by entry, up to half an ulp of the FP32 theta (|theta| < 0.5 here)
        np.testing.assert_allclose(step, want - before, rtol=1e-3, atol=3e-8)
