"""The virtual loss of Eq. 3 behind torch.autograd (inrct.InrVirtualLoss).

Workload: the 256^3 cone workload's network (Fourier features 256, sigma 8, 4 x 256 ReLU) on
its 256^3 grid, |S| = 2^20 listed points, BF16 tensor-core path.  v is zero except at 2000 of
the listed points, so every other term of Eq. 2 and Eq. 3 is exactly zero and the oracle
can evaluate the same loss and gradient at those 2000 points.  Checked:

- the value InrVirtualLoss returns against the oracle's virtual loss (Eq. 3);
- loss.backward() leaves in theta.grad the oracle's estimator (Eq. 2) within the BF16 bar
  (1e-2 relative L2, cosine >= 0.999);
- 64 random entries of theta.grad against central differences of the oracle's FP64 virtual
  loss (1e-2 relative L2 over the 64 entries).  With the ReLU masks fixed, f is linear in
  any single parameter, so a step of 1e-7 that crosses no kink gives the derivative up to
  FP64 rounding; points with a pre-activation within 1e-6 of its layer's RMS of zero get
  no weight.
"""
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


def test_virtual_loss_autograd_matches_the_oracle_and_finite_differences():
    w = synth.workloads()["cone3d_256_ffn256"]
    a, g = w.arch, w.geom
    B32 = synth.fourier_matrix(a.n_feat, a.d, a.sigma, 41).astype(np.float32)
    oa = O.Arch(a.kind, a.d, a.width, a.n_hidden, a.n_feat, B32.astype(np.float64), a.omega0)
    theta32 = synth.init_theta(a, 42).astype(np.float32)
    th64 = theta32.astype(np.float64)
    S = 1 << 20
    idx = synth.index_set(g.n, S, 43)
    pick = np.sort(np.random.default_rng(44).choice(S, 2000, replace=False))
    live = idx[pick].astype(np.int64)
    X = O.grid_coords(3, g.N, live)
    _, _, zs, _ = O.forward(oa, th64, X, keep=True)
    ok = np.ones(live.size, bool)
    for z in zs[:-1]:
        ok &= (np.abs(z) >= 1e-6 * np.sqrt((z ** 2).mean())).all(axis=1)
    live, X = live[ok], X[ok]
    vals = np.random.default_rng(45).normal(size=live.size).astype(np.float32)
    scale = g.n / S
    dev = torch.device("cuda")
    v = torch.zeros(g.n, dtype=torch.float32, device=dev)
    v[torch.from_numpy(live).to(dev)] = torch.from_numpy(vals).to(dev)
    mlp = inrct.mlp_desc(a, inrct.BF16, B32, device=dev)
    theta = torch.tensor(theta32, device=dev, requires_grad=True)
    loss = inrct.InrVirtualLoss.apply(theta, v, torch.from_numpy(idx).to(dev), scale, mlp, g.N)
    loss.backward()
    got = theta.grad.double().cpu().numpy()

    wv = scale * vals.astype(np.float64)
    f = O.forward(oa, th64, X)
    want_value = float(wv @ f)
    assert abs(loss.item() - want_value) <= 1e-4 * float(np.abs(wv * f).sum()), (loss.item(), want_value)
    want = O.vjp(oa, th64, X, wv)
    cosine = float(got @ want / np.linalg.norm(got) / np.linalg.norm(want))
    assert rel(got, want) <= 1e-2 and cosine >= 0.999, (rel(got, want), cosine)

    # central differences of the oracle's virtual loss on 64 random entries
    ent = np.sort(np.random.default_rng(46).choice(a.p, 64, replace=False))
    h = 1e-7
    fd = np.empty(ent.size)
    for k, e in enumerate(ent):
        tp, tm = th64.copy(), th64.copy()
        tp[e] += h
        tm[e] -= h
        fd[k] = (float(wv @ O.forward(oa, tp, X)) - float(wv @ O.forward(oa, tm, X))) / (2 * h)
    assert rel(want[ent], fd) <= 1e-6, rel(want[ent], fd)      # the oracle's own reverse mode
    assert rel(got[ent], fd) <= 1e-2, rel(got[ent], fd)


def test_virtual_loss_backward_scales_with_the_incoming_gradient():
    """A loss built on top of the virtual loss (here 3 L~) passes its factor through backward."""
    spec = synth.ArchSpec("siren", 2, 128, 3, omega0=30.0)
    N = 48
    dev = torch.device("cuda")
    mlp = inrct.mlp_desc(spec, inrct.BF16, device=dev)
    theta = torch.tensor(synth.init_theta(spec, 3).astype(np.float32), device=dev, requires_grad=True)
    v = torch.tensor(np.random.default_rng(4).normal(size=N * N).astype(np.float32), device=dev)
    idx = torch.from_numpy(synth.index_set(N * N, 700, 5)).to(dev)
    (3.0 * inrct.InrVirtualLoss.apply(theta, v, idx, 2.0, mlp, N)).backward()
    g1 = theta.grad.clone()
    theta.grad = None
    inrct.InrVirtualLoss.apply(theta, v, idx, 2.0, mlp, N).backward()
    # grad_out * g is formed in FP64 and then rounded to FP32: equal to an FP32 ulp
    assert torch.allclose(g1, 3.0 * theta.grad, rtol=2e-7, atol=0)


def test_virtual_loss_fp32_path_matches_the_oracle():
    """The FP32 SIMT path of inr_virtual_loss: value (Eq. 3) and gradient (Eq. 2) against the
    oracle at the FP32 bars (1e-5 value relative to sum |w f|, 1e-4 gradient)."""
    spec = synth.ArchSpec("ffn", 3, 128, 3, n_feat=64, sigma=4.0)
    N = 20
    n = N ** 3
    dev = torch.device("cuda")
    B32 = synth.fourier_matrix(spec.n_feat, 3, spec.sigma, 6).astype(np.float32)
    oa = O.Arch("ffn", 3, spec.width, spec.n_hidden, spec.n_feat, B32.astype(np.float64))
    theta32 = synth.init_theta(spec, 7).astype(np.float32)
    idx = synth.index_set(n, 3000, 8)
    _, _, zs, _ = O.forward(oa, theta32.astype(np.float64), O.grid_coords(3, N, idx), keep=True)
    ok = np.ones(idx.size, bool)
    for z in zs[:-1]:
        ok &= (np.abs(z) >= 1e-6 * np.sqrt((z ** 2).mean())).all(axis=1)
    idx = idx[ok].astype(np.int32)
    vv = np.random.default_rng(9).normal(size=n).astype(np.float32)
    scale = n / idx.size
    mlp = inrct.mlp_desc(spec, inrct.FP32, B32, device=dev)
    theta = torch.tensor(theta32, device=dev, requires_grad=True)
    loss = inrct.InrVirtualLoss.apply(theta, torch.from_numpy(vv).to(dev), torch.from_numpy(idx).to(dev),
                                      scale, mlp, N)
    loss.backward()
    X = O.grid_coords(3, N, idx)
    wv = scale * vv.astype(np.float64)[idx]
    f = O.forward(oa, theta32.astype(np.float64), X)
    assert abs(loss.item() - float(wv @ f)) <= 1e-5 * float(np.abs(wv * f).sum())
    want = O.vjp(oa, theta32.astype(np.float64), X, wv)
    assert rel(theta.grad.double().cpu().numpy(), want) <= 1e-4
