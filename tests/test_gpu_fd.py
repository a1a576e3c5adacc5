"""Finite-difference check of the whole GPU chain on a small cone scan.

With |I| = n the estimator of Eq. 2 is the exact gradient of the LS loss (Sec. 3), so
the gradient grad_step returns must match central differences of the loss that
grad_step itself reports, for 64 entries of theta spread over the network: output
weights and bias (the loss is exactly quadratic in them, so central differences are
exact up to rounding), the last hidden layer and the first layer (Richardson
extrapolation of steps h and h/2).  FP32 path, SIREN (smooth: no ReLU kinks inside
the difference step)."""
import math

import numpy as np
import pytest
import torch

from paper_2604_09884_gb300 import inrct, synth

pytestmark = pytest.mark.gpu


def test_gradient_matches_central_differences_of_the_loss():
    dev = torch.device("cuda")
    g = synth.GeomSpec("cone3d", 20, 10, 31, 29, sod=80.0, sdd=120.0, span=2 * math.pi)
    arch = synth.ArchSpec("siren", 3, 128, 2, omega0=30.0)
    mlp = inrct.mlp_desc(arch, inrct.FP32)
    theta0 = torch.tensor(synth.init_theta(arch, 11), dtype=torch.float32, device=dev)
    x_true = torch.tensor(synth.phantom(3, g.N, 6, seed=12).reshape(-1), dtype=torch.float32, device=dev)
    y = inrct.project(g, x_true)
    idx = torch.arange(g.n, dtype=torch.int32, device=dev)
    ws = torch.empty(inrct.step_ws_bytes(g, mlp, g.n), dtype=torch.uint8, device=dev)

    def run(theta):
        gout = torch.empty(arch.p, dtype=torch.float64, device=dev)
        loss = torch.empty(1, dtype=torch.float64, device=dev)
        inrct.grad_step(g, mlp, theta, y, idx, 1.0, None, None, None, loss, gout, ws)
        return loss.item(), gout

    _, grad = run(theta0)
    grad = grad.cpu().numpy()
    shapes = arch.layer_shapes()          # [(out, in)] per layer
    offs, o = [], 0
    for out, inn in shapes:
        offs.append((o, o + out * inn))   # (weight offset, bias offset)
        o += out * inn + out
    rng = np.random.default_rng(3)

    def pick(lo, hi, k):                  # the k largest-|g| entries of a block
        block = np.arange(lo, hi)
        return block[np.argsort(-np.abs(grad[lo:hi]))[:k]]

    (w_first, _), (w_last, b_last), (w_out, b_out) = offs[0], offs[-2], offs[-1]
    exact = np.r_[pick(w_out, w_out + shapes[-1][1], 15), [b_out]]
    smooth = np.r_[pick(w_last, b_last, 16), pick(w_first, w_first + shapes[0][0] * shapes[0][1], 16),
                   pick(b_last, b_last + shapes[-2][0], 16)]
    assert exact.size + smooth.size == 64

    def fd(k, h):
        th = theta0.clone()
        th[k] += h
        lp, _ = run(th)
        th[k] -= 2 * h
        lm, _ = run(th)
        return (lp - lm) / (2 * h)

    scale = np.abs(grad[np.r_[exact, smooth]]).max()
    for k in exact:
        h = 1e-2 * max(1.0, abs(theta0[k].item()))
        assert abs(fd(int(k), h) - grad[k]) <= 1e-2 * abs(grad[k]) + 1e-3 * scale, k
    for k in smooth:
        h = 2e-3 * max(0.05, abs(theta0[k].item()))
        d1, d2 = fd(int(k), h), fd(int(k), h / 2)
        richardson = (4 * d2 - d1) / 3
        assert abs(richardson - grad[k]) <= 3e-2 * abs(grad[k]) + 1e-3 * scale, (k, richardson, grad[k])
