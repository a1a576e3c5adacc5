"""Pins of the oracle's INR (Sec. 4: Fourier-feature ReLU MLP and SIREN), its
hand-derived reverse mode, the estimator of Eq. (2), the virtual loss of Eq. (3)
and the Adam step.

References used here that are not the oracle: closed-form network values,
PyTorch autograd in FP64 (a library routine), central finite differences,
exhaustive enumeration of index subsets, and torch.optim.Adam.
"""
import itertools
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_09884_gb300 import synth


def _arch(kind, d=2, width=8, n_hidden=3, n_feat=5, seed=0, omega0=30.0):
    B = synth.fourier_matrix(n_feat, d, 2.0, seed) if kind == "ffn" else None
    return O.Arch(kind, d, width, n_hidden, n_feat if kind == "ffn" else 0, B, omega0)


def _theta(arch, seed=0):
    spec = synth.ArchSpec(arch.kind, arch.d, arch.width, arch.n_hidden, arch.n_feat,
                          omega0=arch.omega0)
    th = synth.init_theta(spec, seed)
    if arch.kind == "ffn":   # non-zero biases so that bias gradients are exercised
        th = th + 0.05 * np.random.default_rng(seed + 7).normal(size=th.size)
    return th


def _torch_model(arch, theta, X):
    """The same network written with torch ops, FP64, differentiated by autograd."""
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    x = torch.tensor(X, dtype=torch.float64)
    if arch.kind == "ffn":
        P = 2 * math.pi * x @ torch.tensor(arch.B, dtype=torch.float64).T
        h = torch.cat([torch.cos(P), torch.sin(P)], 1)
    else:
        h = x
    off = 0
    shapes = arch.layer_shapes()
    for li, (o, i) in enumerate(shapes):
        W = th[off:off + o * i].view(o, i)
        off += o * i
        b = th[off:off + o]
        off += o
        z = torch.nn.functional.linear(h, W, b)
        if li == len(shapes) - 1:
            h = z
        elif arch.kind == "ffn":
            h = torch.relu(z)
        else:
            h = torch.sin(arch.omega0 * z)
    return th, h[:, 0]


def test_layer_sizes_match_workloads():
    want = {"par2d_128_ffn64": 16641, "fan2d_512_siren256": 264193,
            "cone3d_256_ffn256": 328961, "cone3d_501_ffn512": 525825,
            "fan2d_512_hash64": 16 * 2 ** 19 * 2 + (64 * 32 + 64) + (64 * 64 + 64) + 65}
    for name, w in synth.workloads().items():
        s = w.arch
        a = O.Arch(s.kind, s.d, s.width, s.n_hidden, s.n_feat, hash_levels=s.hash_levels,
                   hash_feats=s.hash_feats, hash_log2_T=s.hash_log2_T, hash_base=s.hash_base,
                   hash_growth=s.hash_growth)
        assert a.p == want[name] == w.arch.p


def test_fourier_encoding_closed_form():
    arch = O.Arch("ffn", 2, 4, 1, 2, np.array([[0.25, 0.0], [0.0, 0.5]]))
    g = O.encode(arch, np.array([[1.0, 0.5], [0.0, 0.0], [-2.0, 1.0]]))
    want = np.array([[0.0, 0.0, 1.0, 1.0],
                     [1.0, 1.0, 0.0, 0.0],
                     [-1.0, -1.0, 0.0, 0.0]])
    np.testing.assert_allclose(g, want, atol=1e-15)


def test_siren_one_hidden_layer_closed_form():
    arch = O.Arch("siren", 2, 3, 1, omega0=30.0)
    W1 = np.array([[0.1, -0.2], [0.05, 0.3], [-0.4, 0.01]])
    b1 = np.array([0.02, -0.1, 0.3])
    w2 = np.array([[0.7, -1.1, 0.4]])
    b2 = np.array([0.25])
    theta = np.concatenate([W1.ravel(), b1, w2.ravel(), b2])
    x = np.array([0.3, -0.6])
    want = sum(w2[0, k] * math.sin(30.0 * (W1[k] @ x + b1[k])) for k in range(3)) + 0.25
    assert abs(O.forward(arch, theta, x[None])[0] - want) < 1e-14
    # gradient wrt b1[k] is w2_k * 30 cos(30 z_k); wrt W1[k, j] that times x_j
    g = O.vjp(arch, theta, x[None], np.array([1.0]))
    for k in range(3):
        dz = w2[0, k] * 30.0 * math.cos(30.0 * (W1[k] @ x + b1[k]))
        assert abs(g[6 + k] - dz) < 1e-13
        assert abs(g[2 * k] - dz * x[0]) < 1e-13 and abs(g[2 * k + 1] - dz * x[1]) < 1e-13


@pytest.mark.parametrize("kind,d", [("ffn", 2), ("ffn", 3), ("siren", 2), ("siren", 3)])
def test_vjp_matches_torch_autograd(kind, d):
    arch = _arch(kind, d=d)
    theta = _theta(arch, 3)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (37, d))
    w = rng.normal(size=37)
    th, f = _torch_model(arch, theta, X)
    np.testing.assert_allclose(O.forward(arch, theta, X), f.detach().numpy(), rtol=1e-13,
                               atol=1e-14)
    (f @ torch.tensor(w)).backward()
    np.testing.assert_allclose(O.vjp(arch, theta, X, w), th.grad.numpy(), rtol=1e-11,
                               atol=1e-12)


@pytest.mark.parametrize("kind", ["ffn", "siren"])
def test_vjp_matches_finite_differences(kind):
    arch = _arch(kind, omega0=3.0)
    theta = _theta(arch, 5)
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 1, (11, 2))
    w = rng.normal(size=11)
    g = O.vjp(arch, theta, X, w)
    h = 1e-6
    for j in rng.choice(theta.size, 25, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (w @ O.forward(arch, tp, X) - w @ O.forward(arch, tm, X)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-7 * max(1.0, abs(g[j])), (j, fd, g[j])


def _tiny_problem(kind="ffn", N=6):
    g = O.Geometry("par2d", N, 5, 9)
    arch = _arch(kind, width=6, n_hidden=2, n_feat=3, omega0=2.0)
    theta = _theta(arch, 11)
    y = O.project(g, synth.phantom(2, N, 3, 12))
    return g, arch, theta, y


@pytest.mark.parametrize("kind", ["ffn", "siren"])
def test_full_gradient_is_chain_rule_of_total_loss(kind):
    # grad of L(theta) = 1/2 || P E{f_theta} - y ||^2 by central differences on the
    # whole pipeline must equal sum_i v_i grad f(x_i) with v = P^T (z - y).
    g, arch, theta, y = _tiny_problem(kind)
    L0, grad, _ = O.full_gradient(arch, theta, g, y)

    def loss(t):
        return O.ls_loss(O.project(g, O.evaluate_image(arch, t, g)), y)[0]

    assert abs(loss(theta) - L0) < 1e-14 * max(1, L0)
    h = 1e-6
    rng = np.random.default_rng(13)
    for j in rng.choice(theta.size, 30, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert abs(fd - grad[j]) <= 1e-7 * max(1.0, abs(grad[j])), (j, fd, grad[j])


def test_estimator_full_index_set_is_full_gradient():
    g, arch, theta, y = _tiny_problem("siren")
    _, grad, v = O.full_gradient(arch, theta, g, y)
    ghat = O.estimator(arch, theta, g, v, np.arange(g.n))
    np.testing.assert_allclose(ghat, grad, rtol=1e-13, atol=1e-15)


def test_estimator_unbiased_exhaustive():
    # n = 16, |I| = 4: the mean of Eq. (2) over all C(16, 4) = 1820 subsets is the
    # full gradient (Sec. 3: E_I[estimate] = grad L for uniform I).
    g = O.Geometry("par2d", 4, 3, 7)
    arch = _arch("ffn", width=5, n_hidden=2, n_feat=2)
    theta = _theta(arch, 21)
    y = O.project(g, synth.uniform(16, 22, 0, 1))
    _, grad, v = O.full_gradient(arch, theta, g, y)
    acc = np.zeros_like(grad)
    count = 0
    for I in itertools.combinations(range(16), 4):
        acc += O.estimator(arch, theta, g, v, np.array(I))
        count += 1
    assert count == 1820
    np.testing.assert_allclose(acc / count, grad, rtol=1e-12, atol=1e-13)


def test_estimator_monte_carlo_error_shrinks():
    g, arch, theta, y = _tiny_problem("ffn", N=8)
    _, grad, v = O.full_gradient(arch, theta, g, y)
    errs = []
    for K in (16, 256):
        acc = np.zeros_like(grad)
        for s in range(K):
            acc += O.estimator(arch, theta, g, v, synth.index_set(g.n, 8, 100 + s))
        errs.append(np.linalg.norm(acc / K - grad) / np.linalg.norm(grad))
    assert errs[1] < errs[0] / 2.0, errs


def test_virtual_loss_gradient_is_estimator():
    # Eq. (3): with v frozen, grad of the virtual loss equals Eq. (2).
    g, arch, theta, y = _tiny_problem("siren")
    _, _, v = O.full_gradient(arch, theta, g, y)
    I = synth.index_set(g.n, 9, 3)
    ghat = O.estimator(arch, theta, g, v, I)
    h = 1e-6
    for j in np.random.default_rng(1).choice(theta.size, 25, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (O.virtual_loss(arch, tp, g, v, I) - O.virtual_loss(arch, tm, g, v, I)) / (2 * h)
        assert abs(fd - ghat[j]) <= 1e-7 * max(1.0, abs(ghat[j]))


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(0)
    th0 = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(5)]
    st = O.AdamState(np.zeros(50), np.zeros(50))
    th = th0.copy()
    for gr in grads:
        th = O.adam_step(th, gr, st, lr=1e-3)
    p = torch.nn.Parameter(torch.tensor(th0))
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for gr in grads:
        opt.zero_grad()
        p.grad = torch.tensor(gr)
        opt.step()
    np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_adam_first_step_closed_form():
    # after one step m_hat = g and s_hat = g^2, so the move is -lr g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    st = O.AdamState(np.zeros(4), np.zeros(4))
    th = O.adam_step(np.zeros(4), g, st, lr=0.1)
    np.testing.assert_allclose(th, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=0)


