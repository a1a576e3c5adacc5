"""GPU checks of the BF16 tcgen05 path: the weight-gradient GEMM against a library
matmul on the same BF16 inputs, and the fused MLP tile engine (grid evaluation,
weighted VJP, virtual loss) against the FP64 oracle (bar: BF16 grad within 1e-2
relative L2 with cosine >= 0.999).  ReLU masks are the oracle's own FP64 decisions;
the only points given no weight are those with a pre-activation within 1e-6 of its
layer's RMS of zero, where FP32-accurate arithmetic may decide either way."""
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


def cos(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("K,M,N,y16", [(64, 128, 64, True), (1000, 128, 256, True),
                                       (70000, 256, 128, False), (4160, 256, 0, True),
                                       (8, 128, 192, True)])
def test_gemm_tn_matches_matmul(K, M, N, y16):
    g = torch.Generator(device="cuda").manual_seed(K + M + N)
    X = torch.randn(K, M, device="cuda", generator=g).bfloat16()
    Y = torch.randn(K, N, device="cuda", generator=g).bfloat16() if N else None
    Y16 = torch.randn(16, K, device="cuda", generator=g).bfloat16() if y16 else None
    C = inrct.gemm_tn(X, Y, Y16).double()
    Xd = X.double()
    if N:
        assert rel(C[:, :N].cpu(), (Xd.T @ Y.double()).cpu()) <= 1e-5
    assert rel(C[:, N].cpu(), Xd.sum(0).cpu()) <= 1e-5
    if y16:
        assert rel(C[:, N + 16:].cpu(), (Xd.T @ Y16.double().T).cpu()) <= 1e-5
    else:
        assert float(C[:, N + 16:].abs().max()) == 0.0


def arch_pair(spec, seed=0):
    B = synth.fourier_matrix(spec.n_feat, spec.d, spec.sigma, seed) if spec.kind == "ffn" else None
    B32 = B.astype(np.float32) if B is not None else None
    oa = O.Arch(spec.kind, spec.d, spec.width, spec.n_hidden, spec.n_feat,
                B32.astype(np.float64) if B32 is not None else None, spec.omega0)
    return oa, B32


ARCHS = [
    synth.ArchSpec("siren", 2, 256, 5, omega0=30.0),        # 512^2 fan workload's network
    synth.ArchSpec("ffn", 3, 256, 4, n_feat=256, sigma=8.0),  # 256^3 cone workload's network
    synth.ArchSpec("siren", 2, 128, 3, omega0=30.0),        # batched workload's network
    synth.ArchSpec("ffn", 2, 128, 2, n_feat=32, sigma=4.0),
]


@pytest.mark.parametrize("spec", ARCHS, ids=lambda a: f"{a.kind}{a.d}d_{a.width}x{a.n_hidden}")
def test_eval_grid_bf16_matches_oracle(spec):
    N = 67 if spec.d == 2 else 21          # ragged: the grid is not a multiple of the tile
    oa, B32 = arch_pair(spec, 1)
    theta = synth.init_theta(spec, 2).astype(np.float32)
    h = inrct.mlp_desc(spec, inrct.BF16, B32)
    img = inrct.inr_eval_grid(h, cuda(theta), N).cpu().numpy()
    want = O.forward(oa, theta.astype(np.float64), O.grid_coords(spec.d, N))
    err = rel(img, want)
    assert err <= 2e-2, err


@pytest.mark.parametrize("spec", [a for a in ARCHS if a.kind == "ffn"],
                         ids=lambda a: f"{a.kind}{a.d}d_{a.width}x{a.n_hidden}")
def test_eval_grid_coefficients_as_launch_parameters_change_nothing(spec):
    """With B_host the Fourier coefficients reach the kernel as launch parameters instead of a
    shared-memory table: the image must be bit-identical (the same values, the same arithmetic)."""
    N = 67 if spec.d == 2 else 21
    _, B32 = arch_pair(spec, 1)
    theta = cuda(synth.init_theta(spec, 2).astype(np.float32))
    h = inrct.mlp_desc(spec, inrct.BF16, B32)
    assert h.desc.B_host
    with_params = inrct.inr_eval_grid(h, theta, N)
    h.desc.B_host = None
    from_shared = inrct.inr_eval_grid(h, theta, N)
    assert torch.equal(with_params, from_shared)


def kink_free(oa, theta, X, tau=1e-6):
    """Points whose ReLU pre-activations (FP64) all stay at least tau * rms away from zero."""
    if oa.kind != "ffn":
        return np.ones(len(X), bool)
    _, _, zs, _ = O.forward(oa, np.asarray(theta, np.float64), X, keep=True)
    ok = np.ones(len(X), bool)
    for z in zs[:-1]:
        ok &= (np.abs(z) >= tau * np.sqrt((z ** 2).mean())).all(axis=1)
    return ok


@pytest.mark.parametrize("spec", ARCHS, ids=lambda a: f"{a.kind}{a.d}d_{a.width}x{a.n_hidden}")
def test_weighted_vjp_bf16_matches_oracle(spec):
    N = 67 if spec.d == 2 else 21
    n = N ** spec.d
    oa, B32 = arch_pair(spec, 3)
    theta = synth.init_theta(spec, 4).astype(np.float32)
    v = np.random.default_rng(5).normal(size=n).astype(np.float32)
    idx = synth.index_set(n, 1337, 6)
    idx = idx[kink_free(oa, theta, O.grid_coords(spec.d, N, idx))]
    idx = np.concatenate([idx, idx[:2], idx[:1]]).astype(np.int32)      # repeats are allowed
    scale = n / idx.size
    h = inrct.mlp_desc(spec, inrct.BF16, B32)
    g64, g32 = inrct.inr_weighted_vjp(h, cuda(theta), N, cuda(idx, torch.int32), cuda(v), scale,
                                      want_f32=True)
    want = O.vjp(oa, theta.astype(np.float64), O.grid_coords(spec.d, N, idx),
                 scale * v.astype(np.float64)[idx])
    got = g64.cpu().numpy()
    assert rel(got, want) <= 1e-2, rel(got, want)
    assert cos(got, want) >= 0.999
    assert rel(g32.cpu().numpy(), got) <= 1e-6


@pytest.mark.parametrize("spec", ARCHS, ids=lambda a: f"{a.kind}{a.d}d_{a.width}x{a.n_hidden}")
def test_virtual_loss_bf16_matches_oracle(spec):
    """inr_virtual_loss: the value of Eq. 3 from the VJP's forward pass, and the same gradient
    as inr_weighted_vjp, bit for bit."""
    N = 67 if spec.d == 2 else 21
    n = N ** spec.d
    oa, B32 = arch_pair(spec, 3)
    theta = synth.init_theta(spec, 4).astype(np.float32)
    v = np.random.default_rng(7).uniform(0.5, 1.5, size=n).astype(np.float32)   # a coherent sum
    idx = synth.index_set(n, 1337, 8)
    scale = n / idx.size
    h = inrct.mlp_desc(spec, inrct.BF16, B32)
    val, g = inrct.inr_virtual_loss(h, cuda(theta), N, cuda(idx, torch.int32), cuda(v), scale)
    g_ref = inrct.inr_weighted_vjp(h, cuda(theta), N, cuda(idx, torch.int32), cuda(v), scale)
    f = O.forward(oa, theta.astype(np.float64), O.grid_coords(spec.d, N, idx))
    vi = v.astype(np.float64)[idx]
    want = scale * float(vi @ f)
    # per-point bound: f to BF16 accuracy (SIREN), or to FP32 accuracy where the forward stages
    # run on split operands (ReLU networks)
    tol = (1e-4 if spec.kind == "ffn" else 1e-2) * scale * float(np.abs(vi * f).sum())
    assert abs(val.item() - want) <= tol, (val.item(), want, tol)
    assert torch.equal(g, g_ref)


def test_feature_sin_cos_accuracy():
    """The Fourier features' sin / cos (exact phase reduction to [-1/2, 1/2], then sincospif)
    against an FP64 reference: about an FP32 ulp (2 ulp where the value exceeds 1e-4, and
    1.2e-7 absolute everywhere), and exact at the quadrant points."""
    rng = np.random.default_rng(8)
    x = np.r_[rng.uniform(-1, 1, 1 << 20), np.linspace(-1, 1, 4097), [1e-30, -1e-30, 2 ** -24]].astype(np.float32)
    s, c = inrct.sincospi(torch.tensor(x, device="cuda"))
    s, c = s.double().cpu().numpy(), c.double().cpu().numpy()
    xs = x.astype(np.float64)
    rs, rc = np.sin(np.pi * xs), np.cos(np.pi * xs)
    assert np.abs(s - rs).max() <= 1.2e-7 and np.abs(c - rc).max() <= 1.2e-7
    for got, ref in ((s, rs), (c, rc)):
        big = np.abs(ref) > 1e-4
        ulp = np.spacing(np.abs(ref[big]).astype(np.float32)).astype(np.float64)
        assert (np.abs(got[big] - ref[big]) / ulp).max() <= 2.0
    q = np.float32([-1, -0.5, 0, 0.5, 1])
    sq, cq = inrct.sincospi(torch.tensor(q, device="cuda"))
    assert [abs(v) for v in sq.cpu().tolist()] == [0.0, 1.0, 0.0, 1.0, 0.0]
    assert [abs(v) for v in cq.cpu().tolist()] == [1.0, 0.0, 1.0, 0.0, 1.0]
