"""GPU parity of the hash-encoded INR (Sec. 4, "Hash Enc."; FP32 SIMT path) against the
FP64 oracle: grid evaluation, the weighted VJP of Eq. (2) including the table
scatter (bar: FP32 gradient within 1e-4 relative L2), the chunked VJP beyond one
scratch chunk, and one grad_step (Algorithm 1 plus Adam) on a fan-beam problem."""
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


def oarch(s: synth.ArchSpec) -> O.Arch:
    return O.Arch("hash", s.d, s.width, s.n_hidden, hash_levels=s.hash_levels, hash_feats=s.hash_feats,
                  hash_log2_T=s.hash_log2_T, hash_base=s.hash_base, hash_growth=s.hash_growth)


def kink_free(oa, theta, X, N, tau=1e-4):
    """Points whose ReLU pre-activations all stay at least tau * rms away from 0, where
    FP32 and FP64 take the same mask decisions."""
    _, _, zs, _ = O.forward(oa, np.asarray(theta, np.float64), X, keep=True, N=N)
    ok = np.ones(len(X), bool)
    for z in zs[:-1]:
        ok &= (np.abs(z) >= tau * np.sqrt((z ** 2).mean())).all(axis=1)
    return ok


def hash_spec(d=2, width=64, n_hidden=2, **kw):
    base = dict(hash_levels=6, hash_feats=2, hash_log2_T=10, hash_base=4, hash_growth=1.7)
    base.update(kw)
    return synth.ArchSpec("hash", d, width, n_hidden, **base)


SPECS = [
    hash_spec(),                                                       # dense and hashed levels
    hash_spec(width=128, n_hidden=3, hash_levels=16, hash_feats=4, hash_log2_T=12, hash_base=2,
              hash_growth=1.4),                                        # 64 inputs, fine levels hashed
    hash_spec(width=256, n_hidden=1, hash_levels=3, hash_feats=1, hash_log2_T=16, hash_base=8,
              hash_growth=2.0),                                        # all dense, one hidden layer
    hash_spec(d=3, width=64, hash_levels=5, hash_feats=2, hash_log2_T=11, hash_base=3, hash_growth=1.8),
    hash_spec(d=3, width=128, hash_levels=8, hash_feats=8, hash_log2_T=9, hash_base=2, hash_growth=1.5),
]


def ids(s):
    return f"{s.d}d_w{s.width}x{s.n_hidden}_L{s.hash_levels}F{s.hash_feats}T{s.hash_log2_T}"


@pytest.mark.parametrize("spec", SPECS, ids=ids)
def test_eval_grid_matches_oracle(spec):
    N = 64 if spec.d == 2 else 18
    oa = oarch(spec)
    theta = synth.init_theta(spec, 1, table_scale=0.5).astype(np.float32)
    img = inrct.inr_eval_grid(inrct.mlp_desc(spec, inrct.FP32), cuda(theta), N).cpu().numpy()
    want = O.forward(oa, theta.astype(np.float64), O.grid_coords(spec.d, N), N=N)
    assert rel(img, want) <= 1e-5


@pytest.mark.parametrize("spec", SPECS, ids=ids)
def test_weighted_vjp_matches_oracle(spec):
    N = 64 if spec.d == 2 else 18
    n = N ** spec.d
    oa = oarch(spec)
    theta = synth.init_theta(spec, 2, table_scale=0.5).astype(np.float32)
    v = np.random.default_rng(3).normal(size=n).astype(np.float32)
    idx = synth.index_set(n, 1500, 4)
    idx = idx[kink_free(oa, theta, O.grid_coords(spec.d, N, idx), N)]
    idx = np.concatenate([idx, idx[:7]]).astype(np.int32)      # repeats are allowed
    scale = n / idx.size
    g64, g32 = inrct.inr_weighted_vjp(inrct.mlp_desc(spec, inrct.FP32), cuda(theta), N,
                                      cuda(idx, torch.int32), cuda(v), scale, want_f32=True)
    want = O.vjp(oa, theta.astype(np.float64), O.grid_coords(spec.d, N, idx),
                 scale * v.astype(np.float64)[idx], N=N)
    got = g64.cpu().numpy()
    assert rel(got, want) <= 1e-4
    assert rel(g32.cpu().numpy(), want) <= 1e-4
    # the table block and the MLP block each meet the bar on their own
    nt = oa.table_params
    assert rel(got[:nt], want[:nt]) <= 1e-4
    assert rel(got[nt:], want[nt:]) <= 1e-4
    # entries no listed point touches stay exactly zero
    assert np.all(got[:nt][want[:nt] == 0.0] == 0.0)


def test_vjp_over_several_chunks_matches_oracle():
    """More points than one scratch chunk (2^20): the table gradient is cleared once and
    accumulated over the chunks like the layer gradients."""
    spec = hash_spec(hash_levels=4, hash_log2_T=12, hash_base=16, hash_growth=2.0)
    N = 1100
    n = N * N
    oa = oarch(spec)
    theta = synth.init_theta(spec, 5, table_scale=0.5).astype(np.float32)
    v = np.random.default_rng(6).normal(size=n).astype(np.float32)
    idx = np.arange(n, dtype=np.int64)
    idx = idx[kink_free(oa, theta, O.grid_coords(2, N, idx), N)].astype(np.int32)
    assert idx.size > (1 << 20)
    got = inrct.inr_weighted_vjp(inrct.mlp_desc(spec, inrct.FP32), cuda(theta), N, cuda(idx, torch.int32),
                                 cuda(v), 1.0).cpu().numpy()
    want = O.vjp(oa, theta.astype(np.float64), O.grid_coords(2, N, idx), v.astype(np.float64)[idx], N=N)
    assert rel(got, want) <= 1e-4


@pytest.mark.parametrize("N,levels,growth", [(64, 2, 2.5), (2100, 3, 4.0)], ids=["32bit", "64bit"])
def test_fine_levels_split_their_coordinates_exactly(N, levels, growth):
    """Level coordinates (2k + 1) N_l / (2N) whose numerator exceeds 2^24 (and 2^32) are split
    by the integer paths of the kernel; the VJP (which also carries the forward's layer-1
    input into dW_1) matches the oracle."""
    base = 60000 if N == 64 else 65536
    spec = hash_spec(hash_levels=levels, hash_log2_T=10, hash_base=base, hash_growth=growth)
    n = N * N
    oa = oarch(spec)
    top = O.hash_resolutions(oa)[-1]
    assert 2 * N * top > (1 << 24) and (N < 1000 or 2 * N * top > (1 << 32))
    theta = synth.init_theta(spec, 14, table_scale=0.5).astype(np.float32)
    idx = synth.index_set(n, 800, 15)
    idx = idx[kink_free(oa, theta, O.grid_coords(2, N, idx), N)].astype(np.int32)
    v = np.random.default_rng(16).normal(size=n).astype(np.float32)
    got = inrct.inr_weighted_vjp(inrct.mlp_desc(spec, inrct.FP32), cuda(theta), N, cuda(idx, torch.int32),
                                 cuda(v), 1.0).cpu().numpy()
    want = O.vjp(oa, theta.astype(np.float64), O.grid_coords(2, N, idx), v.astype(np.float64)[idx], N=N)
    assert rel(got, want) <= 1e-4


def test_out_of_range_indices_contribute_nothing():
    """Indices outside [0, n) add nothing.  The two lists differ in length, so the dW
    point splits (and the grouping of their FP32 partial sums) may differ: the bar is
    FP32 reordering, and the oracle over the valid indices alone."""
    spec = hash_spec()
    N = 48
    n = N * N
    oa = oarch(spec)
    theta = synth.init_theta(spec, 7, table_scale=0.5).astype(np.float32)
    v = np.random.default_rng(8).normal(size=n).astype(np.float32)
    idx = synth.index_set(n, 300, 9)
    idx = idx[kink_free(oa, theta, O.grid_coords(2, N, idx), N)].astype(np.int32)
    h = inrct.mlp_desc(spec, inrct.FP32)
    a = inrct.inr_weighted_vjp(h, cuda(theta), N, cuda(idx, torch.int32), cuda(v), 2.0).cpu().numpy()
    bad = np.concatenate([idx, [-1, n, n + 5, -(1 << 30)]]).astype(np.int32)
    b = inrct.inr_weighted_vjp(h, cuda(theta), N, cuda(bad, torch.int32), cuda(v), 2.0).cpu().numpy()
    assert rel(b, a) <= 1e-6
    want = O.vjp(oa, theta.astype(np.float64), O.grid_coords(2, N, idx), 2.0 * v.astype(np.float64)[idx], N=N)
    assert rel(b, want) <= 1e-4


def test_grad_step_matches_oracle():
    g = synth.GeomSpec("fan2d", 64, 24, 97, sod=120.0, sdd=180.0, span=2 * math.pi)
    spec = hash_spec(hash_levels=8, hash_log2_T=9, hash_base=4, hash_growth=1.5)
    oa = oarch(spec)
    og = O.Geometry(g.kind, g.N, g.V, g.A, g.B, g.du, g.dv, g.sod, g.sdd, g.angle0, g.span)
    theta = synth.init_theta(spec, 10, table_scale=0.5).astype(np.float32)
    y = synth.noisy(O.project(og, synth.phantom(2, g.N, 6, 11)), 0.01, 12).astype(np.float32)
    idx = synth.index_set(g.n, g.n // 4, 13)
    idx = idx[kink_free(oa, theta, O.grid_coords(2, g.N, idx), g.N)].astype(np.int32)
    scale = g.n / idx.size
    L0, _, _, v0 = O.backprojected_residual(oa, theta.astype(np.float64), og, y.astype(np.float64))
    want = O.estimator(oa, theta.astype(np.float64), og, v0, idx, scale)
    h = inrct.mlp_desc(spec, inrct.FP32)
    th = cuda(theta)
    m, s = torch.zeros_like(th), torch.zeros_like(th)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros(spec.p, dtype=torch.float64, device="cuda")
    inrct.grad_step(g, h, th, cuda(y), cuda(idx, torch.int32), scale, inrct.adam(lr=1e-3, t=1), m, s, loss, grad)
    torch.cuda.synchronize()
    assert abs(loss.item() - L0) <= 1e-5 * L0
    gg = grad.cpu().numpy()
    assert rel(gg, want) <= 1e-4
    # first Adam step: -lr g / (|g| + eps) wherever the gradient is not zero, up to the
    # FP32 rounding of theta (|theta| < 1: half an ulp is below 6e-8); untouched table
    # entries (zero gradient) do not move
    step = th.double().cpu().numpy() - theta.astype(np.float64)
    assert np.abs(theta).max() < 1.0
    np.testing.assert_allclose(step, -1e-3 * gg / (np.abs(gg) + 1e-8), rtol=2e-5, atol=6e-8)
    assert np.all(step[gg == 0.0] == 0.0)


def test_bf16_is_refused_for_the_hash_encoding():
    spec = hash_spec()
    h = inrct.mlp_desc(spec, inrct.BF16)
    with pytest.raises(RuntimeError, match="hash"):
        inrct.inr_eval_grid(h, cuda(synth.init_theta(spec, 0)), 32)
