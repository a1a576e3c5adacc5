"""Pins of the oracle's multiresolution hash encoding (the "Hash Enc." INR of Sec. 4).

Nothing here compares the oracle with itself: the interpolation is checked against
closed forms (partition of unity; multilinear interpolation reproduces affine
functions exactly on dense levels), the spatial hash against the same definition
evaluated with Python's unbounded integers, and the reverse mode (tables and MLP)
against torch autograd in FP64 and against central differences (the encoding is
linear in the table entries and the ReLU network piecewise linear, so differences there
are exact unless a step crosses a kink).
"""
import numpy as np
import pytest

import oracle as O


def _arch(d=2, **kw):
    base = dict(kind="hash", d=d, width=16, n_hidden=2, hash_levels=4, hash_feats=2, hash_log2_T=10,
                hash_base=4, hash_growth=1.7)
    base.update(kw)
    return O.Arch(**base)


def _theta(arch, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, arch.p)


@pytest.mark.parametrize("d", [2, 3])
def test_interpolation_weights_are_a_partition_of_unity(d):
    arch = _arch(d, hash_levels=5, hash_log2_T=8)
    N = 11 if d == 2 else 7
    K = np.stack(np.meshgrid(*[np.arange(N)] * d, indexing="ij"), -1).reshape(-1, d)
    for l in range(arch.hash_levels):
        idx, w = O.hash_corners(arch, K, N, l)
        assert np.all(w >= 0) and np.allclose(w.sum(1), 1.0, atol=1e-15)
        assert idx.min() >= 0 and idx.max() < (1 << arch.hash_log2_T)


@pytest.mark.parametrize("d", [2, 3])
def test_dense_levels_reproduce_affine_functions_exactly(d):
    """With table entry a . (c / N_l) + e at vertex c of every dense level, each level's
    feature is a . (x + 1)/2 + e at every pixel centre x (multilinear interpolation is exact
    for affine functions, and p / N_l = (x + 1)/2)."""
    arch = _arch(d, hash_levels=3, hash_base=3, hash_growth=2.0, hash_log2_T=12 if d == 3 else 10)
    res = O.hash_resolutions(arch)
    T = 1 << arch.hash_log2_T
    assert all((r + 1) ** d <= T for r in res)     # every level is dense
    rng = np.random.default_rng(1)
    a = rng.normal(size=(arch.hash_feats, d))
    e = rng.normal(size=arch.hash_feats)
    theta = np.zeros(arch.p)
    tab = theta[:arch.table_params].reshape(arch.hash_levels, T, arch.hash_feats)
    for l, Nl in enumerate(res):
        grid = np.stack(np.meshgrid(*[np.arange(Nl + 1)] * d, indexing="ij"), -1).reshape(-1, d)
        dense_idx = sum(grid[:, k] * (Nl + 1) ** k for k in range(d))
        tab[l][dense_idx] = (grid / Nl) @ a.T + e
    N = 13
    X = O.grid_coords(d, N)
    feats = O.hash_encode(arch, theta, X, N)
    want = ((X + 1) / 2) @ a.T + e
    for l in range(arch.hash_levels):
        assert np.allclose(feats[:, 2 * l:2 * l + 2], want, rtol=0, atol=1e-13)


def test_spatial_hash_matches_the_definition_in_python_integers():
    arch = _arch(3, hash_levels=6, hash_base=8, hash_growth=2.0, hash_log2_T=9)
    N = 9
    rng = np.random.default_rng(2)
    K = rng.integers(0, N, size=(40, 3))
    T = 1 << arch.hash_log2_T
    for l, Nl in enumerate(O.hash_resolutions(arch)):
        if (Nl + 1) ** 3 <= T:
            continue
        idx, _ = O.hash_corners(arch, K, N, l)
        for i in range(K.shape[0]):
            c0 = [((2 * int(K[i, k]) + 1) * Nl) // (2 * N) for k in range(3)]
            for v in range(8):
                c = [c0[k] + ((v >> k) & 1) for k in range(3)]
                h = 0
                for k in range(3):
                    h ^= (c[k] * O.HASH_PRIMES[k]) % (1 << 32)
                assert idx[i, v] == h % T


def test_vjp_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    arch = _arch(2, hash_levels=4, hash_log2_T=6, hash_base=5, hash_growth=1.9)  # mixes dense and hashed
    N = 10
    theta = _theta(arch, 3) * 0.5
    I = np.array([0, 3, 11, 27, 54, 61, 77, 98, 99])
    X = O.grid_coords(2, N, I)
    w = np.random.default_rng(4).normal(size=I.size)
    got = O.vjp(arch, theta, X, w, N=N)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    T = 1 << arch.hash_log2_T
    tab = th[:arch.table_params].reshape(arch.hash_levels, T, arch.hash_feats)
    K = O.grid_index_of(X, N)
    feats = []
    for l in range(arch.hash_levels):
        idx, wts = O.hash_corners(arch, K, N, l)
        feats.append((torch.tensor(wts)[:, :, None] * tab[l][torch.tensor(idx)]).sum(1))
    h = torch.cat(feats, 1)
    off = arch.table_params
    shapes = arch.layer_shapes()
    for li, (o, i) in enumerate(shapes):
        Wl = th[off:off + o * i].reshape(o, i)
        off += o * i
        bl = th[off:off + o]
        off += o
        h = h @ Wl.T + bl
        if li < len(shapes) - 1:
            h = torch.relu(h)
    (h[:, 0] @ torch.tensor(w)).backward()
    assert np.allclose(got, th.grad.numpy(), rtol=1e-12, atol=1e-12)


def test_table_gradient_equals_central_differences():
    arch = _arch(2, hash_levels=3, hash_log2_T=5, hash_base=6, hash_growth=2.0)
    N = 8
    theta = _theta(arch, 5) * 0.3
    I = np.arange(N * N)
    X = O.grid_coords(2, N, I)
    w = np.random.default_rng(6).normal(size=I.size)
    g = O.vjp(arch, theta, X, w, N=N)
    f = lambda t: float(w @ O.forward(arch, t, X, N=N))
    rng = np.random.default_rng(7)
    for j in rng.choice(arch.table_params, 12, replace=False):
        h = 1e-4
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        assert abs((f(tp) - f(tm)) / (2 * h) - g[j]) <= 1e-8 * max(1.0, abs(g[j]))


def test_three_d_table_gradient_equals_central_differences():
    """The 3-D reverse mode (eight trilinear corners per level, dense and hashed levels) against
    central differences of the forward pass in table entries and in MLP weights."""
    arch = _arch(3, hash_levels=3, hash_log2_T=7, hash_base=2, hash_growth=2.5)  # N_l 2 dense; 5, 12 hashed
    N = 6
    theta = _theta(arch, 9) * 0.3
    I = np.arange(N ** 3)
    X = O.grid_coords(3, N, I)
    w = np.random.default_rng(10).normal(size=I.size)
    g = O.vjp(arch, theta, X, w, N=N)
    f = lambda t: float(w @ O.forward(arch, t, X, N=N))
    rng = np.random.default_rng(11)
    touched = np.flatnonzero(g[:arch.table_params])
    picks = np.concatenate([rng.choice(touched, 16, replace=False),
                            arch.table_params + rng.choice(arch.p - arch.table_params, 8, replace=False)])
    for j in picks:
        h = 1e-4
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        assert abs((f(tp) - f(tm)) / (2 * h) - g[j]) <= 1e-8 * max(1.0, abs(g[j])), j
