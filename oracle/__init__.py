"""FP64 CPU oracle for the memory-efficient INR gradient for CT.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
statement of what the CUDA path computes, written from the paper.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the product package and
never imports it; both sides only consume the same seeded inputs.

Contents, each following the passage named in its docstring:

* grid coordinates (Sec. 3: regular grid x_1..x_n inside the FOV);
* the INR f_theta: Fourier-feature ReLU MLP and SIREN (Sec. 4, the two
  architectures with a forward/backward we can write out), with a
  hand-derived reverse mode;
* the Joseph projector P and its transpose (``joseph.c``; Sec. 3 writes the
  projection as P E{f});
* the LS loss and its residual (Sec. 2, Sec. 3 note after Algorithm 1);
* the full chain-rule gradient (Sec. 3, the sum over all n grid points);
* the subsampled estimator, Eq. (2), and the virtual loss, Eq. (3);
* Algorithm 1 composed with an Adam update (Sec. 4 trains with Adam);
* the ramp filter F of the FLS loss (Sec. 2) as a plain convolution.

Everything is FP64.  Parity pins: see ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "joseph.c")

PAR2D, FAN2D, CONE3D = 0, 1, 2
_KIND = {"par2d": PAR2D, "fan2d": FAN2D, "cone3d": CONE3D}


def build(force: bool = False) -> str:
    """Compile ``joseph.c`` into ``liboracle.so`` with gcc (FP64, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-std=c11", _SRC, "-o", _SO + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_SO + ".tmp", _SO)
    return _SO


class _Geom(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("N", ctypes.c_int), ("V", ctypes.c_int),
                ("A", ctypes.c_int), ("B", ctypes.c_int),
                ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("sod", ctypes.c_double), ("sdd", ctypes.c_double),
                ("angle0", ctypes.c_double), ("span", ctypes.c_double)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        g = ctypes.POINTER(_Geom)
        _lib.orc_project.argtypes = [g, dp, dp]
        _lib.orc_backproject.argtypes = [g, dp, dp]
        _lib.orc_project_at.argtypes = [g, dp, ctypes.c_int64, i64p, dp]
        _lib.orc_backproject_at.argtypes = [g, dp, ctypes.c_int64, i64p, dp]
        _lib.orc_matrix_entry.argtypes = [g, ctypes.c_int64, ctypes.c_int64]
        _lib.orc_matrix_entry.restype = ctypes.c_double
        _lib.orc_num_rays.argtypes = [g]
        _lib.orc_num_rays.restype = ctypes.c_int64
        _lib.orc_ray.argtypes = [g, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
    return _lib


# ----------------------------------------------------------------------------
# Geometry (Sec. 3: P in R^{m x n}; the paper fixes no scan conventions, these are readings)
# ----------------------------------------------------------------------------
@dataclass
class Geometry:
    """Scan geometry.  Lengths in pixel units at the isocentre; angles in radians.

    kind: 'par2d' | 'fan2d' | 'cone3d'.  N: grid side.  V: views over
    [angle0, angle0 + span).  A: detector bins (columns).  B: detector rows
    (cone only).  du, dv: bin pitch at the isocentre in pixels.  sod, sdd:
    source-to-isocentre and source-to-detector distances in pixels.
    """
    kind: str
    N: int
    V: int
    A: int
    B: int = 1
    du: float = 1.0
    dv: float = 1.0
    sod: float = 1000.0
    sdd: float = 1500.0
    angle0: float = 0.0
    span: float = float(np.pi)
    fov: int = 0   # 0: the whole grid; 1: the inscribed disk (2-D) / cylinder (3-D), see fov_mask

    @property
    def d(self) -> int:
        return 3 if self.kind == "cone3d" else 2

    @property
    def n(self) -> int:
        return self.N ** self.d

    @property
    def m(self) -> int:
        return self.V * (self.B if self.kind == "cone3d" else 1) * self.A

    @property
    def sino_shape(self):
        return (self.V, self.B, self.A) if self.kind == "cone3d" else (self.V, self.A)

    @property
    def img_shape(self):
        return (self.N,) * self.d

    def _c(self) -> _Geom:
        return _Geom(_KIND[self.kind], self.N, self.V, self.A,
                     self.B if self.kind == "cone3d" else 1,
                     self.du, self.dv, self.sod, self.sdd, self.angle0, self.span)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def project(g: Geometry, img) -> np.ndarray:
    """z = P x for every ray (Sec. 3).  img: shape (N,)*d or flat; returns flat [m]."""
    x = np.ascontiguousarray(np.asarray(img, dtype=np.float64).reshape(-1))
    assert x.size == g.n
    z = np.empty(g.m, dtype=np.float64)
    gc = g._c()
    _L().orc_project(ctypes.byref(gc), _dp(x), _dp(z))
    return z


def backproject(g: Geometry, sino) -> np.ndarray:
    """v = P^T r (Sec. 3, v = P^T r), as the literal transpose of ``project``."""
    r = np.ascontiguousarray(np.asarray(sino, dtype=np.float64).reshape(-1))
    assert r.size == g.m
    v = np.empty(g.n, dtype=np.float64)
    gc = g._c()
    _L().orc_backproject(ctypes.byref(gc), _dp(r), _dp(v))
    return v


def project_at(g: Geometry, img, rays) -> np.ndarray:
    """(P x)_r for the listed flat ray indices."""
    x = np.ascontiguousarray(np.asarray(img, dtype=np.float64).reshape(-1))
    rr = np.ascontiguousarray(np.asarray(rays, dtype=np.int64))
    out = np.empty(rr.size, dtype=np.float64)
    gc = g._c()
    _L().orc_project_at(ctypes.byref(gc), _dp(x), rr.size,
                        rr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out))
    return out


def backproject_at(g: Geometry, sino, pix) -> np.ndarray:
    """(P^T r)_i for the listed flat pixel indices, from the matrix entries directly."""
    r = np.ascontiguousarray(np.asarray(sino, dtype=np.float64).reshape(-1))
    pp = np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
    out = np.empty(pp.size, dtype=np.float64)
    gc = g._c()
    _L().orc_backproject_at(ctypes.byref(gc), _dp(r), pp.size,
                            pp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out))
    return out


def matrix_entry(g: Geometry, ray: int, pix: int) -> float:
    gc = g._c()
    return _L().orc_matrix_entry(ctypes.byref(gc), int(ray), int(pix))


def ray(g: Geometry, k: int, row: int, col: int):
    """(point, unit direction) of one ray, both length-3 arrays."""
    s = np.zeros(3)
    e = np.zeros(3)
    gc = g._c()
    _L().orc_ray(ctypes.byref(gc), k, row, col, _dp(s), _dp(e))
    return s, e


# ----------------------------------------------------------------------------
# Grid (Sec. 3: regular grid of coordinates x_1..x_n in [-1, 1]^d)
# ----------------------------------------------------------------------------
def grid_coords(d: int, N: int, idx=None) -> np.ndarray:
    """Pixel/voxel centres c_k = -1 + (k + 1/2) 2/N; flat index row-major, x fastest.

    Returns an (n, d) FP64 array whose column 0 is x, 1 is y, 2 is z.
    """
    if idx is None:
        idx = np.arange(N ** d, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    c = lambda k: -1.0 + (k.astype(np.float64) + 0.5) * (2.0 / N)
    cols = [c(idx % N), c((idx // N) % N)]
    if d == 3:
        cols.append(c(idx // (N * N)))
    return np.stack(cols, axis=1)


def fov_mask(d: int, N: int, idx=None) -> np.ndarray:
    """Field of view (Sec. 3 samples the INR on the grid points inside a FOV mask; its shape
    is not given, the reading is the inscribed disk, a cylinder along z in 3-D): pixel centre
    (x, y) inside iff x^2 + y^2 <= 1, tested exactly in integers as
    (2 k_x + 1 - N)^2 + (2 k_y + 1 - N)^2 <= N^2 (x = (2 k_x + 1 - N) / N)."""
    if idx is None:
        idx = np.arange(N ** d, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    a = 2 * (idx % N) + 1 - N
    b = 2 * ((idx // N) % N) + 1 - N
    return a * a + b * b <= N * N


def fov_indices(g) -> np.ndarray:
    """Flat indices of the grid points the method samples: all of them, or those in the FOV."""
    idx = np.arange(g.n, dtype=np.int64)
    return idx[fov_mask(g.d, g.N, idx)] if g.fov else idx


# ----------------------------------------------------------------------------
# INR f_theta (Sec. 4: Fourier-feature ReLU networks and SIREN)
# ----------------------------------------------------------------------------
@dataclass
class Arch:
    """INR architecture.

    kind 'ffn':   gamma(x) = [cos(2 pi B x), sin(2 pi B x)] (F features each),
                  then n_hidden layers Linear + ReLU of the given width, then
                  Linear(width, 1).
    kind 'siren': n_hidden layers h = sin(omega0 (W h + b)) (the first takes
                  x itself), then Linear(width, 1).
    kind 'hash':  multiresolution hash encoding (``hash_encode``: hash_levels levels of
                  hash_feats features, tables of 2^hash_log2_T entries), then n_hidden
                  layers Linear + ReLU and Linear(width, 1).
    theta layout: the hash tables first (hash only, [level][entry][feature]), then for
    every layer in order, W row-major [out][in], then b [out].
    """
    kind: str
    d: int
    width: int
    n_hidden: int
    n_feat: int = 0
    B: np.ndarray | None = None   # F x d, FFN only
    omega0: float = 30.0
    hash_levels: int = 16
    hash_feats: int = 2
    hash_log2_T: int = 19
    hash_base: int = 16
    hash_growth: float = 1.5

    @property
    def d_in(self) -> int:
        if self.kind == "hash":
            return self.hash_levels * self.hash_feats
        return 2 * self.n_feat if self.kind == "ffn" else self.d

    @property
    def table_params(self) -> int:
        return self.hash_levels * (1 << self.hash_log2_T) * self.hash_feats if self.kind == "hash" else 0

    def layer_shapes(self):
        shapes = [(self.width, self.d_in)]
        shapes += [(self.width, self.width)] * (self.n_hidden - 1)
        shapes.append((1, self.width))
        return shapes

    @property
    def p(self) -> int:
        return self.table_params + sum(o * i + o for o, i in self.layer_shapes())


def unpack(arch: Arch, theta):
    """Split the flat theta into [(W_l, b_l)] views in layer order (after the hash tables)."""
    theta = np.asarray(theta, dtype=np.float64)
    out, off = [], arch.table_params
    for o, i in arch.layer_shapes():
        W = theta[off:off + o * i].reshape(o, i)
        off += o * i
        b = theta[off:off + o]
        off += o
        out.append((W, b))
    assert off == theta.size, (off, theta.size)
    return out


# ----------------------------------------------------------------------------
# Multiresolution hash encoding (the "Hash Enc." INR of Sec. 4; the paper gives no details,
# the readings are the usual ones of multiresolution hash encodings): level l has
# resolution N_l = floor(base * growth^l); a point's level coordinate is p = (x + 1)/2 * N_l
# per axis; its 2^d surrounding vertices (integer coordinates in [0, N_l]) are looked up
# densely (index sum_k c_k (N_l+1)^k) when (N_l+1)^d <= T, else by the spatial hash
# (XOR over k of c_k * pi_k, in 32-bit unsigned arithmetic, pi = (1, 2654435761, 805459861))
# modulo T = 2^log2_T; the level's features are the multilinear interpolation of the
# vertices' table entries.
# ----------------------------------------------------------------------------
HASH_PRIMES = (1, 2654435761, 805459861)


def hash_resolutions(arch: Arch) -> list[int]:
    return [int(np.floor(arch.hash_base * arch.hash_growth ** l)) for l in range(arch.hash_levels)]


def grid_index_of(X: np.ndarray, N: int) -> np.ndarray:
    """Integer pixel indices k of pixel centres x = (2k + 1 - N)/N (exact)."""
    return np.rint((np.asarray(X, dtype=np.float64) * N + N - 1) / 2).astype(np.int64)


def hash_corners(arch: Arch, K: np.ndarray, N: int, l: int):
    """Vertex table indices [n, 2^d] and interpolation weights [n, 2^d] of level l for points
    with integer grid indices K [n, d] on an N^d grid.  The level coordinate of index k is
    (2k + 1) N_l / (2N); its integer part and fraction are formed exactly from that ratio."""
    Nl = hash_resolutions(arch)[l]
    T = 1 << arch.hash_log2_T
    num = (2 * K + 1) * Nl                       # level coordinate = num / (2N)
    c0 = num // (2 * N)
    fr = (num % (2 * N)) / (2.0 * N)
    n, d = K.shape
    dense = (Nl + 1) ** d <= T
    idx = np.zeros((n, 1 << d), dtype=np.int64)
    wts = np.ones((n, 1 << d))
    for v in range(1 << d):
        c = c0 + np.array([(v >> k) & 1 for k in range(d)])[None, :]
        for k in range(d):
            wts[:, v] *= np.where((v >> k) & 1, fr[:, k], 1.0 - fr[:, k])
        if dense:
            idx[:, v] = sum(c[:, k] * (Nl + 1) ** k for k in range(d))
        else:
            h = np.zeros(n, dtype=np.uint64)
            for k in range(d):
                h ^= (c[:, k].astype(np.uint64) * np.uint64(HASH_PRIMES[k])) & np.uint64(0xFFFFFFFF)
            idx[:, v] = (h & np.uint64(T - 1)).astype(np.int64)
    return idx, wts


def hash_tables(arch: Arch, theta) -> np.ndarray:
    """The tables as [level][entry][feature] (a view of theta)."""
    T = 1 << arch.hash_log2_T
    return np.asarray(theta, dtype=np.float64)[:arch.table_params].reshape(arch.hash_levels, T, arch.hash_feats)


def hash_encode(arch: Arch, theta, X: np.ndarray, N: int) -> np.ndarray:
    """Concatenated level features [n, levels * feats] of the pixel centres X of an N^d grid."""
    K = grid_index_of(X, N)
    tab = hash_tables(arch, theta)
    out = []
    for l in range(arch.hash_levels):
        idx, wts = hash_corners(arch, K, N, l)
        out.append(np.einsum("nv,nvf->nf", wts, tab[l][idx]))
    return np.concatenate(out, axis=1)


def encode(arch: Arch, X: np.ndarray, theta=None, N: int | None = None) -> np.ndarray:
    """Network input: gamma(x) for FFN (cos block first, then sin), x for SIREN, the hash
    encoding (needs theta and the grid side N) for hash."""
    if arch.kind == "hash":
        return hash_encode(arch, theta, X, N)
    X = np.asarray(X, dtype=np.float64)
    if arch.kind == "ffn":
        P = 2.0 * np.pi * (X @ np.asarray(arch.B, dtype=np.float64).T)
        return np.concatenate([np.cos(P), np.sin(P)], axis=1)
    return X


def forward(arch: Arch, theta, X: np.ndarray, keep: bool = False, N: int | None = None):
    """f_theta(x_i) for every row of X.  With keep=True also returns the
    per-layer inputs h_{l-1}, pre-activations z_l and ReLU masks used by ``vjp``
    (a mask is z > 0, decided on the FP64 pre-activation)."""
    layers = unpack(arch, theta)
    h = encode(arch, X, theta, N)
    hs, zs, masks = [h], [], []
    for li, (W, b) in enumerate(layers):
        z = h @ W.T + b
        zs.append(z)
        if li == len(layers) - 1:
            h = z
        elif arch.kind in ("ffn", "hash"):
            m = z > 0.0
            masks.append(m)
            h = np.where(m, z, 0.0)
        else:
            h = np.sin(arch.omega0 * z)
        hs.append(h)
    f = h[:, 0]
    return (f, hs, zs, masks) if keep else f


def vjp(arch: Arch, theta, X: np.ndarray, w: np.ndarray, N: int | None = None) -> np.ndarray:
    """sum_i w_i grad_theta f_theta(x_i), by reverse mode written out layer by layer.

    This is the Jacobian-transpose product [d E{f}/d theta]^T w of Sec. 3.
    ReLU'(0) is taken as 0.
    """
    layers = unpack(arch, theta)
    _, hs, zs, masks = forward(arch, theta, X, keep=True, N=N)
    w = np.asarray(w, dtype=np.float64)
    grads = [None] * len(layers)
    # df/dz_out = 1, weighted per point by w_i
    delta = w[:, None]                                  # (n, 1)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        h_in = hs[li]
        grads[li] = (delta.T @ h_in, delta.sum(axis=0))   # dW = delta^T h, db = sum delta
        g_h = delta @ W                                 # dL/dh_{li}
        if li == 0:
            break
        z_prev = zs[li - 1]
        if arch.kind in ("ffn", "hash"):
            delta = g_h * masks[li - 1]
        else:
            delta = g_h * (arch.omega0 * np.cos(arch.omega0 * z_prev))
    flat = []
    if arch.kind == "hash":
        # the encoding is linear in the table entries: each vertex entry receives its
        # interpolation weight times the gradient of its level's feature
        gt = np.zeros_like(hash_tables(arch, theta))
        K = grid_index_of(X, N)
        F = arch.hash_feats
        for l in range(arch.hash_levels):
            idx, wts = hash_corners(arch, K, N, l)
            for v in range(idx.shape[1]):
                np.add.at(gt[l], idx[:, v], wts[:, v:v + 1] * g_h[:, l * F:(l + 1) * F])
        flat.append(gt.reshape(-1))
    for gW, gb in grads:
        flat.append(gW.reshape(-1))
        flat.append(gb.reshape(-1))
    return np.concatenate(flat)


# ----------------------------------------------------------------------------
# Loss, full gradient, estimator (Sec. 2, Sec. 3, Eq. (2), Eq. (3), Algorithm 1)
# ----------------------------------------------------------------------------
def ls_loss(z, y):
    """L_LS(z, y) = 1/2 ||z - y||^2 and its gradient r = z - y (Sec. 2; Sec. 3)."""
    r = np.asarray(z, dtype=np.float64) - np.asarray(y, dtype=np.float64)
    return 0.5 * float(r @ r), r


def evaluate_image(arch: Arch, theta, g: Geometry) -> np.ndarray:
    """E{f_theta} = [f(x_1) .. f(x_n)] on the grid (Sec. 3), flat; zero outside the FOV
    when the geometry has one."""
    x = forward(arch, theta, grid_coords(g.d, g.N), N=g.N)
    return x * fov_mask(g.d, g.N) if g.fov else x


def backprojected_residual(arch: Arch, theta, g: Geometry, y):
    """Algorithm 1, its projection and backprojection: z = P E{f}, v = P^T dL/dz.  Returns (L, z, r, v)."""
    x = evaluate_image(arch, theta, g)
    z = project(g, x)
    L, r = ls_loss(z, y)
    v = backproject(g, r)
    return L, z, r, v


def full_gradient(arch: Arch, theta, g: Geometry, y):
    """grad L(theta) = sum_{i=1..n} v_i grad f(x_i) over the sampled grid points (Sec. 3).
    Returns (L, grad, v)."""
    L, _, _, v = backprojected_residual(arch, theta, g, y)
    I = fov_indices(g)
    grad = vjp(arch, theta, grid_coords(g.d, g.N, I), np.asarray(v, dtype=np.float64)[I], N=g.N)
    return L, grad, v


def estimator(arch: Arch, theta, g: Geometry, v, I, scale=None) -> np.ndarray:
    """Eq. (2): (n/|I|) sum_{i in I} v_i grad f(x_i), for the given index set I.

    ``scale`` defaults to n/|I|; v is the backprojected residual (P^T r).
    """
    I = np.asarray(I, dtype=np.int64)
    n = fov_indices(g).size          # the number of sampled points (all, or those in the FOV)
    if scale is None:
        scale = n / I.size
    if g.fov:                        # listed points outside the FOV contribute nothing
        I = I[fov_mask(g.d, g.N, I)]
    X = grid_coords(g.d, g.N, I)
    return vjp(arch, theta, X, scale * np.asarray(v, dtype=np.float64)[I], N=g.N)


def virtual_loss(arch: Arch, theta, g: Geometry, v, I, scale=None) -> float:
    """Eq. (3): (n/|I|) sum_{i in I} v_i f(x_i), with v held constant."""
    I = np.asarray(I, dtype=np.int64)
    if scale is None:
        scale = fov_indices(g).size / I.size
    if g.fov:
        I = I[fov_mask(g.d, g.N, I)]
    X = grid_coords(g.d, g.N, I)
    return float(scale * (np.asarray(v, dtype=np.float64)[I] @ forward(arch, theta, X, N=g.N)))


@dataclass
class AdamState:
    m: np.ndarray
    s: np.ndarray
    t: int = 0


def adam_step(theta, grad, st: AdamState, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update with bias correction (Kingma & Ba; the paper trains with Adam
    and gives no hyper-parameters, so these are the usual defaults)."""
    st.t += 1
    st.m = beta1 * st.m + (1.0 - beta1) * grad
    st.s = beta2 * st.s + (1.0 - beta2) * grad * grad
    mhat = st.m / (1.0 - beta1 ** st.t)
    shat = st.s / (1.0 - beta2 ** st.t)
    return theta - lr * mhat / (np.sqrt(shat) + eps)


def grad_step(arch: Arch, theta, g: Geometry, y, I, st: AdamState, lr: float,
              scale=None, beta1=0.9, beta2=0.999, eps=1e-8):
    """Algorithm 1 followed by an Adam update.  Returns (new_theta, L, ghat)."""
    L, _, _, v = backprojected_residual(arch, theta, g, y)
    ghat = estimator(arch, theta, g, v, I, scale)
    return adam_step(theta, ghat, st, lr, beta1, beta2, eps), L, ghat


# ----------------------------------------------------------------------------
# FLS loss (Sec. 2: L_FLS(z, y) = 1/2 (z - y)^T F (z - y), F a ramp filter)
# ----------------------------------------------------------------------------
def ramp_kernel(A: int, tau: float) -> np.ndarray:
    """Band-limited ramp (Ram-Lak) taps h[k], k = -(A-1)..(A-1), sampled at pitch tau
    (Kak & Slaney's FBP kernel): h[0] = 1/(4 tau^2), h[odd k] = -1/(pi^2 k^2 tau^2),
    h[even k != 0] = 0."""
    k = np.arange(-(A - 1), A)
    h = np.zeros(k.size)
    h[k == 0] = 1.0 / (4 * tau * tau)
    odd = (k % 2) != 0
    h[odd] = -1.0 / (np.pi ** 2 * k[odd].astype(np.float64) ** 2 * tau * tau)
    return h


def ramp_filter(g: Geometry, r) -> np.ndarray:
    """F r: every detector row (one view; one row v for the cone) convolved along the
    bin axis with tau * h, tau = du * D, bins outside the detector taken as zero."""
    tau = g.du * 2.0 / g.N
    rows = np.asarray(r, dtype=np.float64).reshape(-1, g.A)
    h = ramp_kernel(g.A, tau)
    # full convolution of a length-A row with the length-(2A-1) kernel; the entries
    # aligned with the detector bins are those from index A-1 to 2A-2
    out = np.stack([tau * np.convolve(row, h)[g.A - 1:2 * g.A - 1] for row in rows])
    return out.reshape(-1)


def fls_loss(g: Geometry, z, y):
    """L_FLS = 1/2 (z - y)^T F (z - y) and its gradient F (z - y) (Sec. 3)."""
    d = np.asarray(z, dtype=np.float64) - np.asarray(y, dtype=np.float64)
    Fd = ramp_filter(g, d)
    return 0.5 * float(d @ Fd), Fd
