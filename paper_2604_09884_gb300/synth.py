"""Seeded synthetic inputs shared by the CUDA path, its tests and the benchmark.

This module holds no arithmetic of the method itself: it only draws
phantoms, INR initialisations, Fourier matrices, index sets and noise, and it
describes the workloads.  It imports nothing else from this package and
nothing from the oracle, so both sides can consume the same arrays.

Workloads stand in for the paper's experiments (Sec. 4: a 2-D fan-beam
FORBILD study on 512^2 and a 3-D cone-beam walnut study on 501^3), whose
phantom definition and data are not available: every phantom here is a sum
of random ellipses (2-D) or ellipsoids (3-D).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class GeomSpec:
    kind: str          # 'par2d' | 'fan2d' | 'cone3d'
    N: int
    V: int
    A: int
    B: int = 1
    du: float = 1.0
    dv: float = 1.0
    sod: float = 1000.0
    sdd: float = 1500.0
    angle0: float = 0.0
    span: float = math.pi
    fov: int = 0       # grid points sampled: 0 all, 1 the inscribed disk / cylinder

    @property
    def d(self):
        return 3 if self.kind == "cone3d" else 2

    @property
    def n(self):
        return self.N ** self.d

    @property
    def m(self):
        return self.V * (self.B if self.kind == "cone3d" else 1) * self.A

    def as_dict(self):
        return dict(kind=self.kind, N=self.N, V=self.V, A=self.A, B=self.B, du=self.du,
                    dv=self.dv, sod=self.sod, sdd=self.sdd, angle0=self.angle0, span=self.span, fov=self.fov)


@dataclass
class ArchSpec:
    kind: str          # 'ffn' | 'siren' | 'hash'
    d: int
    width: int
    n_hidden: int
    n_feat: int = 0
    sigma: float = 10.0
    omega0: float = 30.0
    hash_levels: int = 16
    hash_feats: int = 2
    hash_log2_T: int = 19
    hash_base: int = 16
    hash_growth: float = 1.5

    @property
    def d_in(self):
        if self.kind == "hash":
            return self.hash_levels * self.hash_feats
        return 2 * self.n_feat if self.kind == "ffn" else self.d

    @property
    def table_params(self):
        return self.hash_levels * (1 << self.hash_log2_T) * self.hash_feats if self.kind == "hash" else 0

    def layer_shapes(self):
        s = [(self.width, self.d_in)] + [(self.width, self.width)] * (self.n_hidden - 1)
        return s + [(1, self.width)]

    @property
    def p(self):
        return self.table_params + sum(o * i + o for o, i in self.layer_shapes())


@dataclass
class Workload:
    name: str
    geom: GeomSpec
    arch: ArchSpec
    n_shapes: int
    noise: float
    batch: int          # |I| used by the stochastic gradient (n means full grid)
    lr: float = 1e-4
    seed: int = 0
    note: str = ""


def workloads() -> dict[str, Workload]:
    """The synthetic workloads (sizes from the paper's 2-D/3-D studies, Sec. 4)."""
    w = {}
    g1 = GeomSpec("par2d", 128, 60, 183, span=math.pi)
    w["par2d_128_ffn64"] = Workload(
        "par2d_128_ffn64", g1, ArchSpec("ffn", 2, 64, 3, n_feat=64, sigma=10.0),
        n_shapes=10, noise=0.01, batch=g1.n, seed=1,
        note="2-D parallel 128^2, 60 views/[0,pi), 183 bins; FF64 sigma 10, 3x64 ReLU; full grid")
    g2 = GeomSpec("fan2d", 512, 90, 729, sod=1000.0, sdd=1500.0, span=2 * math.pi)
    w["fan2d_512_siren256"] = Workload(
        "fan2d_512_siren256", g2, ArchSpec("siren", 2, 256, 5, omega0=30.0),
        n_shapes=20, noise=0.01, batch=g2.n // 4, lr=1e-4, seed=2,
        note="2-D fan 512^2, 90 views/360deg, 729 curved bins, SOD/SDD 1000/1500; SIREN 5x256 w0=30")
    w["fan2d_512_hash64"] = Workload(
        "fan2d_512_hash64", g2, ArchSpec("hash", 2, 64, 2, hash_levels=16, hash_feats=2, hash_log2_T=19,
                                         hash_base=16, hash_growth=1.26),
        n_shapes=20, noise=0.01, batch=g2.n // 4, lr=1e-3, seed=6,
        note="2-D fan 512^2 as above; hash encoding 16 levels x 2 features, T=2^19, N_l=16..512 "
             "(growth 1.26), 2x64 ReLU; FP32")
    g3 = GeomSpec("cone3d", 256, 40, 384, 384, sod=1000.0, sdd=1500.0, span=2 * math.pi)
    w["cone3d_256_ffn256"] = Workload(
        "cone3d_256_ffn256", g3, ArchSpec("ffn", 3, 256, 4, n_feat=256, sigma=8.0),
        n_shapes=30, noise=0.0, batch=1 << 20, seed=3,
        note="3-D cone 256^3, 40 views/360deg, 384^2 flat panel; FF256 sigma 8, 4x256 ReLU; |I|=2^20")
    g5 = GeomSpec("cone3d", 501, 60, 768, 768, sod=1000.0, sdd=1500.0, span=2 * math.pi)
    w["cone3d_501_ffn512"] = Workload(
        "cone3d_501_ffn512", g5, ArchSpec("ffn", 3, 256, 5, n_feat=512, sigma=8.0),
        n_shapes=40, noise=0.01, batch=1 << 22, seed=5,
        note="3-D cone 501^3, 60 views/360deg, 768^2 flat panel; FF512, 5x256 ReLU; |I|=2^22")
    return w


def batched_problems(seed: int = 4, count: int = 16) -> list[Workload]:
    """Sixteen uneven 2-D problems (parallel/fan mixed), SIREN 3x128 each, |I| = n/4."""
    rng = np.random.default_rng(seed)
    sizes = [128, 256, 384, 512, 768, 1024]
    out = []
    for k in range(count):
        N = int(rng.choice(sizes))
        V = int(rng.integers(30, 181))
        A = int(math.ceil(1.42 * N))
        kind = "par2d" if k % 2 == 0 else "fan2d"
        span = math.pi if kind == "par2d" else 2 * math.pi
        g = GeomSpec(kind, N, V, A, sod=4.0 * N, sdd=6.0 * N, span=span)
        out.append(Workload(f"batch{k}_{kind}_{N}", g, ArchSpec("siren", 2, 128, 3, omega0=30.0),
                            n_shapes=10, noise=0.01, batch=g.n // 4, seed=1000 + k))
    return out


# ----------------------------------------------------------------------------
# draws
# ----------------------------------------------------------------------------
def _coords_1d(N):
    return -1.0 + (np.arange(N, dtype=np.float64) + 0.5) * (2.0 / N)


def phantom(d: int, N: int, count: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Sum of `count` random ellipses (d=2) or ellipsoids (d=3), rasterised by a
    pixel-centre inside test.  Centres U[-0.7, 0.7]^d, semi-axes U[0.05, 0.5],
    intensities U[0, 1]; 2-D angle U[0, pi); 3-D orientation a uniform rotation."""
    rng = np.random.default_rng(seed)
    c = _coords_1d(N)
    img = np.zeros((N,) * d, dtype=dtype)
    for _ in range(count):
        ctr = rng.uniform(-0.7, 0.7, size=d)
        ax = rng.uniform(0.05, 0.5, size=d)
        mu = rng.uniform(0.0, 1.0)
        if d == 2:
            ang = rng.uniform(0.0, math.pi)
            Rm = np.array([[math.cos(ang), -math.sin(ang)], [math.sin(ang), math.cos(ang)]])
        else:
            q = rng.normal(size=4)
            q /= np.linalg.norm(q)
            a, b, cq, dq = q
            Rm = np.array([[a*a+b*b-cq*cq-dq*dq, 2*(b*cq-a*dq), 2*(b*dq+a*cq)],
                           [2*(b*cq+a*dq), a*a-b*b+cq*cq-dq*dq, 2*(cq*dq-a*b)],
                           [2*(b*dq-a*cq), 2*(cq*dq+a*b), a*a-b*b-cq*cq+dq*dq]])
        r = float(ax.max())
        lo = [max(0, int(np.searchsorted(c, ctr[k] - r)) - 1) for k in range(d)]
        hi = [min(N, int(np.searchsorted(c, ctr[k] + r)) + 1) for k in range(d)]
        if d == 2:
            X, Y = np.meshgrid(c[lo[0]:hi[0]] - ctr[0], c[lo[1]:hi[1]] - ctr[1], indexing="xy")
            loc = np.stack([X, Y], -1) @ Rm          # coordinates in the ellipse frame
            inside = ((loc / ax) ** 2).sum(-1) <= 1.0
            img[lo[1]:hi[1], lo[0]:hi[0]] += mu * inside
        else:
            for iz in range(lo[2], hi[2]):
                X, Y = np.meshgrid(c[lo[0]:hi[0]] - ctr[0], c[lo[1]:hi[1]] - ctr[1],
                                   indexing="xy")
                Z = np.full_like(X, c[iz] - ctr[2])
                loc = np.stack([X, Y, Z], -1) @ Rm
                inside = ((loc / ax) ** 2).sum(-1) <= 1.0
                img[iz, lo[1]:hi[1], lo[0]:hi[0]] += mu * inside
    return img


def fourier_matrix(F: int, d: int, sigma: float, seed: int) -> np.ndarray:
    """Gaussian Fourier-feature matrix B ~ N(0, sigma^2), shape F x d (fixed, not trained)."""
    return np.random.default_rng(seed).normal(0.0, sigma, size=(F, d))


def init_theta(arch: ArchSpec, seed: int, table_scale: float = 1e-4) -> np.ndarray:
    """Flat theta in the layer order [W_1, b_1, ..., W_out, b_out] (W row-major [out][in]),
    preceded by the hash tables [level][entry][feature] for the hash-encoded INR.

    FFN and hash: Xavier-uniform weights, zero biases; hash tables U(+-table_scale).
    SIREN: first layer U(-1/d, 1/d), later layers U(+-sqrt(6/fan_in)/omega0); biases
    U(+-1/sqrt(fan_in))."""
    rng = np.random.default_rng(seed)
    parts = []
    if arch.kind == "hash":
        parts.append(rng.uniform(-table_scale, table_scale, size=arch.table_params))
    shapes = arch.layer_shapes()
    for li, (o, i) in enumerate(shapes):
        if arch.kind in ("ffn", "hash"):
            a = math.sqrt(6.0 / (i + o))
            W = rng.uniform(-a, a, size=(o, i))
            b = np.zeros(o)
        else:
            a = 1.0 / i if li == 0 else math.sqrt(6.0 / i) / arch.omega0
            W = rng.uniform(-a, a, size=(o, i))
            bb = 1.0 / math.sqrt(i)
            b = rng.uniform(-bb, bb, size=o)
        parts += [W.reshape(-1), b]
    return np.concatenate(parts)


def index_set(n: int, k: int, seed: int) -> np.ndarray:
    """Uniform random subset of [0, n) of size k without replacement, sorted, int32."""
    if k >= n:
        return np.arange(n, dtype=np.int32)
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int32)


def noisy(y_clean: np.ndarray, level: float, seed: int) -> np.ndarray:
    """y = y_clean + N(0, (level * max y_clean)^2)."""
    if level <= 0:
        return np.array(y_clean, copy=True)
    rng = np.random.default_rng(seed)
    sd = level * float(np.max(y_clean))
    return y_clean + rng.normal(0.0, sd, size=y_clean.shape).astype(y_clean.dtype)


def uniform(shape, seed: int, lo=-1.0, hi=1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)
