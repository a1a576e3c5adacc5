"""Pins of the oracle's Joseph projector P and its transpose (Sec. 3: z = P x, v = P^T r).

Nothing here compares the oracle with itself: every check is against a closed
form (chords through disks and balls, line integrals of Gaussians), an exact
special case (axis-aligned rays through a constant image), a brute-force dense
matrix, or a symmetry of the geometry.
"""
import math

import numpy as np
import pytest

import oracle as O


def _perp_dist(s, e, c):
    w = np.asarray(c, float) - s[: len(c)] if len(c) == 3 else np.r_[np.asarray(c, float), 0.0] - s
    w = w - (w @ e) * e
    return float(np.linalg.norm(w))


def _disk(N, ctr, R, mu=1.0, d=2):
    c = -1.0 + (np.arange(N) + 0.5) * 2.0 / N
    if d == 2:
        X, Y = np.meshgrid(c, c, indexing="xy")
        return mu * (((X - ctr[0]) ** 2 + (Y - ctr[1]) ** 2) <= R * R)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    return mu * (((X - ctr[0]) ** 2 + (Y - ctr[1]) ** 2 + (Z - ctr[2]) ** 2) <= R * R)


def _gauss(N, ctr, s, d=2):
    c = -1.0 + (np.arange(N) + 0.5) * 2.0 / N
    if d == 2:
        X, Y = np.meshgrid(c, c, indexing="xy")
        r2 = (X - ctr[0]) ** 2 + (Y - ctr[1]) ** 2
    else:
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        r2 = (X - ctr[0]) ** 2 + (Y - ctr[1]) ** 2 + (Z - ctr[2]) ** 2
    return np.exp(-r2 / (2 * s * s))


GEOMS_SMALL = [
    O.Geometry("par2d", 16, 7, 25),
    O.Geometry("fan2d", 16, 9, 31, sod=40.0, sdd=60.0, span=2 * math.pi),
    O.Geometry("cone3d", 8, 5, 15, 13, sod=30.0, sdd=45.0, span=2 * math.pi),
]


def test_parallel_constant_image_axis_aligned_exact():
    # view 0 (angle 0): rays run along +y and sit halfway between pixel columns,
    # so every interior slice contributes exactly c and the ray sum is N*D*c = 2c.
    N, A, c = 128, 183, 0.75
    g = O.Geometry("par2d", N, 60, A)
    z = O.project(g, np.full((N, N), c)).reshape(60, A)
    b = np.arange(A)
    u = b - (A - 1) / 2 + N / 2 - 0.5          # transverse fractional index of bin b
    want = np.where((u >= 0) & (u <= N - 1), 2 * c, 0.0)
    want[np.isclose(u, -0.5) | np.isclose(u, N - 0.5)] = c   # half-covered edge bins
    np.testing.assert_allclose(z[0], want, rtol=0, atol=1e-13)
    # view V/2 is angle pi/2: x-driving, same values with the bin axis reversed in sign
    np.testing.assert_allclose(z[30], want[::-1], rtol=0, atol=1e-12)


@pytest.mark.parametrize("ctr", [(0.0, 0.0), (0.31, -0.22)])
def test_parallel_disk_chords(ctr):
    N, R = 512, 0.4
    g = O.Geometry("par2d", N, 12, 729)
    z = O.project(g, _disk(N, ctr, R)).reshape(12, 729)
    errs = []
    for k in range(12):
        for b in range(0, 729, 7):
            s, e = O.ray(g, k, 0, b)
            dd = _perp_dist(s, e, ctr)
            if dd <= 0.8 * R:
                want = 2 * math.sqrt(R * R - dd * dd)
                errs.append(abs(z[k, b] - want) / want)
    assert len(errs) > 100
    assert max(errs) < 0.01, max(errs)


def test_fan_disk_chords_offcentre():
    N, R, ctr = 512, 0.35, (-0.25, 0.4)
    g = O.Geometry("fan2d", N, 10, 729, sod=1000.0, sdd=1500.0, span=2 * math.pi)
    z = O.project(g, _disk(N, ctr, R)).reshape(10, 729)
    errs = []
    for k in range(10):
        for b in range(0, 729, 5):
            s, e = O.ray(g, k, 0, b)
            dd = _perp_dist(s, e, ctr)
            if dd <= 0.8 * R:
                want = 2 * math.sqrt(R * R - dd * dd)
                errs.append(abs(z[k, b] - want) / want)
    assert len(errs) > 100
    assert max(errs) < 0.01, max(errs)


def test_cone_ball_chords_offcentre():
    N, R, ctr = 96, 0.45, (0.2, -0.15, 0.1)
    g = O.Geometry("cone3d", N, 4, 64, 64, du=2.0, dv=2.0, sod=300.0, sdd=450.0,
                   span=2 * math.pi)
    z = O.project(g, _disk(N, ctr, R, d=3)).reshape(4, 64, 64)
    errs = []
    for k in range(4):
        for row in range(0, 64, 2):
            for col in range(0, 64, 2):
                s, e = O.ray(g, k, row, col)
                dd = _perp_dist(s, e, ctr)
                if dd <= 0.7 * R:
                    want = 2 * math.sqrt(R * R - dd * dd)
                    errs.append(abs(z[k, row, col] - want) / want)
    assert len(errs) > 100
    assert max(errs) < 0.03, max(errs)


def _gauss_err(g, ctr, sd, rays):
    img = _gauss(g.N, ctr, sd, d=g.d)
    z = O.project_at(g, img, rays)
    errs = []
    for q, r in enumerate(rays):
        A = g.A
        rows = g.B if g.kind == "cone3d" else 1
        col, row, k = r % A, (r // A) % rows, r // (A * rows)
        s, e = O.ray(g, k, row, col)
        dd = _perp_dist(s, e, ctr)
        want = math.sqrt(2 * math.pi) * sd * math.exp(-dd * dd / (2 * sd * sd))
        errs.append(abs(z[q] - want))
    return max(errs)


@pytest.mark.parametrize("kind", ["par2d", "fan2d"])
def test_gaussian_line_integrals_converge_second_order(kind):
    # Joseph interpolation of a smooth function is second-order accurate; halving D
    # must cut the error by about four.
    ctr, sd = (0.12, -0.07), 0.18
    errs = []
    for N in (64, 128, 256):
        A = int(1.5 * N) | 1
        g = O.Geometry(kind, N, 7, A, du=1.0, sod=4.0 * N, sdd=6.0 * N,
                       span=math.pi if kind == "par2d" else 2 * math.pi)
        # the same physical rays at every N: fixed fractions of the detector
        rays = [k * A + int(f * (A - 1)) for k in range(7) for f in (0.3, 0.42, 0.5, 0.61)]
        errs.append(_gauss_err(g, ctr, sd, rays))
    assert errs[0] < 2e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


def test_cone_gaussian_line_integral():
    ctr, sd = (0.1, 0.05, -0.08), 0.2
    errs = []
    for N in (32, 64):
        g = O.Geometry("cone3d", N, 3, 2 * N + 1, 2 * N + 1, du=1.0, dv=1.0, sod=6.0 * N,
                       sdd=9.0 * N, span=2 * math.pi)
        A = g.A
        rays = [(k * A + int(fr * (A - 1))) * A + int(fc * (A - 1))
                for k in range(3) for fr in (0.35, 0.5, 0.6) for fc in (0.4, 0.5, 0.57)]
        errs.append(_gauss_err(g, ctr, sd, rays))
    assert errs[0] < 2e-2 and errs[1] < 3e-3
    assert errs[0] / errs[1] > 3.0, errs


@pytest.mark.parametrize("g", GEOMS_SMALL, ids=lambda g: g.kind)
def test_dense_matrix_transpose_and_entries(g):
    # Build P column by column from unit images and P^T column by column from
    # unit sinograms; P^T must be P's transpose entry by entry, and each entry
    # must equal the directly written-out interpolation weight.
    n, m = g.n, g.m
    P = np.zeros((m, n))
    for i in range(n):
        x = np.zeros(n)
        x[i] = 1.0
        P[:, i] = O.project(g, x)
    PT = np.zeros((n, m))
    for r in range(m):
        y = np.zeros(m)
        y[r] = 1.0
        PT[:, r] = O.backproject(g, y)
    np.testing.assert_allclose(PT, P.T, rtol=0, atol=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(300):
        r, i = int(rng.integers(m)), int(rng.integers(n))
        assert abs(O.matrix_entry(g, r, i) - P[r, i]) <= 1e-15
    nz = np.argwhere(P != 0)
    for r, i in nz[rng.choice(len(nz), 200)]:
        assert abs(O.matrix_entry(g, r, i) - P[r, i]) <= 1e-15
    assert (P >= 0).all()


@pytest.mark.parametrize("g", [
    O.Geometry("par2d", 64, 31, 91),
    O.Geometry("fan2d", 64, 33, 95, sod=150.0, sdd=220.0, span=2 * math.pi),
    O.Geometry("cone3d", 24, 7, 37, 33, sod=80.0, sdd=120.0, span=2 * math.pi),
], ids=lambda g: g.kind)
def test_adjoint_identity(g):
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, g.n)
    r = rng.uniform(0, 1, g.m)
    lhs = O.project(g, x) @ r
    rhs = x @ O.backproject(g, r)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    pix = rng.choice(g.n, 12, replace=False)
    np.testing.assert_allclose(O.backproject_at(g, r, pix), O.backproject(g, r)[pix],
                               rtol=1e-13, atol=0)


def test_parallel_rotation_symmetry():
    # Rotating the image by 90 degrees (counter-clockwise) shifts the parallel views by
    # V/2 (pi/2): P(rot x)(phi + pi/2, t) = P(x)(phi, t).
    N, V, A = 48, 16, 71
    g = O.Geometry("par2d", N, V, A, span=math.pi)
    x = np.random.default_rng(2).uniform(0, 1, (N, N))
    z = O.project(g, x).reshape(V, A)
    # rot: new[y, x] = old at the point rotated back by -90 deg: (x, y) -> (y, -x)
    xr = np.empty_like(x)
    for iy in range(N):
        for ix in range(N):
            # rotated image value at pixel (ix, iy) = original at (iy, N-1-ix)
            xr[iy, ix] = x[N - 1 - ix, iy]
    zr = O.project(g, xr).reshape(V, A)
    np.testing.assert_allclose(zr[V // 2:], z[: V // 2], rtol=1e-12, atol=1e-12)


def test_ray_definitions():
    # Each ray must be the one the geometry defines, checked from the definition
    # (not from the oracle's own formulas): parallel rays pass through t_b (cos, sin)
    # orthogonally; fan rays leave the source at fan angle gamma_b from the central
    # ray; cone rays join the source to the bin centre on the flat panel.
    N = 64
    D = 2.0 / N
    g = O.Geometry("par2d", N, 8, 21, du=1.5)
    for k in range(8):
        ang = g.span * k / g.V
        for b in (0, 7, 20):
            s, e = O.ray(g, k, 0, b)
            t = (b - 10) * 1.5 * D
            p = t * np.array([math.cos(ang), math.sin(ang), 0.0])
            assert np.linalg.norm(np.cross(s - p, e)) < 1e-14          # p on the ray
            assert abs(e @ np.array([math.cos(ang), math.sin(ang), 0])) < 1e-15
            assert abs(np.linalg.norm(e) - 1) < 1e-15
    g = O.Geometry("fan2d", N, 8, 21, du=1.0, sod=100.0, sdd=150.0, span=2 * math.pi)
    for k in range(8):
        ang = g.span * k / g.V
        S = 100.0 * D * np.array([math.cos(ang), math.sin(ang), 0.0])
        for b in (0, 3, 10, 20):
            s, e = O.ray(g, k, 0, b)
            gam = (b - 10) / 100.0
            assert np.linalg.norm(s - S) < 1e-14
            c = -S / np.linalg.norm(S)
            assert abs(e @ c - math.cos(gam)) < 1e-14
            assert abs(np.cross(c, e)[2] - math.sin(gam)) < 1e-14   # counter-clockwise
    g = O.Geometry("cone3d", N, 6, 11, 7, du=1.0, dv=2.0, sod=100.0, sdd=160.0,
                   span=2 * math.pi)
    for k in range(6):
        ang = g.span * k / g.V
        cb, sb = math.cos(ang), math.sin(ang)
        S = 100.0 * D * np.array([cb, sb, 0.0])
        ctr = -60.0 * D * np.array([cb, sb, 0.0])
        for row, col in ((0, 0), (3, 5), (6, 10)):
            s, e = O.ray(g, k, row, col)
            bin_ = ctr + (col - 5) * 1.6 * D * np.array([-sb, cb, 0]) \
                + (row - 3) * 3.2 * D * np.array([0, 0, 1.0])
            assert np.linalg.norm(s - S) < 1e-14
            w = (bin_ - S) / np.linalg.norm(bin_ - S)
            assert np.linalg.norm(e - w) < 1e-14


def test_ramp_filter_matrix_and_spectrum():
    # F as an explicit Toeplitz matrix from the textbook taps, and the ramp's
    # properties: zero response to a constant (away from the detector edges),
    # symmetric, positive semi-definite (its spectrum is |omega| >= 0).
    g = O.Geometry("par2d", 32, 2, 41, du=1.0)
    tau = 2.0 / 32
    A = g.A

    def h(k):
        if k == 0:
            return 1 / (4 * tau * tau)
        return -1 / (math.pi ** 2 * k * k * tau * tau) if k % 2 else 0.0

    F = np.array([[tau * h(b - c) for c in range(A)] for b in range(A)])
    r = np.random.default_rng(3).normal(size=g.m)
    np.testing.assert_allclose(O.ramp_filter(g, r), (r.reshape(2, A) @ F.T).reshape(-1),
                               rtol=0, atol=1e-12)
    assert np.allclose(F, F.T)
    assert np.linalg.eigvalsh(F).min() > -1e-9
    # long constant row: the centre of the output tends to zero like 1/A
    g2 = O.Geometry("par2d", 32, 1, 4001, du=1.0)
    out = O.ramp_filter(g2, np.ones(g2.m))
    assert abs(out[2000]) < 1e-3 * abs(out[0])
    L, Fd = O.fls_loss(g, r + 1.0, np.ones(g.m))
    want = 0.5 * sum(rr @ F @ rr for rr in r.reshape(2, A))
    assert abs(L - want) < 1e-9 * abs(want)


@pytest.mark.parametrize("kind", ["par2d", "fan2d", "cone3d"])
def test_view_subsets_partition_the_rays(kind):
    """Ordered subsets of views (Sec. 3): interleaved subset s of S, written as a scan of V/S
    views starting S-times-coarser at angle0 + span s / V, holds exactly the full scan's rays
    of views s, s + S, ...; hence its residual backprojections sum to the full one."""
    S, V = 3, 9
    kw = dict(sod=40.0, sdd=60.0, span=2 * math.pi) if kind != "par2d" else dict(span=math.pi)
    full = O.Geometry(kind, 12 if kind != "cone3d" else 8, V, 19, 11 if kind == "cone3d" else 1,
                      angle0=0.2, **kw)
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, full.n)
    y = rng.uniform(0, 1, full.m)
    rows = full.m // V
    total = np.zeros(full.n)
    for s in range(S):
        sub = O.Geometry(kind, full.N, V // S, full.A, full.B, angle0=0.2 + full.span * s / V, **kw)
        for kp in range(V // S):
            for b in range(0, full.A, 6):
                p_sub, e_sub = O.ray(sub, kp, 0, b)
                p_full, e_full = O.ray(full, s + S * kp, 0, b)
                assert np.allclose(p_sub, p_full, atol=1e-12) and np.allclose(e_sub, e_full, atol=1e-12)
        ys = y.reshape(V, rows)[s::S].reshape(-1)
        total += O.backproject(sub, O.project(sub, x) - ys)
    ref = O.backproject(full, O.project(full, x) - y)
    assert np.allclose(total, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("kind", ["par2d", "cone3d"])
def test_fls_loss_gradient_matches_central_differences(kind):
    """The gradient fls_loss returns, F (z - y), against central differences of the loss value
    itself (Sec. 3's filtered least squares; F from the band-limited ramp)."""
    g = O.Geometry("par2d", 16, 3, 23) if kind == "par2d" else O.Geometry("cone3d", 8, 2, 9, 5, sod=40.0,
                                                                           sdd=60.0)
    rng = np.random.default_rng(11)
    z, y = rng.normal(size=g.m), rng.normal(size=g.m)
    _, grad = O.fls_loss(g, z, y)
    h = 1e-6
    for j in rng.choice(g.m, 12, replace=False):
        zp, zm = z.copy(), z.copy()
        zp[j] += h
        zm[j] -= h
        fd = (O.fls_loss(g, zp, y)[0] - O.fls_loss(g, zm, y)[0]) / (2 * h)
        assert abs(fd - grad[j]) <= 1e-6 * max(1.0, abs(grad[j])), (j, fd, grad[j])
