"""Pins of the oracle's field of view (Sec. 3 samples the INR on the grid points inside a FOV
mask; the reading is the inscribed disk, a cylinder along z in 3-D).

The integer test is checked against the same condition x^2 + y^2 <= 1 evaluated on FP64 pixel
centres away from the boundary, against the disk's area and symmetries, and the masked
pipeline's gradient against central differences of the loss it defines."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2604_09884_gb300 import synth


@pytest.mark.parametrize("N", [5, 8, 33, 64, 101])
def test_integer_test_is_the_disk_at_pixel_centres(N):
    X = O.grid_coords(2, N)
    r2 = (X ** 2).sum(axis=1)
    m = O.fov_mask(2, N)
    clear = np.abs(r2 - 1.0) > 1e-12
    assert np.array_equal(m[clear], (r2 <= 1.0)[clear])
    # centres exactly on the circle count as inside
    assert np.all(m[~clear])


@pytest.mark.parametrize("N", [64, 128, 257])
def test_pixel_count_and_symmetry(N):
    m = O.fov_mask(2, N).reshape(N, N)
    # the area pi N^2 / 4 up to pixels the circle cuts (at most 4 N of them)
    assert abs(m.sum() - math.pi * N * N / 4) <= 4 * N
    assert np.array_equal(m, m.T) and np.array_equal(m, m[::-1]) and np.array_equal(m, m[:, ::-1])


def test_three_d_mask_is_a_cylinder():
    N = 12
    m3 = O.fov_mask(3, N).reshape(N, N, N)
    m2 = O.fov_mask(2, N).reshape(N, N)
    for z in range(N):
        assert np.array_equal(m3[z], m2)


def _problem(kind):
    g = O.Geometry("par2d", 8, 5, 11, fov=1)
    if kind == "ffn":
        arch = O.Arch("ffn", 2, 6, 2, 3, np.random.default_rng(1).normal(0, 1.5, (3, 2)))
    else:
        arch = O.Arch("siren", 2, 6, 2, omega0=2.0)
    theta = np.random.default_rng(2).uniform(-1, 1, arch.p)
    y = O.project(g, synth.phantom(2, 8, 3, 3))
    return g, arch, theta, y


@pytest.mark.parametrize("kind", ["ffn", "siren"])
def test_masked_gradient_is_the_chain_rule_of_the_masked_loss(kind):
    g, arch, theta, y = _problem(kind)
    L0, grad, _ = O.full_gradient(arch, theta, g, y)
    x = O.evaluate_image(arch, theta, g)
    assert np.all(x[~O.fov_mask(2, g.N)] == 0.0) and np.any(x != 0.0)

    def loss(t):
        return O.ls_loss(O.project(g, O.evaluate_image(arch, t, g)), y)[0]

    assert abs(loss(theta) - L0) < 1e-14 * max(1, L0)
    h = 1e-6
    for j in np.random.default_rng(4).choice(theta.size, 25, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert abs(fd - grad[j]) <= 1e-7 * max(1.0, abs(grad[j])), (j, fd, grad[j])


def test_estimator_over_the_fov_is_the_full_gradient_and_ignores_outside_points():
    g, arch, theta, y = _problem("siren")
    _, grad, v = O.full_gradient(arch, theta, g, y)
    inside = O.fov_indices(g)
    assert 0 < inside.size < g.n
    np.testing.assert_allclose(O.estimator(arch, theta, g, v, inside), grad, rtol=1e-13, atol=1e-15)
    outside = np.setdiff1d(np.arange(g.n), inside)
    both = np.concatenate([inside, outside])
    np.testing.assert_allclose(O.estimator(arch, theta, g, v, both, scale=1.0), grad, rtol=1e-13, atol=1e-15)
