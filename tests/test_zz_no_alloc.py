"""project_noalloc: the allocation-free projection entry point.

It serves callers that may not allocate device memory (their memory belongs to
another allocator, or is reserved once at start-up), so its scratch is a fixed
array inside the library.  Checked through the C ABI against project(), the
entry point with a caller workspace, on two calls in a row with different
inputs, so that contents left in the shared array by the first call cannot
leak into the second.  This file is collected last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from paper_2604_09884_gb300 import inrct, synth

pytestmark = pytest.mark.gpu
TOL = 1e-5  # the projector's parity tolerance


def rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _call_noalloc(g, image, y):
    """project_noalloc through the raw C ABI (no workspace argument exists)."""
    L = inrct.lib()
    gd, grd = inrct.geom_desc(g), inrct.grid_desc(g.d, g.N)
    z = torch.empty(g.m, dtype=torch.float32, device=image.device)
    r = torch.empty(g.m, dtype=torch.float32, device=image.device)
    loss = torch.empty(1, dtype=torch.float64, device=image.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.project_noalloc(ctypes.byref(gd), ctypes.byref(grd), ctypes.c_void_p(image.data_ptr()),
                           ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                           ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(loss.data_ptr()), stream)
    assert rc == 0, L.inrct_last_error().decode()
    return z, r, loss


@pytest.mark.parametrize("g", [
    synth.GeomSpec("fan2d", 512, 90, 729, sod=1000.0, sdd=1500.0, span=2 * math.pi),
    synth.GeomSpec("par2d", 128, 60, 183),
], ids=["fan512", "par128"])
def test_project_noalloc_matches_project_on_two_calls(g):
    dev = torch.device("cuda")
    for call in range(2):
        x = torch.tensor(synth.phantom(2, g.N, 6 + call, seed=40 + call).reshape(-1),
                         dtype=torch.float32, device=dev)
        y = torch.tensor(synth.uniform(g.m, seed=50 + call, lo=0.0, hi=2.0), dtype=torch.float32,
                         device=dev)
        z_ref, r_ref, l_ref = inrct.project(g, x, y)
        z, r, loss = _call_noalloc(g, x, y)
        torch.cuda.synchronize()
        assert rel(z, z_ref) <= TOL
        assert rel(r, r_ref) <= TOL
        assert abs(loss.item() - l_ref.item()) <= TOL * abs(l_ref.item())


def test_project_noalloc_after_a_different_geometry():
    """The second call uses another geometry than the first: ray tables left in the shared array
    by the first call must not be taken for the second one's (a missing rebuild would change z)."""
    dev = torch.device("cuda")
    geoms = [synth.GeomSpec("fan2d", 512, 90, 729, sod=1000.0, sdd=1500.0, span=2 * math.pi),
             synth.GeomSpec("par2d", 128, 60, 183),
             synth.GeomSpec("fan2d", 512, 90, 729, sod=1000.0, sdd=1500.0, span=2 * math.pi)]
    for call, g in enumerate(geoms):
        x = torch.tensor(synth.phantom(2, g.N, 5, seed=60 + call).reshape(-1), dtype=torch.float32,
                         device=dev)
        y = torch.tensor(synth.uniform(g.m, seed=70 + call, lo=0.0, hi=2.0), dtype=torch.float32,
                         device=dev)
        z_ref, r_ref, l_ref = inrct.project(g, x, y)
        z, r, loss = _call_noalloc(g, x, y)
        torch.cuda.synchronize()
        assert rel(z, z_ref) <= TOL, call
        assert rel(r, r_ref) <= TOL, call
        assert abs(loss.item() - l_ref.item()) <= TOL * abs(l_ref.item()), call


def test_project_noalloc_rejects_geometry_beyond_its_buffer():
    g = synth.GeomSpec("cone3d", 256, 40, 384, 384, sod=1000.0, sdd=1500.0, span=2 * math.pi)
    L = inrct.lib()
    gd, grd = inrct.geom_desc(g), inrct.grid_desc(3, g.N)
    assert L.inrct_project_ws_bytes(ctypes.byref(gd), ctypes.byref(grd)) > 16 * 1024 * 1024
    fake = ctypes.c_void_p(256)
    rc = L.project_noalloc(ctypes.byref(gd), ctypes.byref(grd), fake, fake, None, None, None, None)
    assert rc == 3 and b"static buffer" in L.inrct_last_error()
