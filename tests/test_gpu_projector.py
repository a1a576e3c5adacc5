"""GPU parity of the projector P, its adjoint P^T and the ramp filter against the
FP64 oracle (bar: FP32 P / P^T within 1e-5 relative L2)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_09884_gb300 import inrct, synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def og(g: synth.GeomSpec) -> O.Geometry:
    return O.Geometry(g.kind, g.N, g.V, g.A, g.B, g.du, g.dv, g.sod, g.sdd, g.angle0, g.span)


def cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


CASES = [
    synth.GeomSpec("par2d", 128, 60, 183),                                   # 128^2 workload
    synth.GeomSpec("par2d", 37, 7, 53, du=0.8, angle0=0.3),                  # ragged, odd sizes
    synth.GeomSpec("par2d", 64, 8, 91, span=math.pi),                        # 45-degree views
    synth.GeomSpec("fan2d", 512, 90, 729, sod=1000.0, sdd=1500.0, span=2 * math.pi),  # 512^2 fan
    synth.GeomSpec("fan2d", 45, 13, 67, du=1.3, sod=90.0, sdd=140.0, span=2 * math.pi),
    synth.GeomSpec("cone3d", 48, 12, 80, 72, sod=150.0, sdd=230.0, span=2 * math.pi),
    synth.GeomSpec("cone3d", 33, 5, 47, 39, du=1.2, dv=0.9, sod=70.0, sdd=100.0, span=2 * math.pi),
    synth.GeomSpec("par2d", 2, 1, 3),                                        # degenerate tiny
    # odd view count with rows a multiple of 4: the cone adjoint's 16-byte strip copies
    synth.GeomSpec("cone3d", 40, 7, 52, 44, du=1.1, sod=120.0, sdd=180.0, span=2 * math.pi),
]


@pytest.mark.parametrize("g", CASES, ids=lambda g: f"{g.kind}_{g.N}_{g.V}x{g.A}")
def test_project_and_backproject_match_oracle(g):
    x = synth.phantom(g.d, g.N, 8, seed=g.N + g.V).astype(np.float32)
    z = inrct.project(g, cuda(x.reshape(-1))).cpu().numpy()
    assert rel(z, O.project(og(g), x)) <= TOL
    r = synth.uniform(g.m, seed=g.A, lo=-1.0, hi=1.0).astype(np.float32)
    v = inrct.backproject(g, cuda(r)).cpu().numpy()
    assert rel(v, O.backproject(og(g), r)) <= TOL


@pytest.mark.parametrize("g", CASES[:6], ids=lambda g: f"{g.kind}_{g.N}")
def test_adjoint_identity_on_gpu(g):
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, g.n).astype(np.float32)
    r = rng.uniform(0, 1, g.m).astype(np.float32)
    Px = inrct.project(g, cuda(x)).double().cpu().numpy()
    PTr = inrct.backproject(g, cuda(r)).double().cpu().numpy()
    lhs, rhs = Px @ r.astype(np.float64), x.astype(np.float64) @ PTr
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def test_loss_epilogue_matches_oracle():
    g = CASES[3]
    x = synth.phantom(2, g.N, 20, seed=5).astype(np.float32)
    y = (O.project(og(g), synth.phantom(2, g.N, 20, seed=6))).astype(np.float32)
    z, r, L = inrct.project(g, cuda(x), cuda(y))
    L0, r0 = O.ls_loss(O.project(og(g), x), y)
    assert rel(r.cpu().numpy(), r0) <= TOL
    assert abs(L.item() - L0) <= 2 * TOL * L0


@pytest.mark.parametrize("name,shapes,n_vox", [("cone3d_256_ffn256", 30, 24), ("cone3d_501_ffn512", 12, 8)],
                         ids=["cone256", "cone501"])
def test_cone_full_size_sampled_parity(name, shapes, n_vox):
    # the cone workloads at full size (their volumes exceed L2, so P runs in z-slab order):
    # sampled rays and voxels against the oracle, and the adjoint identity
    g = synth.workloads()[name].geom
    x = synth.phantom(3, g.N, shapes, seed=3).astype(np.float32)
    z = inrct.project(g, cuda(x.reshape(-1))).cpu().numpy()
    rng = np.random.default_rng(11)
    rays = rng.choice(g.m, 3000, replace=False)
    assert rel(z[rays], O.project_at(og(g), x, rays)) <= TOL
    r = rng.uniform(-1, 1, g.m).astype(np.float32)
    v = inrct.backproject(g, cuda(r)).cpu().numpy()
    vox = rng.choice(g.n, n_vox, replace=False)
    assert rel(v[vox], O.backproject_at(og(g), r, vox)) <= TOL
    lhs = z.astype(np.float64) @ r.astype(np.float64)
    rhs = x.reshape(-1).astype(np.float64) @ v.astype(np.float64)
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


@pytest.mark.parametrize("g", [CASES[3], CASES[5]], ids=["fan2d", "cone3d"])
def test_ramp_filter_matches_oracle(g):
    r = synth.uniform(g.m, seed=4).astype(np.float32)
    out, loss = inrct.ramp_filter(g, cuda(r))
    want = O.ramp_filter(og(g), r)
    assert rel(out.cpu().numpy(), want) <= TOL
    L0 = 0.5 * float(r.astype(np.float64) @ want)
    assert abs(loss.item() - L0) <= 1e-4 * abs(L0)


def _project_with(L, g, x, ws):
    import ctypes
    gd, grd = inrct.geom_desc(g), inrct.grid_desc(g.d, g.N)
    z = torch.empty(g.m, dtype=torch.float32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.project(ctypes.byref(gd), ctypes.byref(grd), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                   None, None, None, ctypes.c_void_p(ws.data_ptr()), ws.numel(), s)
    assert rc == 0, L.inrct_last_error().decode()
    return z


def test_ray_tables_persist_in_a_workspace_only_while_valid():
    """The ray tables stay in the workspace between calls and are reused only when the seals
    at both ends of their region carry this geometry's fingerprint: reusing one workspace
    for geometry A, then B, then A, and clobbering it between calls, gives exactly the
    projections of fresh workspaces."""
    L = inrct.lib()
    ga = synth.GeomSpec("fan2d", 96, 30, 137, sod=300.0, sdd=450.0, span=2 * math.pi)
    gb = synth.GeomSpec("fan2d", 96, 31, 137, sod=300.0, sdd=450.0, span=2 * math.pi)
    import ctypes
    nb = max(L.inrct_project_ws_bytes(ctypes.byref(inrct.geom_desc(g)), ctypes.byref(inrct.grid_desc(2, 96)))
             for g in (ga, gb))
    x = cuda(synth.phantom(2, 96, 5, seed=3).reshape(-1))
    ref = {id(g): _project_with(L, g, x, torch.zeros(nb, dtype=torch.uint8, device="cuda")) for g in (ga, gb)}
    ws = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    for g in (ga, ga, gb, ga, gb, gb):
        assert torch.equal(_project_with(L, g, x, ws), ref[id(g)])
    ws.fill_(7)  # clobbered workspace: the seals no longer match, the tables are rebuilt
    assert torch.equal(_project_with(L, ga, x, ws), ref[id(ga)])
    ws[: nb // 2].fill_(0)  # only the first half (the leading seal) overwritten
    assert torch.equal(_project_with(L, ga, x, ws), ref[id(ga)])
