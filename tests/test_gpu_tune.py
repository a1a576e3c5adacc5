"""The projector autotuner (inrct_tune): every plan computes the same operator, so after
tuning P and P^T still match the oracle at the FP32 bar (1e-5); workspaces sized before
tuning stay valid; creating a batch tunes every problem's geometry."""
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


def og(g):
    return O.Geometry(g.kind, g.N, g.V, g.A, g.B, g.du, g.dv, g.sod, g.sdd, g.angle0, g.span)


GEOMS = [
    synth.GeomSpec("par2d", 96, 60, 137, span=math.pi),
    synth.GeomSpec("fan2d", 200, 45, 285, sod=800.0, sdd=1200.0, span=2 * math.pi),
    synth.GeomSpec("cone3d", 40, 12, 64, 48, sod=160.0, sdd=240.0, span=2 * math.pi),
]


@pytest.mark.parametrize("g", GEOMS, ids=lambda g: f"{g.kind}_{g.N}")
def test_tuned_plans_match_the_oracle(g):
    inrct.tune_reset()
    x = synth.phantom(g.d, g.N, 5, 3).reshape(-1)
    r = np.random.default_rng(4).normal(size=g.m)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    rd = torch.tensor(r, dtype=torch.float32, device="cuda")
    z0 = inrct.project(g, xd).cpu().numpy()
    v0 = inrct.backproject(g, rd).cpu().numpy()
    plan = inrct.tune(g)
    assert plan["tuned"]
    assert plan["seg"] in ((1, 2, 4, 8) if g.kind == "cone3d" else (4, 8, 16))
    assert plan["zc"] in ((0, 4, 8, 16, 32) if g.kind == "cone3d" and g.N <= 512 else (4, 8, 16, 32))
    assert plan["bp_splits"] >= 1
    if g.kind != "cone3d":
        assert plan["bp_splits"] <= max(1, g.V // 8)
    z = inrct.project(g, xd).cpu().numpy()
    v = inrct.backproject(g, rd).cpu().numpy()
    assert rel(z, O.project(og(g), x)) <= 1e-5
    assert rel(v, O.backproject(og(g), r)) <= 1e-5
    # the plans differ only in the order of FP32 additions
    assert rel(z, z0) <= 1e-6 and rel(v, v0) <= 1e-6


def test_workspace_sized_before_tuning_stays_valid():
    import ctypes
    inrct.tune_reset()
    g = GEOMS[1]
    L = inrct.lib()
    gd, grd = inrct.geom_desc(g), inrct.grid_desc(2, g.N)
    nb = L.inrct_backproject_ws_bytes(ctypes.byref(gd), ctypes.byref(grd))
    inrct.tune(g)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    r = torch.randn(g.m, device="cuda")
    img = torch.empty(g.n, device="cuda")
    rc = L.backproject(ctypes.byref(gd), ctypes.byref(grd), ctypes.c_void_p(r.data_ptr()),
                       ctypes.c_void_p(img.data_ptr()), ctypes.c_void_p(ws.data_ptr()), nb,
                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    want = O.backproject(og(g), r.cpu().numpy().astype(np.float64))
    assert rel(img.cpu().numpy(), want) <= 1e-5


def test_batch_creation_tunes_every_geometry():
    inrct.tune_reset()
    arch = synth.ArchSpec("siren", 2, 128, 3, omega0=30.0)
    mlp = inrct.mlp_desc(arch, inrct.BF16)
    geoms = [synth.GeomSpec("par2d", 64, 30, 91), synth.GeomSpec("fan2d", 96, 45, 137, sod=384.0, sdd=576.0,
                                                                   span=2 * math.pi)]
    probs = []
    for k, g in enumerate(geoms):
        theta = torch.tensor(synth.init_theta(arch, k), dtype=torch.float32, device="cuda")
        probs.append({"geom": g, "theta": theta, "y": torch.zeros(g.m, device="cuda"),
                      "idx": torch.arange(g.n // 4, dtype=torch.int32, device="cuda"), "scale": 4.0,
                      "m": torch.zeros_like(theta), "s": torch.zeros_like(theta),
                      "loss": torch.zeros(1, dtype=torch.float64, device="cuda")})
    assert not any(inrct.tune_plan(g)["tuned"] for g in geoms)
    batch = inrct.Batch(mlp, probs, inrct.adam(lr=1e-3))
    assert all(inrct.tune_plan(g)["tuned"] for g in geoms)
    batch.step()
    torch.cuda.synchronize()
    assert all(np.isfinite(q["loss"].item()) for q in probs)
    batch.close()


@pytest.mark.parametrize("g", GEOMS, ids=lambda g: f"{g.kind}_{g.N}")
def test_every_candidate_plan_matches_the_oracle(g):
    """Each launch shape the tuner may choose, pinned in turn with inrct_tune_set."""
    x = synth.phantom(g.d, g.N, 5, 7).reshape(-1)
    r = np.random.default_rng(8).normal(size=g.m)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    rd = torch.tensor(r, dtype=torch.float32, device="cuda")
    zw = O.project(og(g), x)
    vw = O.backproject(og(g), r)
    cone = g.kind == "cone3d"
    plans = []
    if cone:
        plans += [(s, 1, 8) for s in (1, 2, 4, 8)] + [(4, 1, z) for z in (0, 4, 8, 16, 32)]
    else:
        inrct.tune_reset()
        default = inrct.tune_plan(g)["bp_splits"]
        most = max(1, min(g.V // 8, 2 * default))  # view splits go up to twice the default
        plans += [(s, 1, 8) for s in (4, 8, 16)] + [(8, b, 8) for b in sorted({1, 2, default, most}) if b <= most]
    for plan in plans:
        inrct.tune_set(g, *plan)
        assert rel(inrct.project(g, xd).cpu().numpy(), zw) <= 1e-5, plan
        assert rel(inrct.backproject(g, rd).cpu().numpy(), vw) <= 1e-5, plan
    inrct.tune_reset()


@pytest.mark.parametrize("g", [
    GEOMS[2],
    synth.GeomSpec("cone3d", 40, 7, 52, 44, du=1.1, sod=120.0, sdd=180.0, span=2 * math.pi),
    synth.GeomSpec("cone3d", 33, 5, 47, 39, du=1.2, dv=0.9, sod=70.0, sdd=100.0, span=2 * math.pi),
], ids=["cone40", "cone40_odd_views", "cone33_rows_not_4k"])
def test_cone_plans_agree_with_one_another(g):
    """The column adjoint (zc = 0) runs the row sweep of the chunk adjoint with 8 voxels per lane
    (N <= 256), so the two agree bit for bit, with 16-byte strip copies (rows a multiple of 4) and
    without.  The row-patch forward (seg = 1) takes the same samples and weights as the
    two-segment forward and sums them in another order: the sinograms agree to float rounding."""
    r = torch.tensor(np.random.default_rng(9).normal(size=g.m), dtype=torch.float32, device="cuda")
    inrct.tune_set(g, 2, 1, 0)
    v_col = inrct.backproject(g, r)
    inrct.tune_set(g, 2, 1, 8)
    v_chunk = inrct.backproject(g, r)
    assert torch.equal(v_col, v_chunk)
    x = torch.tensor(synth.phantom(g.d, g.N, 5, 3).reshape(-1), dtype=torch.float32, device="cuda")
    inrct.tune_set(g, 1, 1, 0)
    z_rows = inrct.project(g, x).double()
    inrct.tune_set(g, 2, 1, 0)
    z_seg2 = inrct.project(g, x).double()
    assert float((z_rows - z_seg2).norm() / z_seg2.norm()) <= 1e-6
    inrct.tune_reset()
