"""The C-ABI library loads, exports every symbol include/inrct.h declares, and
rejects bad arguments on the host before any GPU work (no compute calls here)."""
import ctypes
import os
import re

import pytest
import torch  # noqa: F401  (loads the CUDA runtime the library links against)

from paper_2604_09884_gb300 import build as B
from paper_2604_09884_gb300 import inrct, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "inrct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return inrct.lib()


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert {"project", "backproject", "inr_eval_grid", "inr_weighted_vjp", "grad_step",
            "grad_step_batched"} <= set(names)
    for n in names:
        assert hasattr(L, n), n


def test_param_and_ray_counts(L):
    for w in synth.workloads().values():
        a = w.arch
        m = inrct.Mlp({"ffn": 0, "siren": 1, "hash": 2}[a.kind], a.d, a.n_feat, ctypes.c_void_p(256).value,
                      a.omega0, a.n_hidden, a.width, inrct.FP32, a.hash_levels, a.hash_feats, a.hash_log2_T,
                      a.hash_base, a.hash_growth)
        assert inrct.num_params(inrct.MlpHandle(m, None, a)) == a.p
        assert inrct.num_rays(w.geom) == w.geom.m


def _fake(n=4096):
    return ctypes.c_void_p(n)


def test_validation_errors_are_reported_on_the_host(L):
    g = synth.GeomSpec("fan2d", 64, 10, 91, sod=100.0, sdd=150.0, span=6.283)
    gd, grd = inrct.geom_desc(g), inrct.grid_desc(2, 64)
    nb = L.inrct_project_ws_bytes(ctypes.byref(gd), ctypes.byref(grd))
    assert nb > 0
    # workspace too small
    rc = L.project(ctypes.byref(gd), ctypes.byref(grd), _fake(), _fake(), None, None, None,
                   _fake(), nb - 512, None)
    assert rc == 3 and b"workspace" in L.inrct_last_error()
    # NULL image
    rc = L.project(ctypes.byref(gd), ctypes.byref(grd), None, _fake(), None, None, None, _fake(),
                   nb, None)
    assert rc == 1
    # grid/geometry dimension mismatch
    grd3 = inrct.grid_desc(3, 64)
    assert L.backproject(ctypes.byref(gd), ctypes.byref(grd3), _fake(), _fake(), _fake(), 1 << 30,
                         None) == 1
    # source inside the grid
    bad = inrct.geom_desc(synth.GeomSpec("fan2d", 64, 10, 91, sod=20.0, sdd=40.0))
    assert L.backproject(ctypes.byref(bad), ctypes.byref(grd), _fake(), _fake(), _fake(), 1 << 30,
                         None) == 1
    # cone too wide for x/y driving axes
    wide = inrct.geom_desc(synth.GeomSpec("cone3d", 64, 4, 64, 2000, sod=100.0, sdd=150.0))
    assert L.project(ctypes.byref(wide), ctypes.byref(grd3), _fake(), _fake(), None, None, None,
                     _fake(), 1 << 40, None) == 2
    # n_idx = 0
    a = synth.ArchSpec("siren", 2, 64, 2)
    m = inrct.Mlp(1, 2, 0, None, 30.0, 2, 64, inrct.FP32)
    rc = L.inr_weighted_vjp(ctypes.byref(m), _fake(), ctypes.byref(grd), _fake(), 0, _fake(), 1.0,
                            _fake(), None, _fake(), 1 << 30, None)
    assert rc == 1 and b"n_idx" in L.inrct_last_error()
    # unsupported width
    m_bad = inrct.Mlp(1, 2, 0, None, 30.0, 2, 96, inrct.FP32)
    assert L.inr_eval_grid(ctypes.byref(m_bad), _fake(), ctypes.byref(grd), _fake(), _fake(),
                           1 << 30, None) == 1
    # FFN without its Fourier matrix
    m_ffn = inrct.Mlp(0, 2, 16, None, 0.0, 2, 64, inrct.FP32)
    assert L.inr_eval_grid(ctypes.byref(m_ffn), _fake(), ctypes.byref(grd), _fake(), _fake(),
                           1 << 30, None) == 1
    assert L.inrct_vjp_ws_bytes(ctypes.byref(m), ctypes.byref(grd), 1000) > 0
    assert L.inrct_step_ws_bytes(ctypes.byref(gd), ctypes.byref(grd), ctypes.byref(m), 1000) > 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(inrct, "_lib", None)
    monkeypatch.setattr(inrct, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(inrct.InrctError):
        inrct.lib()


def _problem(g, ptr=256, n_idx=16):
    p = ctypes.c_void_p(ptr).value
    return inrct.Problem(inrct.geom_desc(g), inrct.grid_desc(g.d, g.N), p, p, p, n_idx, 4.0, p, p, None)


def test_batch_create_rejects_a_bad_problem_by_index(L):
    a = synth.ArchSpec("siren", 2, 128, 3, omega0=30.0)
    h = inrct.MlpHandle(inrct.Mlp(1, 2, 0, None, 30.0, 3, 128, inrct.BF16), None, a)
    good = synth.GeomSpec("par2d", 64, 30, 91)
    bad = synth.GeomSpec("par2d", 64, 0, 91)          # no views
    arr = (inrct.Problem * 2)(_problem(good), _problem(bad))
    out = ctypes.c_void_p()
    counter = ctypes.c_void_p(256)
    rc = L.inrct_batch_create(ctypes.byref(h.desc), 0, arr, 2, ctypes.byref(inrct.adam()), counter,
                              counter, 1 << 30, ctypes.byref(out))
    assert rc == 1 and b"problem 1" in L.inrct_last_error() and not out.value


def test_batch_create_requires_its_workspace(L):
    a = synth.ArchSpec("siren", 2, 128, 3, omega0=30.0)
    h = inrct.MlpHandle(inrct.Mlp(1, 2, 0, None, 30.0, 3, 128, inrct.BF16), None, a)
    g = synth.GeomSpec("fan2d", 64, 30, 91, sod=256.0, sdd=384.0, span=2 * 3.141592653589793)
    arr = (inrct.Problem * 1)(_problem(g))
    need = L.inrct_batch_ws_bytes(ctypes.byref(h.desc), arr, 1)
    assert need > L.inrct_step_ws_bytes(ctypes.byref(inrct.geom_desc(g)), ctypes.byref(inrct.grid_desc(2, 64)),
                                         ctypes.byref(h.desc), 16)
    out = ctypes.c_void_p()
    rc = L.inrct_batch_create(ctypes.byref(h.desc), 0, arr, 1, ctypes.byref(inrct.adam()),
                              ctypes.c_void_p(256), ctypes.c_void_p(256), need - 1, ctypes.byref(out))
    assert rc == 3 and not out.value


def test_view_subset_rejects_uneven_splits_and_keeps_the_scan():
    g = synth.GeomSpec("fan2d", 32, 12, 45, sod=128.0, sdd=192.0, span=6.283185307179586, angle0=0.3)
    with pytest.raises(inrct.InrctError):
        inrct.view_subset(g, 5, 0)
    s = inrct.view_subset(g, 4, 3)
    assert (s.V, s.A, s.sod, s.span) == (3, 45, 128.0, g.span)
    assert abs(s.angle0 - (0.3 + g.span * 3 / 12)) < 1e-15


def test_hash_descriptor_is_validated_on_the_host(L):
    grd = inrct.grid_desc(2, 64)

    def mlp(**kw):
        f = dict(levels=4, feats=2, log2T=10, base=4, growth=1.5, prec=inrct.FP32, width=64)
        f.update(kw)
        return inrct.Mlp(inrct.HASH, 2, 0, None, 0.0, 2, f["width"], f["prec"], f["levels"], f["feats"],
                         f["log2T"], f["base"], f["growth"])

    good = mlp()
    assert L.inrct_num_params(ctypes.byref(good)) == 4 * 1024 * 2 + (64 * 8 + 64) + (64 * 64 + 64) + 65
    assert L.inrct_vjp_ws_bytes(ctypes.byref(good), ctypes.byref(grd), 1000) > 0
    bad = [mlp(levels=0), mlp(levels=17), mlp(feats=3), mlp(levels=16, feats=8), mlp(log2T=3),
           mlp(log2T=25), mlp(base=0), mlp(growth=0.9), mlp(growth=4.5), mlp(prec=inrct.BF16),
           mlp(levels=16, base=65536, growth=4.0)]          # finest resolution above 2^20
    for m in bad:
        assert L.inrct_num_params(ctypes.byref(m)) == 0
        rc = L.inr_eval_grid(ctypes.byref(m), _fake(), ctypes.byref(grd), _fake(), _fake(), 1 << 30, None)
        assert rc == 1, (m.hash_levels, m.hash_feats, m.hash_log2_T, m.hash_base, m.hash_growth, m.prec)
        assert b"hash" in L.inrct_last_error()


def test_projector_plans_default_without_tuning(L):
    """Without inrct_tune the plans are the built-in defaults (host-side lookup, no GPU)."""
    assert inrct.tune_reset() is None
    g2 = synth.GeomSpec("fan2d", 64, 90, 91, sod=100.0, sdd=150.0, span=6.283)
    p = inrct.tune_plan(g2)
    # 2-D: 8 segments; view splits = min(ceil(456 / tiles), views / 8) = min(114, 11)
    assert p == {"seg": 8, "bp_splits": 11, "zc": 8, "tuned": False}
    g3 = synth.GeomSpec("cone3d", 64, 10, 96, 96, sod=200.0, sdd=300.0)
    # cone adjoint: the column kernel (zc = 0) where it fits (N <= 512, <= 1024 detector rows)
    assert inrct.tune_plan(g3) == {"seg": 1, "bp_splits": 1, "zc": 0, "tuned": False}
    g4 = synth.GeomSpec("cone3d", 600, 10, 96, 96, sod=2000.0, sdd=3000.0)
    assert inrct.tune_plan(g4) == {"seg": 1, "bp_splits": 1, "zc": 8, "tuned": False}
    gd, grd = inrct.geom_desc(g2), inrct.grid_desc(2, 64)
    nb = L.inrct_tune_ws_bytes(ctypes.byref(gd), ctypes.byref(grd))
    assert nb > 0
    # too small a workspace is refused before any launch
    assert L.inrct_tune(ctypes.byref(gd), ctypes.byref(grd), _fake(), nb - 1024, None) == 3
    assert b"workspace" in L.inrct_last_error()
    # a mismatched grid is refused
    grd3 = inrct.grid_desc(3, 64)
    assert L.inrct_tune_ws_bytes(ctypes.byref(gd), ctypes.byref(grd3)) == 0


def test_pinned_plans_are_validated_on_the_host(L):
    inrct.tune_reset()
    g2 = synth.GeomSpec("fan2d", 64, 90, 91, sod=100.0, sdd=150.0, span=6.283)
    inrct.tune_set(g2, 16, 3, 8)                        # 16 segments per ray, 3 view splits
    assert inrct.tune_plan(g2) == {"seg": 16, "bp_splits": 3, "zc": 8, "tuned": True}
    g3 = synth.GeomSpec("cone3d", 64, 10, 96, 96, sod=200.0, sdd=300.0)
    inrct.tune_set(g3, 2, 1, 0)                         # the column kernel fits this geometry
    assert inrct.tune_plan(g3)["zc"] == 0
    g4 = synth.GeomSpec("cone3d", 600, 10, 96, 96, sod=2000.0, sdd=3000.0)
    big = synth.GeomSpec("par2d", 2048, 30, 2900)
    for g, plan in [(g2, (3, 1, 8)), (g2, (1, 1, 8)), (g2, (8, 0, 8)), (g2, (8, 12, 8)), (g2, (8, 1, 5)),
                    (g3, (3, 1, 8)), (g3, (16, 1, 8)), (g4, (2, 1, 0)), (big, (8, 1, 64))]:
        with pytest.raises(inrct.InrctError) as e:
            inrct.tune_set(g, *plan)
        assert e.value.code == 1
    inrct.tune_reset()
    assert not inrct.tune_plan(g2)["tuned"]


def test_field_of_view_flag_is_validated_on_the_host(L):
    g = synth.GeomSpec("fan2d", 64, 10, 91, sod=100.0, sdd=150.0, span=6.283)
    gd = inrct.geom_desc(g)
    m = inrct.Mlp(1, 2, 0, None, 30.0, 2, 64, inrct.FP32)
    for fov, ok in [(0, True), (1, True), (2, False), (-1, False)]:
        grd = inrct.grid_desc(2, 64, fov)
        assert (L.inrct_project_ws_bytes(ctypes.byref(gd), ctypes.byref(grd)) > 0) == ok
        assert (L.inrct_vjp_ws_bytes(ctypes.byref(m), ctypes.byref(grd), 100) > 0) == ok
        if not ok:
            rc = L.inr_eval_grid(ctypes.byref(m), _fake(), ctypes.byref(grd), _fake(), _fake(), 1 << 30, None)
            assert rc == 1 and b"fov" in L.inrct_last_error()


def test_index_set_check_refuses_on_the_host(L):
    grd = inrct.grid_desc(2, 64, 1)
    nb = L.inrct_check_index_ws_bytes(ctypes.byref(grd))
    assert nb >= 256 + 64 * 64 // 8
    c = (ctypes.c_longlong * 3)()
    assert L.inrct_check_index_set(ctypes.byref(grd), _fake(), 10, c, _fake(), nb - 256, None) == 3
    bad = inrct.grid_desc(2, 64, 3)
    assert L.inrct_check_index_set(ctypes.byref(bad), _fake(), 10, c, _fake(), nb, None) == 1


def test_binding_refuses_wrong_buffers_before_any_launch(L):
    """The library takes plain pointers; the binding refuses a wrong element type, a buffer
    shorter than the call needs and a non-CUDA or strided tensor (no GPU is touched)."""
    with pytest.raises(TypeError, match="theta"):
        inrct._ptr(torch.zeros(8, dtype=torch.float64), torch.float32, 8, "theta")
    with pytest.raises(ValueError, match="7 elements"):
        inrct._ptr(torch.zeros(7), torch.float32, 8, "m")
    with pytest.raises(ValueError, match="contiguous CUDA"):
        inrct._ptr(torch.zeros(8), torch.float32, 8, "s")
    assert inrct._ptr(None, torch.float32, 8, "grad_out") is None
    g = synth.GeomSpec("par2d", 16, 6, 23)
    with pytest.raises(TypeError, match="image"):
        inrct.project(g, torch.zeros(g.n, dtype=torch.float64))
    with pytest.raises(ValueError, match="image"):
        inrct.project(g, torch.zeros(g.n - 1))
    with pytest.raises(ValueError, match="sino"):
        inrct.backproject(g, torch.zeros(g.m - 1))


def test_mlp_struct_mirrors_the_header():
    """The binding's inrct_mlp mirror has the header's fields, in the header's order."""
    hdr = open(os.path.join(ROOT, "include", "inrct.h")).read()
    body = hdr[:hdr.index("} inrct_mlp;")]
    body = body[body.rindex("typedef struct {") + len("typedef struct {"):]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = [re.findall(r"\**(\w+)\s*$", decl.strip())[0] for decl in body.split(";") if decl.strip()]
    assert names == [f[0] for f in inrct.Mlp._fields_]
