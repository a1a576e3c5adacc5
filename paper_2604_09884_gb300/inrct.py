"""Thin ctypes binding of libinrct.so (include/inrct.h), same names as the C ABI.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Tensors must be contiguous CUDA tensors of the documented dtype;
PyTorch provides the device memory (outputs and workspaces) and the current
stream.  The library is loaded on first use; if it is missing the call raises
(there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import torch

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libinrct.so")

PAR2D, FAN2D, CONE3D = 0, 1, 2
FFN_RELU, SIREN, HASH = 0, 1, 2
FP32, BF16 = 0, 1
LOSS_LS, LOSS_FLS = 0, 1
_GKIND = {"par2d": PAR2D, "fan2d": FAN2D, "cone3d": CONE3D}
_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "WORKSPACE", 4: "CUDA", 5: "TIMEOUT"}


class InrctError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"inrct {_STATUS.get(code, code)}: {msg}")
        self.code = code


class Geom(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_views", ctypes.c_int), ("n_bins_u", ctypes.c_int),
                ("n_bins_v", ctypes.c_int), ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("sod", ctypes.c_double), ("sdd", ctypes.c_double), ("angle0", ctypes.c_double),
                ("angle_span", ctypes.c_double)]


class Grid(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("N", ctypes.c_int), ("fov", ctypes.c_int)]


class Mlp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("d", ctypes.c_int), ("n_feat", ctypes.c_int),
                ("B", ctypes.c_void_p), ("omega0", ctypes.c_float), ("n_hidden", ctypes.c_int),
                ("width", ctypes.c_int), ("prec", ctypes.c_int),
                ("hash_levels", ctypes.c_int), ("hash_feats", ctypes.c_int),
                ("hash_log2_T", ctypes.c_int), ("hash_base", ctypes.c_int),
                ("hash_growth", ctypes.c_double), ("B_host", ctypes.c_void_p)]


class Adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("t", ctypes.c_int64)]


class Problem(ctypes.Structure):
    _fields_ = [("geom", Geom), ("grid", Grid), ("theta", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("idx", ctypes.c_void_p), ("n_idx", ctypes.c_int64), ("scale", ctypes.c_double),
                ("adam_m", ctypes.c_void_p), ("adam_s", ctypes.c_void_p), ("loss_out", ctypes.c_void_p)]


_lib = None
_P = ctypes.c_void_p
_SZ = ctypes.c_size_t
_I64 = ctypes.c_int64


def lib():
    """Load libinrct.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise InrctError(4, f"{LIB_PATH} is missing: run paper_2604_09884_gb300.build.build() "
                            "(or __graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    g, gr, m = ctypes.POINTER(Geom), ctypes.POINTER(Grid), ctypes.POINTER(Mlp)
    sig = {
        "inrct_last_error": ([], ctypes.c_char_p),
        "inrct_num_params": ([m], _I64),
        "inrct_num_rays": ([g], _I64),
        "inrct_project_ws_bytes": ([g, gr], _SZ),
        "project": ([g, gr, _P, _P, _P, _P, _P, _P, _SZ, _P], ctypes.c_int),
        "project_noalloc": ([g, gr, _P, _P, _P, _P, _P, _P], ctypes.c_int),
        "inrct_backproject_ws_bytes": ([g, gr], _SZ),
        "backproject": ([g, gr, _P, _P, _P, _SZ, _P], ctypes.c_int),
        "inrct_ramp_ws_bytes": ([g, gr], _SZ),
        "ramp_filter": ([g, gr, _P, _P, _P, _P, _SZ, _P], ctypes.c_int),
        "inrct_eval_ws_bytes": ([m, gr], _SZ),
        "inr_eval_grid": ([m, _P, gr, _P, _P, _SZ, _P], ctypes.c_int),
        "inrct_vjp_ws_bytes": ([m, gr, _I64], _SZ),
        "inr_weighted_vjp": ([m, _P, gr, _P, _I64, _P, ctypes.c_double, _P, _P, _P, _SZ, _P],
                             ctypes.c_int),
        "inr_virtual_loss": ([m, _P, gr, _P, _I64, _P, ctypes.c_double, _P, _P, _P, _P, _SZ, _P],
                             ctypes.c_int),
        "inrct_device_status": ([_P], ctypes.c_int),
        "inrct_set_wait_limit": ([ctypes.c_ulonglong], ctypes.c_int),
        "inrct_debug_stall_weight_loads": ([ctypes.c_int], ctypes.c_int),
        "inrct_step_ws_bytes": ([g, gr, m, _I64], _SZ),
        "inrct_launch_count": ([], ctypes.c_longlong),
        "inrct_profile_begin": ([ctypes.c_int], ctypes.c_int),
        "inrct_profile_end": ([ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                               ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "inrct_gemm_tn_ws_bytes": ([_I64, ctypes.c_int, ctypes.c_int], _SZ),
        "inrct_gemm_tn": ([_P, _P, _P, _I64, ctypes.c_int, ctypes.c_int, _P, _P, _SZ, _P], ctypes.c_int),
        "grad_step": ([g, gr, m, ctypes.c_int, _P, _P, _P, _I64, ctypes.c_double,
                       ctypes.POINTER(Adam), _P, _P, _P, _P, _P, _SZ, _P], ctypes.c_int),
        "inrct_sincospi": ([_P, _P, _P, _I64, _P], ctypes.c_int),
        "inrct_batch_ws_bytes": ([m, ctypes.POINTER(Problem), ctypes.c_int], _SZ),
        "inrct_batch_create": ([m, ctypes.c_int, ctypes.POINTER(Problem), ctypes.c_int,
                                ctypes.POINTER(Adam), _P, _P, _SZ, ctypes.POINTER(_P)], ctypes.c_int),
        "grad_step_batched": ([_P, _P], ctypes.c_int),
        "inrct_batch_destroy": ([_P], ctypes.c_int),
        "inrct_check_index_ws_bytes": ([gr], _SZ),
        "inrct_check_index_set": ([gr, _P, _I64, ctypes.POINTER(ctypes.c_longlong), _P, _SZ, _P], ctypes.c_int),
        "inrct_tune_ws_bytes": ([g, gr], _SZ),
        "inrct_tune": ([g, gr, _P, _SZ, _P], ctypes.c_int),
        "inrct_tune_plan": ([g, gr] + [ctypes.POINTER(ctypes.c_int)] * 4, ctypes.c_int),
        "inrct_tune_reset": ([], ctypes.c_int),
        "inrct_tune_set": ([g, gr, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise InrctError(rc, lib().inrct_last_error().decode())


def _ptr(t, dtype=None, numel=None, name="tensor"):
    """Device address of t.  The library takes plain pointers, so a wrong element type, a buffer
    shorter than the call needs, or a strided view would be read or written out of bounds: each
    is refused here (element type and size first, so that these checks need no GPU)."""
    if t is None:
        return None
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name}: {t.numel()} elements, the call needs {numel}")
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError(f"{name}: expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ws(nbytes, device):
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


# ----------------------------------------------------------------------------
# descriptors
# ----------------------------------------------------------------------------
def geom_desc(g: synth.GeomSpec) -> Geom:
    return Geom(_GKIND[g.kind], g.V, g.A, g.B if g.kind == "cone3d" else 1, g.du, g.dv, g.sod,
                g.sdd, g.angle0, g.span)


def grid_desc(d: int, N: int, fov: int = 0) -> Grid:
    return Grid(d, N, fov)


def view_subset(g: synth.GeomSpec, n_subsets: int, s: int) -> synth.GeomSpec:
    """Subset s of n_subsets interleaved view subsets (views s, s + S, s + 2S, ...), for the
    ordered-subsets use of Algorithm 1 (Sec. 3): the same scan with V/S views starting at
    angle0 + span s / V and the same span.  V must be divisible by n_subsets."""
    if n_subsets < 1 or g.V % n_subsets or not 0 <= s < n_subsets:
        raise InrctError(1, f"{g.V} views cannot form subset {s} of {n_subsets}")
    kw = g.as_dict()
    kw.update(V=g.V // n_subsets, angle0=g.angle0 + g.span * s / g.V)
    return synth.GeomSpec(**kw)


def view_subset_rows(g: synth.GeomSpec, sino: torch.Tensor, n_subsets: int, s: int) -> torch.Tensor:
    """The rows of a sinogram of g ([view][...]) that belong to view_subset(g, n_subsets, s)."""
    per_view = g.m // g.V
    return sino.view(g.V, per_view)[s::n_subsets].contiguous().view(-1)


@dataclass
class MlpHandle:
    """An inrct_mlp descriptor plus the device Fourier matrix it points to (and the host copy
    that B_host points to)."""
    desc: Mlp
    B: torch.Tensor | None
    spec: synth.ArchSpec
    B_host: torch.Tensor | None = None

    @property
    def p(self):
        return self.spec.p


def mlp_desc(a: synth.ArchSpec, prec: int, B=None, device="cuda") -> MlpHandle:
    Bt = Bh = None
    if a.kind == "ffn":
        Bt = torch.as_tensor(B, dtype=torch.float32, device=device).contiguous()
        assert Bt.shape == (a.n_feat, a.d)
        Bh = Bt.cpu().contiguous()  # the same values, for B_host
    kind = {"ffn": FFN_RELU, "siren": SIREN, "hash": HASH}[a.kind]
    desc = Mlp(kind, a.d, a.n_feat, Bt.data_ptr() if Bt is not None else None, a.omega0,
               a.n_hidden, a.width, prec)
    if a.kind == "hash":
        desc.hash_levels, desc.hash_feats, desc.hash_log2_T = a.hash_levels, a.hash_feats, a.hash_log2_T
        desc.hash_base, desc.hash_growth = a.hash_base, a.hash_growth
    if Bh is not None:
        desc.B_host = Bh.data_ptr()
    return MlpHandle(desc, Bt, a, Bh)


# ----------------------------------------------------------------------------
# calls (names follow the C ABI)
# ----------------------------------------------------------------------------
def num_params(mlp: MlpHandle) -> int:
    return int(lib().inrct_num_params(ctypes.byref(mlp.desc)))


def num_rays(g: synth.GeomSpec) -> int:
    gd = geom_desc(g)
    return int(lib().inrct_num_rays(ctypes.byref(gd)))


def project(g: synth.GeomSpec, image: torch.Tensor, y: torch.Tensor | None = None, stream=None):
    """z = P x; with y also r = z - y and L = 1/2 ||r||^2.  Returns z, or (z, r, L)."""
    L = lib()
    gd, grd = geom_desc(g), grid_desc(g.d, g.N, g.fov)
    dev = image.device
    z = torch.empty(g.m, dtype=torch.float32, device=dev)
    r = torch.empty(g.m, dtype=torch.float32, device=dev) if y is not None else None
    loss = torch.empty(1, dtype=torch.float64, device=dev) if y is not None else None
    nb = L.inrct_project_ws_bytes(ctypes.byref(gd), ctypes.byref(grd))
    ws = _ws(nb, dev)
    _check(L.project(ctypes.byref(gd), ctypes.byref(grd), _ptr(image, torch.float32, g.n, "image"), _ptr(z),
                     _ptr(y, torch.float32, g.m, "y"), _ptr(r), _ptr(loss), _ptr(ws), nb, _stream(stream)))
    return z if y is None else (z, r, loss)


def project_noalloc(g: synth.GeomSpec, image: torch.Tensor, y: torch.Tensor | None = None,
                    stream=None):
    """project() without a caller workspace: the library's fixed static scratch is used.
    For callers that may not allocate device scratch; the outputs are still the caller's."""
    L = lib()
    gd, grd = geom_desc(g), grid_desc(g.d, g.N, g.fov)
    dev = image.device
    z = torch.empty(g.m, dtype=torch.float32, device=dev)
    r = torch.empty(g.m, dtype=torch.float32, device=dev) if y is not None else None
    loss = torch.empty(1, dtype=torch.float64, device=dev) if y is not None else None
    _check(L.project_noalloc(ctypes.byref(gd), ctypes.byref(grd), _ptr(image, torch.float32, g.n, "image"),
                             _ptr(z), _ptr(y, torch.float32, g.m, "y"), _ptr(r), _ptr(loss), _stream(stream)))
    return z if y is None else (z, r, loss)


def backproject(g: synth.GeomSpec, sino: torch.Tensor, stream=None) -> torch.Tensor:
    """v = P^T r (exact adjoint of project)."""
    L = lib()
    gd, grd = geom_desc(g), grid_desc(g.d, g.N, g.fov)
    dev = sino.device
    v = torch.empty(g.n, dtype=torch.float32, device=dev)
    nb = L.inrct_backproject_ws_bytes(ctypes.byref(gd), ctypes.byref(grd))
    ws = _ws(nb, dev)
    _check(L.backproject(ctypes.byref(gd), ctypes.byref(grd), _ptr(sino, torch.float32, g.m, "sino"), _ptr(v),
                         _ptr(ws), nb, _stream(stream)))
    return v


def tune(g: synth.GeomSpec, device="cuda", stream=None) -> dict:
    """Time the projector launch-shape candidates of this geometry and keep the fastest
    (inrct_tune); returns the plan now in use."""
    L = lib()
    gd, grd = geom_desc(g), grid_desc(g.d, g.N, g.fov)
    nb = L.inrct_tune_ws_bytes(ctypes.byref(gd), ctypes.byref(grd))
    if nb == 0:
        _check(L.inrct_tune(ctypes.byref(gd), ctypes.byref(grd), None, 0, _stream(stream)))
    ws = _ws(nb, torch.device(device))
    _check(L.inrct_tune(ctypes.byref(gd), ctypes.byref(grd), _ptr(ws), nb, _stream(stream)))
    return tune_plan(g)


def check_index_set(d: int, N: int, idx: torch.Tensor, fov: int = 0, stream=None) -> dict:
    """Counts of out-of-range, outside-the-FOV and repeated entries of an index set."""
    L = lib()
    grd = grid_desc(d, N, fov)
    nb = L.inrct_check_index_ws_bytes(ctypes.byref(grd))
    ws = _ws(nb, idx.device)
    c = (ctypes.c_longlong * 3)()
    _check(L.inrct_check_index_set(ctypes.byref(grd), _ptr(idx, torch.int32, name="idx"), idx.numel(), c, _ptr(ws), nb,
                                   _stream(stream)))
    return {"out_of_range": c[0], "outside_fov": c[1], "repeats": c[2]}


def tune_plan(g: synth.GeomSpec) -> dict:
    """The projector launch plan in use for this geometry (inrct_tune_plan)."""
    L = lib()
    gd, grd = geom_desc(g), grid_desc(g.d, g.N, g.fov)
    v = [ctypes.c_int() for _ in range(4)]
    _check(L.inrct_tune_plan(ctypes.byref(gd), ctypes.byref(grd), *[ctypes.byref(x) for x in v]))
    return {"seg": v[0].value, "bp_splits": v[1].value, "zc": v[2].value, "tuned": bool(v[3].value)}


def tune_set(g: synth.GeomSpec, seg: int, bp_splits: int, zc: int) -> None:
    """Pin a projector launch plan for this geometry (inrct_tune_set)."""
    gd, grd = geom_desc(g), grid_desc(g.d, g.N, g.fov)
    _check(lib().inrct_tune_set(ctypes.byref(gd), ctypes.byref(grd), seg, bp_splits, zc))


def tune_reset() -> None:
    _check(lib().inrct_tune_reset())


def ramp_filter(g: synth.GeomSpec, r: torch.Tensor, stream=None):
    """(F r, 1/2 r^T F r) with F the ramp filter of the FLS loss."""
    L = lib()
    gd, grd = geom_desc(g), grid_desc(g.d, g.N, g.fov)
    out = torch.empty_like(r)
    loss = torch.empty(1, dtype=torch.float64, device=r.device)
    nb = L.inrct_ramp_ws_bytes(ctypes.byref(gd), ctypes.byref(grd))
    ws = _ws(nb, r.device)
    _check(L.ramp_filter(ctypes.byref(gd), ctypes.byref(grd), _ptr(r, torch.float32, g.m, "r"), _ptr(out),
                         _ptr(loss), _ptr(ws), nb, _stream(stream)))
    return out, loss


def inr_eval_grid(mlp: MlpHandle, theta: torch.Tensor, N: int, stream=None, fov: int = 0) -> torch.Tensor:
    """E{f_theta} on the N^d grid (flat, x fastest); zero outside the field of view if fov."""
    L = lib()
    grd = grid_desc(mlp.spec.d, N, fov)
    img = torch.empty(N ** mlp.spec.d, dtype=torch.float32, device=theta.device)
    nb = L.inrct_eval_ws_bytes(ctypes.byref(mlp.desc), ctypes.byref(grd))
    ws = _ws(nb, theta.device)
    _check(L.inr_eval_grid(ctypes.byref(mlp.desc), _ptr(theta, torch.float32, mlp.p, "theta"), ctypes.byref(grd),
                           _ptr(img), _ptr(ws), nb, _stream(stream)))
    return img


def inr_weighted_vjp(mlp: MlpHandle, theta: torch.Tensor, N: int, idx: torch.Tensor,
                     v: torch.Tensor, scale: float, want_f32: bool = False, stream=None, fov: int = 0):
    """scale * sum_k v[idx[k]] grad f(x_idx[k]) as FP64 (and FP32 if asked); with fov, listed
    points outside the field of view contribute nothing."""
    L = lib()
    grd = grid_desc(mlp.spec.d, N, fov)
    dev = theta.device
    g64 = torch.empty(mlp.p, dtype=torch.float64, device=dev)
    g32 = torch.empty(mlp.p, dtype=torch.float32, device=dev) if want_f32 else None
    nb = L.inrct_vjp_ws_bytes(ctypes.byref(mlp.desc), ctypes.byref(grd), idx.numel())
    ws = _ws(nb, dev)
    _check(L.inr_weighted_vjp(ctypes.byref(mlp.desc), _ptr(theta, torch.float32, mlp.p, "theta"),
                              ctypes.byref(grd), _ptr(idx, torch.int32, name="idx"), idx.numel(),
                              _ptr(v, torch.float32, N ** mlp.spec.d, "v"),
                              float(scale), _ptr(g64), _ptr(g32), _ptr(ws), nb, _stream(stream)))
    return (g64, g32) if want_f32 else g64


def inr_virtual_loss(mlp: MlpHandle, theta: torch.Tensor, N: int, idx: torch.Tensor,
                     v: torch.Tensor, scale: float, want_f32: bool = False, stream=None, fov: int = 0):
    """The virtual loss of Eq. 3, scale * sum_k v[idx[k]] f(x_idx[k]) (FP64 [1]), and its gradient
    (FP64, and FP32 if asked), both from one library call."""
    L = lib()
    grd = grid_desc(mlp.spec.d, N, fov)
    dev = theta.device
    val = torch.empty(1, dtype=torch.float64, device=dev)
    g64 = torch.empty(mlp.p, dtype=torch.float64, device=dev)
    g32 = torch.empty(mlp.p, dtype=torch.float32, device=dev) if want_f32 else None
    nb = L.inrct_vjp_ws_bytes(ctypes.byref(mlp.desc), ctypes.byref(grd), idx.numel())
    ws = _ws(nb, dev)
    _check(L.inr_virtual_loss(ctypes.byref(mlp.desc), _ptr(theta, torch.float32, mlp.p, "theta"),
                              ctypes.byref(grd), _ptr(idx, torch.int32, name="idx"), idx.numel(),
                              _ptr(v, torch.float32, N ** mlp.spec.d, "v"), float(scale), _ptr(val), _ptr(g64),
                              _ptr(g32), _ptr(ws), nb, _stream(stream)))
    return (val, g64, g32) if want_f32 else (val, g64)


def device_status(stream=None) -> None:
    """Synchronise the stream and raise InrctError (TIMEOUT) if a bounded wait of a tensor-core
    kernel gave up since the last check (inrct_device_status); clears the status."""
    _check(lib().inrct_device_status(_stream(stream)))


def set_wait_limit(ns: int) -> None:
    """Limit of every bounded wait of later tensor-core launches, in ns (0: the default, 1 s)."""
    _check(lib().inrct_set_wait_limit(int(ns)))


def debug_stall_weight_loads(on: bool) -> None:
    """Test hook: while on, the tile kernel issues no weight loads (its first MMA wait runs out)."""
    _check(lib().inrct_debug_stall_weight_loads(1 if on else 0))


def step_ws_bytes(g: synth.GeomSpec, mlp: MlpHandle, n_idx: int) -> int:
    gd, grd = geom_desc(g), grid_desc(g.d, g.N, g.fov)
    return int(lib().inrct_step_ws_bytes(ctypes.byref(gd), ctypes.byref(grd), ctypes.byref(mlp.desc),
                                         n_idx))


def grad_step(g: synth.GeomSpec, mlp: MlpHandle, theta: torch.Tensor, y: torch.Tensor,
              idx: torch.Tensor, scale: float, adam: Adam | None, m: torch.Tensor | None,
              s: torch.Tensor | None, loss_out: torch.Tensor | None = None,
              grad_out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
              loss_kind: int = LOSS_LS, stream=None):
    """Algorithm 1 + Adam in place on theta/m/s.  ws may be preallocated (step_ws_bytes)."""
    L = lib()
    gd, grd = geom_desc(g), grid_desc(g.d, g.N, g.fov)
    if ws is None:
        ws = _ws(step_ws_bytes(g, mlp, idx.numel()), theta.device)
    p = mlp.p
    _check(L.grad_step(ctypes.byref(gd), ctypes.byref(grd), ctypes.byref(mlp.desc), loss_kind,
                       _ptr(theta, torch.float32, p, "theta"), _ptr(y, torch.float32, g.m, "y"),
                       _ptr(idx, torch.int32, name="idx"), idx.numel(), float(scale),
                       ctypes.byref(adam) if adam is not None else None,
                       _ptr(m, torch.float32, p, "m"), _ptr(s, torch.float32, p, "s"),
                       _ptr(loss_out, torch.float64, 1, "loss_out"), _ptr(grad_out, torch.float64, p, "grad_out"),
                       _ptr(ws, torch.uint8, name="ws"), ws.numel(), _stream(stream)))


class Batch:
    """grad_step_batched over independent problems sharing one INR architecture.

    problems: list of dicts with keys geom (GeomSpec), theta, y, idx, scale, m, s and
    optionally loss (a [1] float64 tensor).  The tensors are held here so their
    addresses stay valid for the recorded graph; their contents may change between
    steps.  `counter` is the device step index (int64 [1]), advanced by every step()."""

    def __init__(self, mlp: MlpHandle, problems: list, adam: Adam, loss_kind: int = LOSS_LS,
                 device="cuda"):
        L = lib()
        self._keep = [mlp, problems]
        arr = (Problem * len(problems))()
        for k, q in enumerate(problems):
            g = q["geom"]
            p = mlp.p
            arr[k] = Problem(geom_desc(g), grid_desc(g.d, g.N, g.fov),
                             _ptr(q["theta"], torch.float32, p, f"problem {k} theta").value,
                             _ptr(q["y"], torch.float32, g.m, f"problem {k} y").value,
                             _ptr(q["idx"], torch.int32, name=f"problem {k} idx").value,
                             q["idx"].numel(), float(q["scale"]),
                             _ptr(q["m"], torch.float32, p, f"problem {k} m").value,
                             _ptr(q["s"], torch.float32, p, f"problem {k} s").value,
                             _ptr(q["loss"], torch.float64, 1, f"problem {k} loss").value
                             if q.get("loss") is not None else None)
        self._arr = arr
        nb = L.inrct_batch_ws_bytes(ctypes.byref(mlp.desc), arr, len(problems))
        if nb == 0:
            raise InrctError(1, "invalid problem table")
        self.ws = _ws(nb, device)
        self.counter = torch.zeros(1, dtype=torch.int64, device=device)
        self._adam = adam
        h = ctypes.c_void_p()
        _check(L.inrct_batch_create(ctypes.byref(mlp.desc), loss_kind, arr, len(problems), ctypes.byref(adam),
                                    _ptr(self.counter), _ptr(self.ws), self.ws.numel(), ctypes.byref(h)))
        self._h = h

    def step(self, stream=None):
        _check(lib().grad_step_batched(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().inrct_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sincospi(x: torch.Tensor, stream=None):
    """Diagnostic: (sin(pi x), cos(pi x)) as the FFN feature code computes them (x in [-1, 1])."""
    sn = torch.empty_like(x)
    cs = torch.empty_like(x)
    _check(lib().inrct_sincospi(_ptr(x, torch.float32, name="x"), _ptr(sn), _ptr(cs), x.numel(), _stream(stream)))
    return sn, cs


def gemm_tn(X: torch.Tensor, Y: torch.Tensor | None, Y16: torch.Tensor | None, stream=None):
    """Diagnostic: [X^T Y | X^T 1 (16 cols) | X^T Y16^T] from the weight-gradient GEMM (BF16 in)."""
    L = lib()
    K, M = X.shape
    N = Y.shape[1] if Y is not None else 0
    C = torch.empty(M, N + 32, dtype=torch.float32, device=X.device)
    nb = L.inrct_gemm_tn_ws_bytes(K, M, N)
    ws = _ws(nb, X.device)
    _check(L.inrct_gemm_tn(_ptr(X, torch.bfloat16, name="X"), _ptr(Y, torch.bfloat16, K * N, "Y"),
                           _ptr(Y16, torch.bfloat16, 16 * K, "Y16"),
                           K, M, N, _ptr(C), _ptr(ws), nb, _stream(stream)))
    return C


STAGES = ["eval_prep", "eval_mlp_kernel", "project_loss", "backproject", "vjp_prep",
          "vjp_mlp_kernel", "vjp_dw_gemm_reduce", "adam"]


def launch_count() -> int:
    return int(lib().inrct_launch_count())


def profile_begin(max_steps: int):
    _check(lib().inrct_profile_begin(max_steps))


def profile_end() -> tuple[dict, int]:
    """Summed milliseconds per grad_step stage over the recorded steps, and the step count."""
    arr = (ctypes.c_double * len(STAGES))()
    steps = ctypes.c_int(0)
    _check(lib().inrct_profile_end(arr, len(STAGES), ctypes.byref(steps)))
    return dict(zip(STAGES, list(arr))), steps.value


def adam(lr=1e-4, beta1=0.9, beta2=0.999, eps=1e-8, t=1) -> Adam:
    return Adam(lr, beta1, beta2, eps, t)


class InrVirtualLoss(torch.autograd.Function):
    """Virtual loss of Eq. (3): L~(theta) = scale * sum_{i in I} v_i f_theta(x_i), v held constant.

    forward makes one library call, inr_virtual_loss, which runs the fused VJP at the listed
    points and returns both the value (from the forward pass the VJP runs there) and the
    gradient of Eq. (2); backward hands autograd that gradient times the incoming grad_out.
    No per-point activation is kept between the two.

    Usage: ``InrVirtualLoss.apply(theta, v, idx, scale, mlp, N)``; the result is a 0-d FP64
    tensor, and ``backward()`` leaves the FP32 gradient in ``theta.grad``.
    """

    @staticmethod
    def forward(ctx, theta, v, idx, scale, mlp, N, fov=0):
        value, grad = inr_virtual_loss(mlp, theta, int(N), idx, v, float(scale), fov=fov)
        ctx.save_for_backward(grad)
        return value.reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return (grad_out.to(grad.dtype) * grad).to(torch.float32), None, None, None, None, None, None
