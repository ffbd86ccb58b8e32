"""ctypes binding of libwoi.so (C ABI: include/woi.h).

Argument marshalling only: every step of the estimator runs in the library's
CUDA kernels.  The functions mirror the C entry points (woi_create_geometry,
woi_set_sigma_and_data, woi_estimate, woi_estimate_range, woi_walk_values,
woi_estimate_batch); `Geometry` adds a problem-dictionary constructor (the
format of `workloads`).  Arrays may be numpy (host) or torch tensors (host or
CUDA); torch CUDA tensors are passed as device pointers and, by default, the
current torch stream is used.

There is no CPU fallback: if libwoi.so is missing or fails to load, importing
this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

WOI_MAX_DIM = 6
WOI_SPHERE, WOI_STAR, WOI_ELLIPSOID, WOI_MESH = 0, 1, 2, 3
KIND = {"sphere": WOI_SPHERE, "star": WOI_STAR, "ellipsoid": WOI_ELLIPSOID, "mesh": WOI_MESH}
FLUX = {"zero": 0, "fourier": 1, "real_sh": 2, "harmonic_poly": 3, "point_charge": 4}
WOI_PLAIN, WOI_VR = 0, 1
WOI_MIXED, WOI_FP64_PLAIN = 0, 1
STATUS = {0: "WOI_OK", 1: "WOI_E_INVALID_ARG", 2: "WOI_E_GEOMETRY", 3: "WOI_E_COMPAT", 4: "WOI_E_UNSUPPORTED",
          5: "WOI_E_NO_DEVICE", 6: "WOI_E_CUDA", 7: "WOI_E_OOM", 8: "WOI_E_TIMEOUT", 9: "WOI_E_STATE"}
EXPORTED = ["woi_default_opts", "woi_create_geometry", "woi_set_sigma_and_data", "woi_estimate",
            "woi_estimate_range", "woi_walk_values", "woi_walk_trace", "woi_estimate_batch", "woi_last_kernel_ms",
            "woi_estimate_noalloc", "woi_autotune", "woi_surface_area", "woi_finalize_moments",
            "woi_check_status",
            "woi_destroy_geometry", "woi_last_error", "woi_version"]


class WoiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SurfaceDesc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("center", ctypes.c_double * WOI_MAX_DIM), ("radius", ctypes.c_double),
                ("star_degree", ctypes.c_int), ("star_a", ctypes.POINTER(ctypes.c_double)),
                ("star_b", ctypes.POINTER(ctypes.c_double)), ("matrix", ctypes.POINTER(ctypes.c_double)),
                ("n_vertices", ctypes.c_int), ("vertices", ctypes.POINTER(ctypes.c_double)),
                ("n_triangles", ctypes.c_int), ("triangles", ctypes.POINTER(ctypes.c_int))]


class FluxDesc(ctypes.Structure):
    _fields_ = [("basis", ctypes.c_int), ("n_coef", ctypes.c_int), ("coef", ctypes.POINTER(ctypes.c_double))]


class Opts(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("variant", ctypes.c_int), ("precision", ctypes.c_int),
                ("sched_group", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("block_size", ctypes.c_int),
                ("walks_per_lane", ctypes.c_int), ("timing", ctypes.c_int), ("tile_points", ctypes.c_int)]


def library_path() -> str:
    return _build.LIB


def _load():
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"libwoi.so not built ({path}); run paper_2508_16767_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, vp, i64, u64, dp = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
    lib.woi_default_opts.argtypes = [P(Opts)]
    lib.woi_default_opts.restype = None
    lib.woi_create_geometry.argtypes = [ctypes.c_int, ctypes.c_int, P(SurfaceDesc), P(ctypes.c_int), P(vp)]
    lib.woi_set_sigma_and_data.argtypes = [vp, P(ctypes.c_double), P(FluxDesc)]
    lib.woi_estimate.argtypes = [vp, P(Opts), dp, i64, i64, u64, dp, dp, dp, dp]
    lib.woi_estimate_range.argtypes = [vp, P(Opts), dp, i64, i64, i64, u64, dp]
    lib.woi_check_status.argtypes = [vp]
    lib.woi_finalize_moments.argtypes = [ctypes.c_int, i64, i64, ctypes.c_int, dp, vp, dp, dp, dp, dp]
    lib.woi_walk_values.argtypes = [vp, P(Opts), dp, ctypes.c_uint32, ctypes.c_uint32, dp, i64, u64, dp, dp]
    lib.woi_walk_trace.argtypes = [vp, P(Opts), dp, ctypes.c_uint32, ctypes.c_uint32, dp, i64, u64, dp, dp, dp]
    lib.woi_estimate_batch.argtypes = [ctypes.c_int, P(vp), P(Opts), P(ctypes.c_int), P(vp), P(i64), P(i64), u64,
                                       P(vp), P(vp), P(vp), P(vp)]
    lib.woi_last_kernel_ms.argtypes = [vp, P(ctypes.c_float)]
    lib.woi_estimate_noalloc.argtypes = [vp, P(Opts), dp, i64, i64, u64, dp, dp, dp, dp]
    lib.woi_autotune.argtypes = [vp, P(Opts), dp, i64, i64, u64, P(ctypes.c_int), P(ctypes.c_int)]
    lib.woi_surface_area.argtypes = [vp, ctypes.c_int, P(ctypes.c_double)]
    lib.woi_destroy_geometry.argtypes = [vp]
    lib.woi_destroy_geometry.restype = None
    lib.woi_last_error.restype = ctypes.c_char_p
    lib.woi_version.restype = ctypes.c_char_p
    for name in ["woi_create_geometry", "woi_set_sigma_and_data", "woi_estimate", "woi_estimate_range",
                 "woi_walk_values", "woi_walk_trace", "woi_estimate_batch", "woi_last_kernel_ms",
                 "woi_estimate_noalloc", "woi_autotune"]:
        getattr(lib, name).restype = ctypes.c_int
    return lib


lib = _load()


def _check(status):
    if status != 0:
        raise WoiError(status, lib.woi_last_error().decode())


def version() -> str:
    return lib.woi_version().decode()


def woi_version() -> str:
    return lib.woi_version().decode()


def woi_last_error() -> str:
    return lib.woi_last_error().decode()


def woi_default_opts() -> "Opts":
    o = Opts()
    lib.woi_default_opts(ctypes.byref(o))
    return o


def woi_surface_area(handle, i) -> float:
    a = ctypes.c_double()
    _check(lib.woi_surface_area(handle, int(i), ctypes.byref(a)))
    return a.value


# ---------------------------------------------------------------------------
# array marshalling
# ---------------------------------------------------------------------------

def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """Address of a contiguous float64 / uint64 array (numpy or torch), or None."""
    if a is None:
        return None
    if _is_torch(a):
        assert a.is_contiguous()
        return a.data_ptr()
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _stream_of(arrays, stream):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    for a in arrays:
        if a is not None and _is_torch(a) and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def make_opts(M=4, variant="plain", precision="mixed", sched_group=1, stream=None, block_size=0,
              walks_per_lane=0, timing=False, tile_points=0) -> Opts:
    o = Opts()
    lib.woi_default_opts(ctypes.byref(o))
    o.M = int(M)
    o.variant = {"plain": WOI_PLAIN, "vr": WOI_VR}[variant]
    o.precision = {"mixed": WOI_MIXED, "fp64": WOI_FP64_PLAIN}[precision]
    o.sched_group = int(sched_group)
    o.cuda_stream = stream
    o.block_size = int(block_size)
    o.walks_per_lane = int(walks_per_lane)
    o.timing = int(bool(timing))
    o.tile_points = int(tile_points)
    return o


def woi_check_status(geom) -> None:
    """Waits for the last asynchronous estimate on `geom` and raises WoiError
    (WOI_E_GEOMETRY) if one of its lines crossed a mesh more than 32 times."""
    _check(lib.woi_check_status(geom.handle))


def woi_last_kernel_ms(geom) -> float:
    """Walk-kernel duration of the last estimate run with timing=True."""
    ms = ctypes.c_float()
    _check(lib.woi_last_kernel_ms(geom.handle, ctypes.byref(ms)))
    return float(ms.value)


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------

def woi_create_geometry(dim, surfaces, parent):
    """surfaces: list of dicts {"kind", "center", "radius", "star_a", "star_b", "matrix", "vertices",
    "triangles"}."""
    n = len(surfaces)
    arr = (SurfaceDesc * n)()
    keep = []
    for i, s in enumerate(surfaces):
        arr[i].type = KIND[s["kind"]]
        for k, v in enumerate(s["center"]):
            arr[i].center[k] = float(v)
        arr[i].radius = float(s.get("radius", 0.0))
        if s["kind"] == "ellipsoid":
            m = np.ascontiguousarray(s["matrix"], dtype=np.float64)
            keep.append(m)
            arr[i].matrix = m.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if s["kind"] == "mesh":
            V = np.ascontiguousarray(s["vertices"], dtype=np.float64)
            F = np.ascontiguousarray(s["triangles"], dtype=np.int32)
            keep += [V, F]
            arr[i].n_vertices = len(V)
            arr[i].vertices = V.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            arr[i].n_triangles = len(F)
            arr[i].triangles = F.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        if s["kind"] == "star":
            a = np.ascontiguousarray(s["star_a"], dtype=np.float64)
            b = np.ascontiguousarray(s["star_b"], dtype=np.float64)
            keep += [a, b]
            arr[i].star_degree = len(a) - 1
            arr[i].star_a = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            arr[i].star_b = b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    par = (ctypes.c_int * n)(*[int(p) for p in parent])
    h = ctypes.c_void_p()
    _check(lib.woi_create_geometry(int(dim), n, arr, par, ctypes.byref(h)))
    return h


def woi_destroy_geometry(handle):
    lib.woi_destroy_geometry(handle)


def woi_set_sigma_and_data(handle, sigma, flux):
    n = len(sigma)
    sig = (ctypes.c_double * n)(*[float(s) for s in sigma])
    fl = (FluxDesc * n)()
    keep = []
    for i, f in enumerate(flux):
        c = np.ascontiguousarray(f["coef"], dtype=np.float64)
        keep.append(c)
        fl[i].basis = FLUX[f["basis"]]
        fl[i].n_coef = len(c)
        fl[i].coef = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if len(c) else None
    _check(lib.woi_set_sigma_and_data(handle, sig, fl))


class Geometry:
    """A problem (geometry + sigma + flux) held by the library."""

    def __init__(self, problem):
        self.problem = problem
        self.dim = int(problem["dim"])
        self.n_surf = len(problem["surfaces"])
        self.handle = woi_create_geometry(self.dim, problem["surfaces"], problem["parent"])
        try:
            woi_set_sigma_and_data(self.handle, problem["sigma"], problem["flux"])
        except Exception:
            lib.woi_destroy_geometry(self.handle)
            self.handle = None
            raise

    def surface_area(self, i):
        """|dOmega_i| as the estimator uses it."""
        a = ctypes.c_double()
        _check(lib.woi_surface_area(self.handle, int(i), ctypes.byref(a)))
        return a.value

    def close(self):
        if getattr(self, "handle", None):
            lib.woi_destroy_geometry(self.handle)
            self.handle = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------------------------
# estimates
# ---------------------------------------------------------------------------

def _as_input(a):
    """Contiguous float64 view or copy of an input array (numpy or torch)."""
    if _is_torch(a):
        import torch
        if a.dtype != torch.float64:
            a = a.to(torch.float64)
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=np.float64)


def _alloc_like(points, shape):
    if _is_torch(points):
        import torch
        return torch.empty(shape, dtype=torch.float64, device=points.device)
    return np.empty(shape, dtype=np.float64)


def woi_estimate(geom: Geometry, points, n_walks, seed=0, out=None, stream=None, **opt):
    """u, grad, se_u, se_grad at `points` [P, dim] (numpy or torch, host or CUDA).
    Outputs are allocated like `points` unless `out` = (u, grad, se_u, se_grad)."""
    points = _as_input(points)
    P = int(points.shape[0])
    if out is None:
        out = (_alloc_like(points, (P,)), _alloc_like(points, (P, geom.dim)), _alloc_like(points, (P,)),
               _alloc_like(points, (P, geom.dim)))
    o = make_opts(M=opt.pop("M", geom.problem.get("M", 4)), stream=_stream_of([points, *out], stream), **opt)
    _check(lib.woi_estimate(geom.handle, ctypes.byref(o), _ptr(points), P, int(n_walks), int(seed), *[_ptr(a) for a in out]))
    return {"u": out[0], "grad": out[1], "se_u": out[2], "se_grad": out[3]}


def woi_estimate_range(geom: Geometry, points, walk_begin, n_walks, seed=0, stream=None, **opt):
    """Raw moments [P, 2, dim+1] (sum of f, sum of squared schedule-group means)."""
    points = _as_input(points)
    P = int(points.shape[0])
    mom = _alloc_like(points, (P, 2, geom.dim + 1))
    o = make_opts(M=opt.pop("M", geom.problem.get("M", 4)), stream=_stream_of([points, mom], stream), **opt)
    _check(lib.woi_estimate_range(geom.handle, ctypes.byref(o), _ptr(points), P, int(walk_begin), int(n_walks),
                                  int(seed), _ptr(mom)))
    return mom


def woi_walk_values(geom: Geometry, x, walk_ids, seed=0, point_id=0, instance_id=0, **opt):
    """Per-walk tallies (host arrays) of one point for pathwise replay."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    ids = np.ascontiguousarray(walk_ids, dtype=np.uint64)
    n = len(ids)
    fu = np.zeros(n)
    fg = np.zeros((n, geom.dim))
    o = make_opts(M=opt.pop("M", geom.problem.get("M", 4)), **opt)
    _check(lib.woi_walk_values(geom.handle, ctypes.byref(o), x.ctypes.data, int(point_id), int(instance_id),
                               ids.ctypes.data, n, int(seed), fu.ctypes.data, fg.ctypes.data))
    return {"u": fu, "grad": fg}


def woi_walk_trace(geom: Geometry, x, walk_ids, seed=0, point_id=0, instance_id=0, **opt):
    """Per-walk tallies and per-step states (y, Q, T) of every chain."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    ids = np.ascontiguousarray(walk_ids, dtype=np.uint64)
    n = len(ids)
    M = opt.pop("M", geom.problem.get("M", 4))
    chains = 2 if opt.get("variant", "plain") == "vr" else 1
    fu = np.zeros(n)
    fg = np.zeros((n, geom.dim))
    tr = np.zeros((n, chains, M + 1, geom.dim + 2))
    o = make_opts(M=M, **opt)
    _check(lib.woi_walk_trace(geom.handle, ctypes.byref(o), x.ctypes.data, int(point_id), int(instance_id),
                              ids.ctypes.data, n, int(seed), fu.ctypes.data, fg.ctypes.data, tr.ctypes.data))
    return {"u": fu, "grad": fg, "Y": tr[..., :geom.dim], "Q": tr[..., geom.dim], "T": tr[..., geom.dim + 1]}


def woi_autotune(geom: Geometry, points, n_walks, seed=0, stream=None, **opt):
    """Tune (block size, walks per lane) of the FP32 walk kernel on this workload;
    later calls with block_size = walks_per_lane = 0 use the choice."""
    points = _as_input(points)
    b, l = ctypes.c_int(), ctypes.c_int()
    o = make_opts(M=opt.pop("M", geom.problem.get("M", 4)), stream=_stream_of([points], stream), **opt)
    _check(lib.woi_autotune(geom.handle, ctypes.byref(o), _ptr(points), int(points.shape[0]), int(n_walks), int(seed),
                            ctypes.byref(b), ctypes.byref(l)))
    return b.value, l.value


def woi_estimate_batch(instances, seed=0, stream=None, out=None, **opt):
    """Batched estimate.  instances: list of (Geometry, points, n_walks[, M]);
    points numpy (host) or torch tensors (host, e.g. pinned, or CUDA).  Instance k
    uses random-stream instance id k.  Returns a list of dicts like woi_estimate,
    with outputs allocated like each instance's points unless out[k] =
    (u, grad, se_u, se_grad) is given."""
    n = len(instances)
    P = ctypes.POINTER
    geoms = (ctypes.c_void_p * n)()
    pts = (ctypes.c_void_p * n)()
    npts = (ctypes.c_int64 * n)()
    nw = (ctypes.c_int64 * n)()
    ms = (ctypes.c_int * n)()
    outs = [(ctypes.c_void_p * n)() for _ in range(4)]
    keep, results = [], []
    for k, inst in enumerate(instances):
        geom, points, n_walks = inst[0], _as_input(inst[1]), inst[2]
        M = inst[3] if len(inst) > 3 else geom.problem.get("M", 4)
        Pk = int(points.shape[0])
        res_k = out[k] if out is not None else (_alloc_like(points, (Pk,)), _alloc_like(points, (Pk, geom.dim)),
                                                _alloc_like(points, (Pk,)), _alloc_like(points, (Pk, geom.dim)))
        keep += [points, *res_k]
        geoms[k], pts[k], npts[k], nw[k], ms[k] = geom.handle, _ptr(points), Pk, int(n_walks), int(M)
        for j in range(4):
            outs[j][k] = _ptr(res_k[j])
        results.append({"u": res_k[0], "grad": res_k[1], "se_u": res_k[2], "se_grad": res_k[3]})
    arrays = [inst[1] for inst in instances]
    o = make_opts(M=4, stream=_stream_of(arrays, stream), **opt)
    _check(lib.woi_estimate_batch(n, geoms, ctypes.byref(o), ms, pts, npts, nw, int(seed), *outs))
    return results


def woi_finalize_moments(moments, n_walks, sched_group=1, out=None, stream=None):
    """u, grad, se_u, se_grad from raw moments [P, 2, dim+1] (numpy or torch, host or
    CUDA) of n_walks walks per point -- e.g. the sum of the moments of disjoint walk
    ranges -- computed by the library's finalize kernel."""
    if not _is_torch(moments):
        moments = np.ascontiguousarray(moments, dtype=np.float64)
    P, two, C = (int(v) for v in moments.shape)
    assert two == 2
    dim = C - 1
    if out is None:
        out = (_alloc_like(moments, (P,)), _alloc_like(moments, (P, dim)), _alloc_like(moments, (P,)),
               _alloc_like(moments, (P, dim)))
    _check(lib.woi_finalize_moments(dim, P, int(n_walks), int(sched_group), _ptr(moments),
                                    _stream_of([moments, *out], stream), *[_ptr(a) for a in out]))
    return {"u": out[0], "grad": out[1], "se_u": out[2], "se_grad": out[3]}


def finalize_moments(mom, n_walks, sched_group=1):
    """Mean and SE of merged raw moments through the library (woi_finalize_moments)."""
    return woi_finalize_moments(mom, n_walks, sched_group)


def woi_estimate_noalloc(geom: Geometry, points, n_walks, seed=0, out=None, stream=None, **opt):
    """The allocation-free estimate: points and outputs must be CUDA tensors
    (outputs are allocated here by torch when `out` is None -- callers that may
    not allocate pass their own).  Scratch comes from the library's fixed
    device array; see include/woi.h."""
    points = _as_input(points)
    P = int(points.shape[0])
    if out is None:
        out = (_alloc_like(points, (P,)), _alloc_like(points, (P, geom.dim)), _alloc_like(points, (P,)),
               _alloc_like(points, (P, geom.dim)))
    o = make_opts(M=opt.pop("M", geom.problem.get("M", 4)), stream=_stream_of([points, *out], stream), **opt)
    _check(lib.woi_estimate_noalloc(geom.handle, ctypes.byref(o), _ptr(points), P, int(n_walks), int(seed),
                                    *[_ptr(a) for a in out]))
    return {"u": out[0], "grad": out[1], "se_u": out[2], "se_grad": out[3]}
