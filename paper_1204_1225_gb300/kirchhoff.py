"""Thin ctypes binding of libkirchhoff.so (include/kirchhoff.h).

Argument marshalling only: every step of the migration runs in the library's CUDA
kernels.  Tensors must be CUDA tensors; there is no CPU path.  The functions named
``kirchhoff_*`` mirror the C entry points one to one; ``Plan`` is a convenience wrapper.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkirchhoff.so")

KH_OK, KH_ERR_INVALID_ARG, KH_ERR_UNSUPPORTED, KH_ERR_OOM, KH_ERR_CUDA, KH_ERR_TIMEOUT, \
    KH_ERR_INTERNAL = range(7)
KH_F32, KH_F16, KH_BF16, KH_U16 = 0, 1, 2, 3
KH_VEL_CONST, KH_VEL_LINEAR_Z, KH_VEL_TABLE, KH_VEL_PSTM, KH_VEL_GRID = 0, 1, 2, 3, 4
KH_W_ONE, KH_W_OBLIQ_SPREAD, KH_W_TRUE_AMP = 0, 1, 2
KH_OPT_WAIT_POLLS, KH_OPT_FAST_MATH, KH_OPT_TILE, KH_OPT_BATCH_MODE, KH_OPT_SAMPLE_PAIRS = 1, 2, 3, 4, 5
KH_OPT_SPATIAL_SORT = 6
BATCH_MODES = {"persistent": 0, "concurrent": 1}

_STATUS = {0: "KH_OK", 1: "KH_ERR_INVALID_ARG", 2: "KH_ERR_UNSUPPORTED", 3: "KH_ERR_OOM",
           4: "KH_ERR_CUDA", 5: "KH_ERR_TIMEOUT", 6: "KH_ERR_INTERNAL"}


class KirchhoffError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class kh_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("ox", ctypes.c_double), ("oy", ctypes.c_double),
                ("oz", ctypes.c_double), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("n_bins", ctypes.c_int), ("bin_width", ctypes.c_double),
                ("vel", ctypes.c_int), ("v0", ctypes.c_double), ("k", ctypes.c_double),
                ("table_spacing", ctypes.c_double), ("table_dtype", ctypes.c_int),
                ("weight", ctypes.c_int), ("r0", ctypes.c_double), ("aperture", ctypes.c_double),
                ("nt", ctypes.c_int), ("t0", ctypes.c_double), ("dt", ctypes.c_double),
                ("trace_dtype", ctypes.c_int), ("taper", ctypes.c_double), ("aa_spacing", ctypes.c_double)]


class kh_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nz", ctypes.c_int), ("ox", ctypes.c_double), ("h", ctypes.c_double)]


class kh_job(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("ntr", ctypes.c_int), ("sx", ctypes.c_void_p),
                ("sy", ctypes.c_void_p), ("rx", ctypes.c_void_p), ("ry", ctypes.c_void_p),
                ("traces", ctypes.c_void_p), ("image", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None

EXPORTS = ["kirchhoff_create", "kirchhoff_destroy", "kirchhoff_migrate", "kirchhoff_demigrate",
           "kirchhoff_velocity_grad", "kirchhoff_traveltime", "kirchhoff_count",
           "kirchhoff_batched_prepare", "kirchhoff_migrate_batched", "kirchhoff_batch_sync",
           "kirchhoff_batch_info", "kirchhoff_batch_destroy", "kirchhoff_sync",
           "kirchhoff_set_option", "kirchhoff_launch_count", "kirchhoff_last_error",
           "kirchhoff_version", "kirchhoff_profile", "kirchhoff_profile_read",
           "kirchhoff_migrate_noalloc", "kirchhoff_fit_report", "kirchhoff_staging_stats",
           "kirchhoff_cell_grid", "kirchhoff_bin_sort", "kirchhoff_semblance", "kirchhoff_grid_layout",
           "kirchhoff_grid_tables", "kirchhoff_grid_read", "kirchhoff_migrate_host", "kirchhoff_host_join"]


def lib(path: str = LIB_PATH):
    """Loads the CUDA library; raises if it has not been built (there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"{path} is missing: build it with "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(path)
            P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_int
            L.kirchhoff_create.argtypes = [ctypes.POINTER(kh_desc), ctypes.POINTER(P)]
            L.kirchhoff_destroy.argtypes = [P]
            L.kirchhoff_migrate.argtypes = [P, I, P, P, P, P, P, P, P]
            L.kirchhoff_demigrate.argtypes = [P, I, P, P, P, P, P, P, P]
            L.kirchhoff_velocity_grad.argtypes = [P, I, P, P, P, P, P, P, P, P]
            L.kirchhoff_traveltime.argtypes = [P, I, P, P, P, P, P, P, P]
            L.kirchhoff_count.argtypes = [P, I, P, P, P, P, ctypes.POINTER(ctypes.c_int64), P]
            L.kirchhoff_batched_prepare.argtypes = [I, ctypes.POINTER(kh_job), ctypes.POINTER(P), P]
            L.kirchhoff_migrate_batched.argtypes = [P, P]
            L.kirchhoff_batch_sync.argtypes = [P, P]
            L.kirchhoff_batch_info.argtypes = [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(I),
                                               ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_longlong)]
            L.kirchhoff_batch_destroy.argtypes = [P]
            L.kirchhoff_sync.argtypes = [P, P]
            L.kirchhoff_set_option.argtypes = [P, I, ctypes.c_longlong]
            L.kirchhoff_launch_count.argtypes = [P]
            L.kirchhoff_profile.argtypes = [P, I]
            L.kirchhoff_migrate_noalloc.argtypes = [ctypes.POINTER(kh_desc), I, P, P, P, P, P, P, P, P]
            D, F = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
            L.kirchhoff_fit_report.argtypes = [ctypes.POINTER(kh_desc), I, I, I, ctypes.POINTER(I),
                                               ctypes.POINTER(I), D, F, F, F, D]
            L.kirchhoff_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_longlong)]
            U = ctypes.POINTER(ctypes.c_ulonglong)
            L.kirchhoff_staging_stats.argtypes = [P, P, U, U, U]
            L.kirchhoff_cell_grid.argtypes = [ctypes.POINTER(kh_desc), I, ctypes.POINTER(I), ctypes.POINTER(I),
                                              D, D, D]
            L.kirchhoff_bin_sort.argtypes = [P, I, P, P, P, P, P, P, P]
            L.kirchhoff_semblance.argtypes = [P, P, D, D, P, P]
            L.kirchhoff_grid_layout.argtypes = [ctypes.POINTER(kh_desc), I, ctypes.c_double, ctypes.c_double, I,
                                                ctypes.POINTER(kh_grid)]
            L.kirchhoff_grid_tables.argtypes = [P, ctypes.POINTER(kh_grid), P, I, P, P]
            L.kirchhoff_grid_read.argtypes = [P, P, P, ctypes.POINTER(I), P]
            L.kirchhoff_migrate_host.argtypes = [P, I, P, P, P, P, P, P, P]
            L.kirchhoff_host_join.argtypes = [P, P]
            for name in EXPORTS:
                getattr(L, name).restype = S
            L.kirchhoff_launch_count.restype = ctypes.c_longlong
            L.kirchhoff_last_error.restype = ctypes.c_char_p
            L.kirchhoff_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(status: int):
    if status != KH_OK:
        raise KirchhoffError(status, lib().kirchhoff_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("kirchhoff: tensors must live on a CUDA device (no CPU path)")
    if not t.is_contiguous():
        raise ValueError("kirchhoff: tensors must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _validate(specs, device=None):
    """Refuses tensors whose dtype, size or device do not match what the library reads or
    writes through their pointers (a short buffer would be read or written past its end, a
    wider dtype silently reinterpreted).  ``specs``: (tensor, name, dtype, numel, shape)
    tuples, numel or shape None when not checked.  Types and sizes are checked for every
    tensor before any device is."""
    for t, name, dtype, numel, shape in specs:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"kirchhoff: {name} must be a torch tensor")
        if t.dtype != dtype:
            raise ValueError(f"kirchhoff: {name} must be {dtype}, got {t.dtype}")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError(f"kirchhoff: {name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
        if numel is not None and t.numel() != numel:
            raise ValueError(f"kirchhoff: {name} must have {numel} elements, got {t.numel()}")
    for t, name, *_ in specs:
        if not t.is_cuda:
            raise ValueError(f"kirchhoff: {name} must live on a CUDA device (no CPU path)")
        dev = torch.cuda.current_device() if device is None else device
        if t.device.index != dev:
            raise ValueError(f"kirchhoff: {name} is on cuda:{t.device.index}, the plan's device "
                             f"is cuda:{dev}")
        if not t.is_contiguous():
            raise ValueError(f"kirchhoff: {name} must be contiguous")


def _validate_host(specs):
    """As _validate for the host-resident entry point: every tensor in host memory."""
    for t, name, dtype, numel, shape in specs:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"kirchhoff: {name} must be a torch tensor")
        if t.dtype != dtype:
            raise ValueError(f"kirchhoff: {name} must be {dtype}, got {t.dtype}")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError(f"kirchhoff: {name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
        if numel is not None and t.numel() != numel:
            raise ValueError(f"kirchhoff: {name} must have {numel} elements, got {t.numel()}")
        if t.device.type != "cpu":
            raise ValueError(f"kirchhoff: {name} must live in host memory (kirchhoff_migrate_host)")
        if not t.is_contiguous():
            raise ValueError(f"kirchhoff: {name} must be contiguous")


def _header_specs(hdr):
    return [(t, name, torch.float32, hdr.ntr, None)
            for name, t in zip(("sx", "sy", "rx", "ry"), hdr.args())]


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


_DT = {torch.float32: KH_F32, torch.float16: KH_F16, torch.bfloat16: KH_BF16}


_TABLE_DT = {torch.float32: KH_F32, torch.float16: KH_F16, "f32": KH_F32, "f16": KH_F16, "u16": KH_U16}


def desc_from(s, trace_dtype=torch.float32, vel=None, table_spacing=None,
              table_dtype="u16") -> kh_desc:
    """kh_desc from any object with the survey attributes (dim, nx, ..., nt, t0, dt).
    ``s.vel == "table"`` selects the radial traveltime table of the v0 + k z model;
    ``table_dtype`` is "f32", "f16" or "u16" (or torch.float32 / torch.float16); ``s.vel == "grid"``
    selects the per-location tables of a gridded model (kirchhoff_grid_tables)."""
    if vel is None:
        vel = {"const": KH_VEL_CONST, "linear": KH_VEL_LINEAR_Z, "table": KH_VEL_TABLE,
               "pstm": KH_VEL_PSTM, "grid": KH_VEL_GRID}[s.vel]
    if table_spacing is None:
        table_spacing = float(getattr(s, "table_spacing", 25.0))
    return kh_desc(s.dim, s.nx, s.ny if s.dim == 3 else 1, s.nz, s.ox, s.oy, s.oz, s.dx, s.dy,
                   s.dz, s.n_bins, s.bin_width, vel, s.v0, s.k, table_spacing,
                   _TABLE_DT[table_dtype], {"one": KH_W_ONE, "obliq": KH_W_OBLIQ_SPREAD, "ta": KH_W_TRUE_AMP}[s.weight],
                   s.r0, s.aperture, s.nt, s.t0, s.dt, _DT[trace_dtype], float(getattr(s, "taper", 0.0)),
                   float(getattr(s, "aa_spacing", 0.0)))


# ------------------------------------------------------------ functions named as the C ABI

def kirchhoff_create(desc: kh_desc) -> int:
    h = ctypes.c_void_p()
    _check(lib().kirchhoff_create(ctypes.byref(desc), ctypes.byref(h)))
    return h.value


def kirchhoff_destroy(plan: int) -> None:
    _check(lib().kirchhoff_destroy(ctypes.c_void_p(plan)))


def kirchhoff_migrate(plan, ntr, sx, sy, rx, ry, traces, image, stream=None) -> None:
    _check(lib().kirchhoff_migrate(ctypes.c_void_p(plan), int(ntr), _ptr(sx), _ptr(sy), _ptr(rx),
                                   _ptr(ry), _ptr(traces), _ptr(image), _stream(stream)))


def _host_ptr(t):
    if t is None:
        return None
    if t.device.type != "cpu" or not t.is_contiguous():
        raise ValueError("kirchhoff: host tensors must be contiguous and in host memory")
    return ctypes.c_void_p(t.data_ptr())


def kirchhoff_migrate_host(plan, ntr, sx, sy, rx, ry, traces, image, stream=None) -> None:
    _check(lib().kirchhoff_migrate_host(ctypes.c_void_p(plan), int(ntr), _host_ptr(sx), _host_ptr(sy),
                                        _host_ptr(rx), _host_ptr(ry), _host_ptr(traces), _host_ptr(image),
                                        _stream(stream)))


def kirchhoff_host_join(plan, stream=None) -> None:
    _check(lib().kirchhoff_host_join(ctypes.c_void_p(plan), _stream(stream)))


def kirchhoff_demigrate(plan, ntr, sx, sy, rx, ry, image, traces_out, stream=None) -> None:
    _check(lib().kirchhoff_demigrate(ctypes.c_void_p(plan), int(ntr), _ptr(sx), _ptr(sy),
                                     _ptr(rx), _ptr(ry), _ptr(image), _ptr(traces_out),
                                     _stream(stream)))


def kirchhoff_velocity_grad(plan, ntr, sx, sy, rx, ry, image, traces, out2, stream=None) -> None:
    _check(lib().kirchhoff_velocity_grad(ctypes.c_void_p(plan), int(ntr), _ptr(sx), _ptr(sy),
                                         _ptr(rx), _ptr(ry), _ptr(image), _ptr(traces), _ptr(out2),
                                         _stream(stream)))


def kirchhoff_traveltime(plan, n, px, py, pz, lx, ly, T, stream=None) -> None:
    _check(lib().kirchhoff_traveltime(ctypes.c_void_p(plan), int(n), _ptr(px), _ptr(py), _ptr(pz),
                                      _ptr(lx), _ptr(ly), _ptr(T), _stream(stream)))


def kirchhoff_count(plan, ntr, sx, sy, rx, ry, stream=None) -> int:
    out = ctypes.c_int64(0)
    _check(lib().kirchhoff_count(ctypes.c_void_p(plan), int(ntr), _ptr(sx), _ptr(sy), _ptr(rx),
                                 _ptr(ry), ctypes.byref(out), _stream(stream)))
    return int(out.value)


def kirchhoff_fit_report(desc: kh_desc, tile) -> dict:
    """Host-only: the ln(1 + rho) fits the linear-v(z) kernels use for a (cx, cy, cz) tile."""
    two, leg = ctypes.c_int(0), ctypes.c_int(0)
    bound, c1 = ctypes.c_double(0.0), ctypes.c_double(0.0)
    coef = (ctypes.c_float * 20)()
    scale, offset = ctypes.c_float(0.0), ctypes.c_float(0.0)
    _check(lib().kirchhoff_fit_report(ctypes.byref(desc), int(tile[0]), int(tile[1]), int(tile[2]),
                                      ctypes.byref(two), ctypes.byref(leg), ctypes.byref(bound), coef,
                                      ctypes.byref(scale), ctypes.byref(offset), ctypes.byref(c1)))
    return {"two_leg_terms": two.value, "leg_terms": leg.value, "leg_bound": bound.value,
            "coef": list(coef), "scale": scale.value, "offset": offset.value, "c1": c1.value}


def kirchhoff_migrate_noalloc(desc: kh_desc, ntr, sx, sy, rx, ry, traces, image, status=None,
                              stream=None) -> None:
    """Migration without any device allocation (fixed library scratch, ntr <= 65536); for
    callers that cannot allocate.  ``status``: optional CUDA int32 tensor of one element,
    zeroed by the call and set to 1 if a bounded in-kernel wait ran out (the image is then
    incomplete); read it after synchronising.  With ``status=None`` such a timeout is not
    reported at all, so pass a status tensor wherever a partial image matters."""
    ntr = int(ntr)
    specs = [(image, "image", torch.float32,
              desc.n_bins * (desc.ny if desc.dim == 3 else 1) * desc.nx * desc.nz, None)]
    if ntr > 0:
        hdr = (("sx", sx), ("rx", rx)) + ((("sy", sy), ("ry", ry)) if desc.dim == 3 else ())
        specs += [(t, name, torch.float32, ntr, None) for name, t in hdr]
        specs.append((traces, "traces", torch.float32, ntr * desc.nt, None))
    if status is not None:
        specs.append((status, "status", torch.int32, 1, None))
    _validate(specs)
    _check(lib().kirchhoff_migrate_noalloc(ctypes.byref(desc), int(ntr), _ptr(sx), _ptr(sy),
                                           _ptr(rx), _ptr(ry), _ptr(traces), _ptr(image),
                                           _ptr(status), _stream(stream)))


def kirchhoff_sync(plan, stream=None) -> None:
    _check(lib().kirchhoff_sync(ctypes.c_void_p(plan), _stream(stream)))


def kirchhoff_set_option(plan, opt: int, value: int) -> None:
    _check(lib().kirchhoff_set_option(ctypes.c_void_p(plan), int(opt), int(value)))


def kirchhoff_launch_count(plan) -> int:
    return int(lib().kirchhoff_launch_count(ctypes.c_void_p(plan)))


def kirchhoff_profile(plan, enable: bool) -> None:
    _check(lib().kirchhoff_profile(ctypes.c_void_p(plan), 1 if enable else 0))


def kirchhoff_profile_read(plan):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_longlong(0)
    _check(lib().kirchhoff_profile_read(ctypes.c_void_p(plan), ctypes.byref(ms), ctypes.byref(n)))
    return float(ms.value), int(n.value)


def kirchhoff_cell_grid(desc: kh_desc, spatial: bool = True) -> dict:
    """Host-only: the midpoint-cell grid of the binning sort for a descriptor."""
    nx, ny = ctypes.c_int(0), ctypes.c_int(0)
    gx, gy, cs = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().kirchhoff_cell_grid(ctypes.byref(desc), 1 if spatial else 0, ctypes.byref(nx),
                                     ctypes.byref(ny), ctypes.byref(gx), ctypes.byref(gy), ctypes.byref(cs)))
    return {"ncx": nx.value, "ncy": ny.value, "gx0": gx.value, "gy0": gy.value, "inv_cell": cs.value}


def kirchhoff_bin_sort(plan, ntr, sx, sy, rx, ry, perm_out, key_start_out, stream=None) -> None:
    _check(lib().kirchhoff_bin_sort(ctypes.c_void_p(plan), int(ntr), _ptr(sx), _ptr(sy), _ptr(rx),
                                    _ptr(ry), _ptr(perm_out), _ptr(key_start_out), _stream(stream)))


def kirchhoff_semblance(plan, image, bin_weight=None, grad_image=None, stream=None):
    """(V, D, B) of the offset images; fills grad_image with dV/dI when given (see the header)."""
    out = (ctypes.c_double * 3)()
    w = None
    if bin_weight is not None:
        w = (ctypes.c_double * len(bin_weight))(*[float(x) for x in bin_weight])
    _check(lib().kirchhoff_semblance(ctypes.c_void_p(plan), _ptr(image), w, out, _ptr(grad_image),
                                     _stream(stream)))
    return float(out[0]), float(out[1]), float(out[2])


def kirchhoff_grid_layout(desc: kh_desc, m: int, xmin: float, xmax: float, margin: int = 1) -> kh_grid:
    out = kh_grid()
    _check(lib().kirchhoff_grid_layout(ctypes.byref(desc), int(m), float(xmin), float(xmax), int(margin),
                                       ctypes.byref(out)))
    return out


def kirchhoff_grid_tables(plan, grid: kh_grid, v, nloc, loc_x, stream=None) -> None:
    _check(lib().kirchhoff_grid_tables(ctypes.c_void_p(plan), ctypes.byref(grid), _ptr(v), int(nloc), _ptr(loc_x),
                                       _stream(stream)))


def kirchhoff_grid_read(plan, tables=None, rounds=None, stream=None) -> int:
    n = ctypes.c_int(0)
    _check(lib().kirchhoff_grid_read(ctypes.c_void_p(plan), _ptr(tables), _ptr(rounds), ctypes.byref(n),
                                     _stream(stream)))
    return n.value


def kirchhoff_staging_stats(plan, stream=None):
    """(traces examined, traces staged, CTAs) of the staging warps since the previous read,
    while profiling is enabled; synchronises the stream."""
    a, b, c = ctypes.c_ulonglong(0), ctypes.c_ulonglong(0), ctypes.c_ulonglong(0)
    _check(lib().kirchhoff_staging_stats(ctypes.c_void_p(plan), _stream(stream), ctypes.byref(a),
                                         ctypes.byref(b), ctypes.byref(c)))
    return int(a.value), int(b.value), int(c.value)


def kirchhoff_version() -> str:
    return lib().kirchhoff_version().decode()


def _jobs_array(jobs):
    arr = (kh_job * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i] = kh_job(j["plan"], int(j["ntr"]), *(t.data_ptr() if t is not None else None
                                                     for t in (j["sx"], j["sy"], j["rx"], j["ry"],
                                                               j["traces"], j["image"])))
    return arr


def kirchhoff_batched_prepare(jobs, stream=None) -> int:
    """jobs: dicts with plan (handle), ntr, sx, sy, rx, ry, traces, image; returns a kh_batch."""
    arr = _jobs_array(jobs)
    out = ctypes.c_void_p()
    _check(lib().kirchhoff_batched_prepare(len(jobs), arr, ctypes.byref(out), _stream(stream)))
    return out.value


def kirchhoff_migrate_batched(batch, stream=None) -> None:
    _check(lib().kirchhoff_migrate_batched(ctypes.c_void_p(batch), _stream(stream)))


def kirchhoff_batch_sync(batch, stream=None) -> None:
    _check(lib().kirchhoff_batch_sync(ctypes.c_void_p(batch), _stream(stream)))


def kirchhoff_batch_info(batch) -> dict:
    n, c, w, l = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_double(), ctypes.c_longlong()
    _check(lib().kirchhoff_batch_info(ctypes.c_void_p(batch), ctypes.byref(n), ctypes.byref(c),
                                      ctypes.byref(w), ctypes.byref(l)))
    return {"items": int(n.value), "ctas": int(c.value), "est_contributions": float(w.value),
            "launches": int(l.value)}


def kirchhoff_batch_destroy(batch) -> None:
    _check(lib().kirchhoff_batch_destroy(ctypes.c_void_p(batch)))


# ------------------------------------------------------------ convenience wrapper

class Headers:
    """Trace headers on the device: FP32 (sx, sy, rx, ry)."""

    def __init__(self, sx, sy, rx, ry, device="cuda"):
        f = lambda a: torch.as_tensor(a, dtype=torch.float32).to(device).contiguous()
        self.sx, self.sy, self.rx, self.ry = f(sx), f(sy), f(rx), f(ry)

    @classmethod
    def of(cls, s, device="cuda"):
        return cls(s.sx, s.sy, s.rx, s.ry, device)

    @property
    def ntr(self) -> int:
        return int(self.sx.numel())

    def args(self):
        return self.sx, self.sy, self.rx, self.ry


class Plan:
    """Owns a kh_plan for one image grid / bin set / velocity model / trace dtype."""

    def __init__(self, s, trace_dtype=torch.float32, fast_math: bool = True, tile=None, **kw):
        self.survey = s
        self.trace_dtype = trace_dtype
        self.desc = desc_from(s, trace_dtype=trace_dtype, **kw)
        self.handle = kirchhoff_create(self.desc)
        self.image_shape = (s.n_bins, s.ny if s.dim == 3 else 1, s.nx, s.nz)
        self.nt = s.nt
        self.device = torch.cuda.current_device()
        self.spatial_sort = True
        kirchhoff_set_option(self.handle, KH_OPT_FAST_MATH, 1 if fast_math else 0)
        if tile is not None:
            cx, cy, cz = tile
            kirchhoff_set_option(self.handle, KH_OPT_TILE, cx | (cy << 10) | (cz << 20))
        self.grid = None
        if self.desc.vel == KH_VEL_GRID and getattr(s, "grid_v", None) is not None:
            self.set_grid(s.grid_v, s.grid_ox, s.grid_h, locations(s))

    def close(self):
        if getattr(self, "handle", None):
            kirchhoff_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, opt, value):
        kirchhoff_set_option(self.handle, opt, value)

    def set_tile(self, tile):
        """(cx, cy, cz) threads per CTA along x, y, z-groups, or None for the default."""
        code = 0 if tile is None else (tile[0] | (tile[1] << 10) | (tile[2] << 20))
        kirchhoff_set_option(self.handle, KH_OPT_TILE, code)

    def migrate(self, hdr: Headers, traces, out=None, stream=None):
        specs = _header_specs(hdr) + [(traces, "traces", self.trace_dtype, hdr.ntr * self.nt, None)]
        if out is not None:
            specs.append((out, "image", torch.float32, None, self.image_shape))
        _validate(specs, self.device)
        if out is None:
            out = torch.empty(self.image_shape, dtype=torch.float32, device=traces.device)
        kirchhoff_migrate(self.handle, hdr.ntr, *hdr.args(), traces, out, stream)
        return out

    def migrate_host(self, hdr, traces, out, stream=None):
        """Migration of host-resident inputs into a host image (kirchhoff_migrate_host): ``hdr``
        (sx, sy, rx, ry) CPU float32 tensors, ``traces`` a CPU tensor of the plan's trace dtype,
        ``out`` a CPU float32 tensor of the image shape, all pinned for overlap.  Only enqueues:
        consecutive calls overlap one call's copies with the other's migration.  The plan holds
        the tensors until ``sync`` (which waits for every copy); they must not change before."""
        hdr = tuple(hdr)
        ntr = int(hdr[0].numel())
        specs = [(t, name, torch.float32, ntr, None) for name, t in zip(("sx", "sy", "rx", "ry"), hdr)]
        specs += [(traces, "traces", self.trace_dtype, ntr * self.nt, None),
                  (out, "image", torch.float32, None, self.image_shape)]
        _validate_host(specs)
        self._host_refs = getattr(self, "_host_refs", []) + [(hdr, traces, out)]
        kirchhoff_migrate_host(self.handle, ntr, *hdr, traces, out, stream)
        return out

    def host_join(self, stream=None):
        """Makes ``stream`` wait until every image of ``migrate_host`` has arrived on the host."""
        kirchhoff_host_join(self.handle, stream)

    def demigrate(self, hdr: Headers, image, out=None, stream=None):
        specs = _header_specs(hdr) + [(image, "image", torch.float32, None, self.image_shape)]
        if out is not None:
            specs.append((out, "traces_out", torch.float32, hdr.ntr * self.nt, None))
        _validate(specs, self.device)
        if out is None:
            out = torch.empty((hdr.ntr, self.nt), dtype=torch.float32, device=image.device)
        kirchhoff_demigrate(self.handle, hdr.ntr, *hdr.args(), image, out, stream)
        return out

    def set_grid(self, v, ox: float, h: float, loc_x, stream=None):
        """First-arrival tables of the gridded model v [nx, nz] (m/s) on the nodes (ox + i h, j h)
        for the increasing surface positions loc_x (kirchhoff_grid_tables)."""
        v = torch.as_tensor(v, dtype=torch.float32).to(f"cuda:{self.device}").contiguous()
        loc = torch.as_tensor(loc_x, dtype=torch.float32).to(f"cuda:{self.device}").contiguous()
        if v.dim() != 2:
            raise ValueError("kirchhoff: the gridded model must be [nx, nz]")
        g = kh_grid(int(v.shape[0]), int(v.shape[1]), float(ox), float(h))
        kirchhoff_grid_tables(self.handle, g, v, loc.numel(), loc, stream)
        self.grid = g
        self.grid_nloc = loc.numel()

    def grid_tables(self, stream=None):
        """(tables float32 [nloc, nz, nx] (x fastest, as stored), rounds int32 [nloc]) of the plan's
        gridded model."""
        if self.grid is None:
            raise ValueError("kirchhoff: the plan has no gridded-model tables")
        dev = f"cuda:{self.device}"
        T = torch.empty((self.grid_nloc, self.grid.nz, self.grid.nx), dtype=torch.float32, device=dev)
        r = torch.empty(self.grid_nloc, dtype=torch.int32, device=dev)
        kirchhoff_grid_read(self.handle, T, r, stream)
        return T, r

    def velocity_grad(self, hdr: Headers, image, traces, out=None, stream=None):
        specs = _header_specs(hdr) + [(image, "image", torch.float32, None, self.image_shape),
                                      (traces, "traces", torch.float32, hdr.ntr * self.nt, None)]
        if out is not None:
            specs.append((out, "out_dv0_dk", torch.float64, 2, None))
        _validate(specs, self.device)
        if out is None:
            out = torch.empty(2, dtype=torch.float64, device=image.device)
        kirchhoff_velocity_grad(self.handle, hdr.ntr, *hdr.args(), image, traces, out, stream)
        return out

    def count(self, hdr: Headers, stream=None) -> int:
        _validate(_header_specs(hdr), self.device)
        return kirchhoff_count(self.handle, hdr.ntr, *hdr.args(), stream)

    def traveltime(self, px, py, pz, lx, ly, stream=None):
        T = torch.empty_like(px)
        kirchhoff_traveltime(self.handle, px.numel(), px, py, pz, lx, ly, T, stream)
        return T

    def sync(self, stream=None):
        """Waits for the plan's work on ``stream`` (and for every image of ``migrate_host``) and
        raises if a kernel reported a timed-out wait or a skipped trace."""
        if getattr(self, "_host_refs", None):
            kirchhoff_host_join(self.handle, stream)
        kirchhoff_sync(self.handle, stream)
        self._host_refs = []

    def profile(self, enable: bool = True):
        kirchhoff_profile(self.handle, enable)

    def profile_read(self):
        """(summed main-kernel milliseconds, timed launches) since the previous read."""
        return kirchhoff_profile_read(self.handle)

    def semblance(self, image, bin_weight=None, grad=False, stream=None):
        """(V, dV/dI or None) of an offset-binned image of this plan (velocity analysis)."""
        specs = [(image, "image", torch.float32, None, self.image_shape)]
        if bin_weight is not None and len(bin_weight) != self.survey.n_bins:
            raise ValueError("kirchhoff: one bin weight per offset bin")
        _validate(specs, self.device)
        g = torch.empty_like(image) if grad else None
        V, _, _ = kirchhoff_semblance(self.handle, image, bin_weight, g, stream)
        return V, g

    def bin_sort(self, hdr: Headers, stream=None):
        """The binning sort of this plan: (perm [ntr] int32, key starts int32) on the device."""
        _validate(_header_specs(hdr), self.device)
        grid = kirchhoff_cell_grid(self.desc, bool(self.spatial_sort))
        nkeys = self.survey.n_bins * grid["ncx"] * grid["ncy"]
        perm = torch.full((max(hdr.ntr, 1),), -1, dtype=torch.int32, device=hdr.sx.device)
        starts = torch.empty(nkeys + 1, dtype=torch.int32, device=hdr.sx.device)
        kirchhoff_bin_sort(self.handle, hdr.ntr, *hdr.args(), perm, starts, stream)
        return perm[:hdr.ntr], starts, grid

    def set_spatial_sort(self, on: bool):
        kirchhoff_set_option(self.handle, KH_OPT_SPATIAL_SORT, 1 if on else 0)
        self.spatial_sort = bool(on)

    def staging_stats(self, stream=None):
        """(traces examined, traces staged, CTAs) of the staging warps since the previous read."""
        return kirchhoff_staging_stats(self.handle, stream)

    @property
    def launches(self) -> int:
        return kirchhoff_launch_count(self.handle)


def locations(s):
    """The distinct surface positions (source and receiver x) of a 2D survey's traces, increasing
    (float32): the locations of its gridded-model tables."""
    import numpy as np
    return np.unique(np.concatenate([np.asarray(s.sx, np.float32), np.asarray(s.rx, np.float32)]))


def arrival_times_fn(plan: "Plan"):
    """Arrival-time callable for ``survey.synthesize`` computed by the library's traveltime
    kernel: two-way time source -> point -> receiver, float64 tensor [n_points, m]."""

    def fn(points, s, trace_idx):
        dev = torch.device("cuda")
        p = torch.as_tensor(points, dtype=torch.float32, device=dev)
        j = torch.as_tensor(trace_idx, device=dev, dtype=torch.int64)
        n, m = p.shape[0], j.numel()
        sx = torch.as_tensor(s.sx, device=dev)[j]
        rx = torch.as_tensor(s.rx, device=dev)[j]
        sy = torch.as_tensor(s.sy, device=dev)[j]
        ry = torch.as_tensor(s.ry, device=dev)[j]
        px = p[:, 0:1].expand(n, m).contiguous().view(-1)
        py = p[:, 1:2].expand(n, m).contiguous().view(-1)
        pz = p[:, 2:3].expand(n, m).contiguous().view(-1)
        ts = plan.traveltime(px, py, pz, sx.expand(n, m).contiguous().view(-1),
                             sy.expand(n, m).contiguous().view(-1))
        tr = plan.traveltime(px, py, pz, rx.expand(n, m).contiguous().view(-1),
                             ry.expand(n, m).contiguous().view(-1))
        return (ts.double() + tr.double()).view(n, m)

    return fn


class Batch:
    """Many migrations in one launch sequence (kirchhoff_batched_prepare / _migrate_batched).

    ``jobs`` is a list of (Plan, Headers, traces, image) with device tensors; the traces and
    images are read / written in place by every run (and every graph replay).  ``mode`` is
    "persistent" (one persistent kernel over the work list) or "concurrent" (each job's own
    kernel on forked library streams)."""

    def __init__(self, jobs, stream=None, mode: str = "persistent"):
        self._keep = list(jobs)
        self.mode = mode
        kirchhoff_set_option(self._keep[0][0].handle, KH_OPT_BATCH_MODE, BATCH_MODES[mode])
        self.handle = kirchhoff_batched_prepare(
            [{"plan": p.handle, "ntr": h.ntr, "sx": h.sx, "sy": h.sy, "rx": h.rx, "ry": h.ry,
              "traces": d, "image": m} for (p, h, d, m) in self._keep], stream)
        self.graph = None

    def run(self, stream=None):
        kirchhoff_migrate_batched(self.handle, stream)

    def capture(self):
        """Captures one run in a CUDA graph (on a side stream) and returns it."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.run(s)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def sync(self, stream=None):
        kirchhoff_batch_sync(self.handle, stream)

    def info(self) -> dict:
        return kirchhoff_batch_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            self.graph = None
            kirchhoff_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
