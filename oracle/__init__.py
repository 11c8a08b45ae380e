"""FP64 CPU oracle for Kirchhoff prestack migration (paper Sec. 3, Eq. 1).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  The product (``paper_1204_1225_gb300``)
never does, and this package never imports the product.

The arithmetic lives in ``kh_oracle.c`` (plain C, double precision, OpenMP over image
columns or traces); this module compiles it with gcc and wraps it with ctypes, and adds
the textbook CGLS iteration in numpy for least-squares migration.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libkh_oracle.so")
_SRC = os.path.join(_HERE, "kh_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("ox", ctypes.c_double), ("oy", ctypes.c_double),
                ("oz", ctypes.c_double), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("n_bins", ctypes.c_int),
                ("bin_width", ctypes.c_double), ("vel", ctypes.c_int), ("v0", ctypes.c_double),
                ("k", ctypes.c_double), ("weight", ctypes.c_int), ("r0", ctypes.c_double),
                ("aperture", ctypes.c_double), ("nt", ctypes.c_int), ("t0", ctypes.c_double),
                ("dt", ctypes.c_double), ("table_spacing", ctypes.c_double), ("taper", ctypes.c_double),
                ("gtab", ctypes.c_void_p), ("gloc", ctypes.c_void_p), ("gnloc", ctypes.c_int),
                ("gnx", ctypes.c_int), ("gnz", ctypes.c_int), ("gox", ctypes.c_double),
                ("gh", ctypes.c_double), ("aa_spacing", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            L = ctypes.c_long
            D = ctypes.POINTER(_Desc)
            for name in ("ko_migrate", "ko_demigrate"):
                getattr(_lib, name).argtypes = [D, L, P, P, P, P, P, P]
                getattr(_lib, name).restype = ctypes.c_int
            _lib.ko_vgrad.argtypes = [D, L, P, P, P, P, P, P, P, P]
            _lib.ko_migrate_points.argtypes = [D, L, P, P, P, P, P, L, P, P, P]
            _lib.ko_migrate_points.restype = ctypes.c_int
            _lib.ko_bins.argtypes = [D, L, P, P, P, P, P]
            _lib.ko_traveltime.argtypes = [D, L, P, P, P, P, P]
            _lib.ko_table_traveltime.argtypes = [D, L, P, P, P]
            _lib.ko_count.argtypes = [D, L, P, P, P, P]
            _lib.ko_arrivals.argtypes = [D, L, P, P, P, L, P, P, P, P, P]
            _lib.ko_count.restype = ctypes.c_longlong
            I = ctypes.c_int
            Dbl = ctypes.c_double
            _lib.ko_eikonal.argtypes = [I, I, Dbl, Dbl, P, Dbl, I, Dbl, P]
            _lib.ko_eikonal.restype = I
            _lib.ko_grid_tables.argtypes = [I, I, Dbl, Dbl, P, I, P, I, Dbl, P, P]
            _lib.ko_grid_tables.restype = I
            _lib.ko_grid_traveltime.argtypes = [D, I, L, P, P, P]
            _lib.ko_ta_weight.argtypes = [D, L, P, P]
            _lib.ko_aa_weight.argtypes = [D, L, P, P]
            _lib.ko_set_mutation.argtypes = [ctypes.c_int]
            _lib.ko_set_threads.argtypes = [ctypes.c_int]
            _lib.ko_max_threads.restype = ctypes.c_int
    return _lib


def desc(s) -> _Desc:
    """Oracle descriptor from a ``Survey`` (any object with the same attribute names).  For vel
    "grid" it carries this oracle's FP64 eikonal tables of the survey's gridded model (built once
    per model and location set, then cached) or the tables given as ``s.oracle_tables``."""
    d = _Desc(s.dim, s.nx, s.ny if s.dim == 3 else 1, s.nz, s.ox, s.oy, s.oz, s.dx, s.dy,
              s.dz, s.n_bins, s.bin_width, {"const": 0, "linear": 1, "table": 2, "pstm": 3, "grid": 4}[s.vel],
              s.v0, s.k, {"one": 0, "obliq": 1, "ta": 2}[s.weight], s.r0, s.aperture, s.nt, s.t0, s.dt,
              float(getattr(s, "table_spacing", 25.0)), float(getattr(s, "taper", 0.0)))
    d.aa_spacing = float(getattr(s, "aa_spacing", 0.0))
    if s.vel == "grid":
        g = getattr(s, "oracle_tables", None)
        if g is None:
            g = grid_tables(s)
        d.gtab, d.gloc = _ptr(g.T), _ptr(g.loc)
        d.gnloc, d.gnx, d.gnz = g.loc.size, g.T.shape[1], g.T.shape[2]
        d.gox, d.gh = g.ox, g.h
        d._keep = g   # the arrays the pointers refer to
    return d


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _hdr(s):
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return f(s.sx), f(s.sy), f(s.rx), f(s.ry)


def set_mutation(m: int) -> None:
    """Plant a deliberate mistake in the oracle (tests of the pins only); 0 restores it."""
    lib().ko_set_mutation(int(m))


def set_threads(n: int) -> None:
    lib().ko_set_threads(int(n))


def max_threads() -> int:
    return int(lib().ko_max_threads())


def bins(s) -> np.ndarray:
    sx, sy, rx, ry = _hdr(s)
    out = np.empty(s.ntr, dtype=np.int32)
    lib().ko_bins(ctypes.byref(desc(s)), s.ntr, _ptr(sx), _ptr(sy), _ptr(rx), _ptr(ry), _ptr(out))
    return out


def traveltime(s, R, z, grad: bool = False):
    """One-way time (and d/dv0, d/dk) from a surface point to distance R, depth z (vel "pstm":
    R is the horizontal distance and z the two-way vertical time; no derivatives)."""
    R = np.asarray(R, dtype=np.float64)
    z = np.ascontiguousarray(np.broadcast_to(np.asarray(z, dtype=np.float64), R.shape)).ravel()
    R = np.ascontiguousarray(R).ravel()
    T = np.empty_like(R)
    gv = np.empty_like(R) if grad else None
    gk = np.empty_like(R) if grad else None
    lib().ko_traveltime(ctypes.byref(desc(s)), R.size, _ptr(R), _ptr(z), _ptr(T), _ptr(gv), _ptr(gk))
    return (T, gv, gk) if grad else T


def ta_weight(s, pts) -> np.ndarray:
    """True-amplitude weight (weight "ta") at rows (x, y, z, sx, sy, rx, ry) of ``pts``."""
    p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 7)
    W = np.empty(p.shape[0], dtype=np.float64)
    lib().ko_ta_weight(ctypes.byref(desc(s)), p.shape[0], _ptr(p), _ptr(W))
    return W


def aa_weight(s, pts) -> np.ndarray:
    """Anti-aliasing weight (constant velocity or v0 + k z, ``s.aa_spacing`` > 0) at rows
    (x, y, z, sx, sy, rx, ry) of ``pts``."""
    p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 7)
    W = np.empty(p.shape[0], dtype=np.float64)
    lib().ko_aa_weight(ctypes.byref(desc(s)), p.shape[0], _ptr(p), _ptr(W))
    return W


def table_traveltime(s, h, z) -> np.ndarray:
    """Traveltime of the radial table (vel "table"): bilinear in (horizontal distance, depth)
    between closed-form node values."""
    h = np.ascontiguousarray(h, dtype=np.float64).ravel()
    z = np.ascontiguousarray(np.broadcast_to(np.asarray(z, dtype=np.float64), h.shape)).ravel()
    T = np.empty_like(h)
    lib().ko_table_traveltime(ctypes.byref(desc(s)), h.size, _ptr(h), _ptr(z), _ptr(T))
    return T


def migrate(s, traces) -> np.ndarray:
    """Eq. 1 for every image sample: returns float64 [n_bins, ny, nx, nz]."""
    sx, sy, rx, ry = _hdr(s)
    d = np.ascontiguousarray(traces, dtype=np.float64).reshape(s.ntr, s.nt)
    img = np.empty(s.image_shape, dtype=np.float64)
    rc = lib().ko_migrate(ctypes.byref(desc(s)), s.ntr, _ptr(sx), _ptr(sy), _ptr(rx), _ptr(ry),
                          _ptr(d), _ptr(img))
    assert rc == 0
    return img


def migrate_points(s, traces, flat_idx, return_count: bool = False):
    """Eq. 1 at selected image samples (flat indices into [n_bins, ny, nx, nz]); with
    ``return_count`` also the number of (point, in-aperture trace) pairs visited."""
    sx, sy, rx, ry = _hdr(s)
    d = np.ascontiguousarray(traces, dtype=np.float64).reshape(s.ntr, s.nt)
    p = np.ascontiguousarray(flat_idx, dtype=np.int64)
    out = np.empty(p.size, dtype=np.float64)
    n = ctypes.c_longlong(0)
    rc = lib().ko_migrate_points(ctypes.byref(desc(s)), s.ntr, _ptr(sx), _ptr(sy), _ptr(rx),
                                 _ptr(ry), _ptr(d), p.size, _ptr(p), _ptr(out), ctypes.byref(n))
    assert rc == 0
    return (out, int(n.value)) if return_count else out


def demigrate(s, image) -> np.ndarray:
    """The transpose of ``migrate``: returns float64 traces [ntr, nt]."""
    sx, sy, rx, ry = _hdr(s)
    m = np.ascontiguousarray(image, dtype=np.float64).reshape(s.image_shape)
    out = np.empty((s.ntr, s.nt), dtype=np.float64)
    rc = lib().ko_demigrate(ctypes.byref(desc(s)), s.ntr, _ptr(sx), _ptr(sy), _ptr(rx), _ptr(ry),
                            _ptr(m), _ptr(out))
    assert rc == 0
    return out


def vgrad(s, image, traces, return_abs: bool = False):
    """[dB/dv0, dB/dk] of B(m, D) = <m, migrate(D)>; with ``return_abs`` also the sums of
    the absolute values of the terms (the summation's condition scale)."""
    sx, sy, rx, ry = _hdr(s)
    m = np.ascontiguousarray(image, dtype=np.float64).reshape(s.image_shape)
    d = np.ascontiguousarray(traces, dtype=np.float64).reshape(s.ntr, s.nt)
    out = np.empty(2, dtype=np.float64)
    ab = np.empty(2, dtype=np.float64)
    rc = lib().ko_vgrad(ctypes.byref(desc(s)), s.ntr, _ptr(sx), _ptr(sy), _ptr(rx), _ptr(ry),
                        _ptr(m), _ptr(d), _ptr(out), _ptr(ab))
    assert rc == 0
    return (out, ab) if return_abs else out


def count(s) -> int:
    """Eq. 2 work count: (image point, in-aperture trace) pairs with a valid offset bin."""
    sx, sy, rx, ry = _hdr(s)
    return int(lib().ko_count(ctypes.byref(desc(s)), s.ntr, _ptr(sx), _ptr(sy), _ptr(rx), _ptr(ry)))


def arrival_times(points, s, trace_idx) -> np.ndarray:
    """Two-way times source -> scatterer -> receiver (for trace synthesis), float64
    [n_points, len(trace_idx)], using this oracle's traveltime."""
    pts = np.asarray(points, dtype=np.float64)
    j = np.asarray(trace_idx)
    px, py, pz = (np.ascontiguousarray(pts[:, i]) for i in range(3))
    sx, sy, rx, ry = (np.ascontiguousarray(np.asarray(a)[j], dtype=np.float32)
                      for a in (s.sx, s.sy, s.rx, s.ry))
    out = np.empty((pts.shape[0], j.size), dtype=np.float64)
    lib().ko_arrivals(ctypes.byref(desc(s)), pts.shape[0], _ptr(px), _ptr(py), _ptr(pz), j.size,
                      _ptr(sx), _ptr(sy), _ptr(rx), _ptr(ry), _ptr(out))
    return out


# ------------------------------------------------------------------ gridded model v(x, z)

MAX_ROUNDS = 64
# A round of sweeps whose largest decrease is at most this many seconds ends the iteration: the
# corrections shrink by about two orders of magnitude from round to round, so what remains is a
# few 1e-9 s, below the resolution of an FP32 table (about 1e-7 s at 1 s).
TOL = 1e-7


def eikonal(v, ox: float, h: float, xs: float, max_rounds: int = MAX_ROUNDS, tol: float = TOL):
    """First-arrival times from the surface point (xs, 0) on the node grid (ox + i h, j h) of the
    model v [nx, nz] (m/s): the factored fast-sweeping solution (kh_oracle.c, ko_eikonal).
    Returns (T float64 [nx, nz], rounds; -1 if it did not settle within max_rounds)."""
    v = np.ascontiguousarray(v, dtype=np.float32)
    T = np.empty(v.shape, dtype=np.float64)
    r = lib().ko_eikonal(v.shape[0], v.shape[1], float(ox), float(h), _ptr(v), float(xs), int(max_rounds),
                         float(tol), _ptr(T))
    return T, int(r)


class GridTables:
    """FP64 tables of one gridded model: T [nloc, nx, nz], the locations (float32, increasing),
    the grid origin and spacing, and the fast-sweeping rounds per location."""

    def __init__(self, T, loc, ox, h, rounds):
        self.T, self.loc, self.ox, self.h, self.rounds = T, loc, float(ox), float(h), rounds


def locations(s) -> np.ndarray:
    """The survey's distinct surface positions (source and receiver x), increasing, float32."""
    return np.unique(np.concatenate([np.asarray(s.sx, np.float32), np.asarray(s.rx, np.float32)]))


_grid_cache = {}


def grid_tables(s, max_rounds: int = MAX_ROUNDS, tol: float = TOL) -> GridTables:
    """Tables of the survey's model ``s.grid_v`` on (``s.grid_ox`` + i ``s.grid_h``, j ``s.grid_h``)
    for every distinct surface position of its traces."""
    v = np.ascontiguousarray(s.grid_v, dtype=np.float32)
    loc = locations(s)
    key = (hash(v.tobytes()), v.shape, float(s.grid_ox), float(s.grid_h), hash(loc.tobytes()), max_rounds, tol)
    if key in _grid_cache:
        return _grid_cache[key]
    T = np.empty((loc.size,) + v.shape, dtype=np.float64)
    rounds = np.empty(loc.size, dtype=np.int32)
    bad = lib().ko_grid_tables(v.shape[0], v.shape[1], float(s.grid_ox), float(s.grid_h), _ptr(v), loc.size,
                               _ptr(loc), int(max_rounds), float(tol), _ptr(T), _ptr(rounds))
    if bad:
        raise RuntimeError(f"eikonal tables: {bad} locations did not settle in {max_rounds} rounds")
    g = GridTables(T, loc, s.grid_ox, s.grid_h, rounds)
    if len(_grid_cache) >= 4:
        _grid_cache.pop(next(iter(_grid_cache)))
    _grid_cache[key] = g
    return g


def grid_traveltime(s, loc_index: int, x, z) -> np.ndarray:
    """Table ``loc_index`` of the survey's model read at (x, z) by the bilinear interpolation of
    the migration."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    z = np.ascontiguousarray(np.broadcast_to(np.asarray(z, dtype=np.float64), x.shape)).ravel()
    T = np.empty_like(x)
    lib().ko_grid_traveltime(ctypes.byref(desc(s)), int(loc_index), x.size, _ptr(x), _ptr(z), _ptr(T))
    return T


def cgls(s, data, n_iter: int, m0=None):
    """Textbook CGLS for min_m ||A m - d||^2 with A = demigrate, A^T = migrate, in FP64.

    Returns (m, residual norms ||r_i||, normal-equation residual norms ||A^T r_i||)."""
    d = np.asarray(data, dtype=np.float64)
    m = np.zeros(s.image_shape) if m0 is None else np.array(m0, dtype=np.float64)
    r = d - demigrate(s, m) if m0 is not None else d.copy()
    g = migrate(s, r)
    p = g.copy()
    gamma = float(np.vdot(g, g))
    rn, gn = [float(np.linalg.norm(r))], [float(np.sqrt(gamma))]
    for _ in range(n_iter):
        q = demigrate(s, p)
        qq = float(np.vdot(q, q))
        if qq == 0.0 or gamma == 0.0:
            break
        alpha = gamma / qq
        m += alpha * p
        r -= alpha * q
        g = migrate(s, r)
        gamma_new = float(np.vdot(g, g))
        p = g + (gamma_new / gamma) * p
        gamma = gamma_new
        rn.append(float(np.linalg.norm(r)))
        gn.append(float(np.sqrt(gamma)))
    return m, np.array(rn), np.array(gn)


# ------------------------------------------------------------------ velocity analysis (FP64)
# Sec. 2: migration with an estimate of the velocity gives a set of redundant images (one per
# offset bin here); differences in the position of the same reflector between them measure the
# error of the velocity model, which is corrected and the data migrated again; once they agree
# the images are stacked.  The measure taken here is the normalised variance of the weighted
# offset images across the bins (one minus the semblance of the stack):
#     V = sum_b ||w_b I_b - m||^2 / sum_b ||w_b I_b||^2,   m = (1/N) sum_b w_b I_b,
# over the N bins that hold traces, with w_b = 1 / (traces in bin b).  Its image gradient is
#     dV/dI_b = (2 w_b / B) ((w_b I_b - m) - V w_b I_b),   B = sum_b ||w_b I_b||^2,
# and its (v0, k) gradient is the velocity gradient of <dV/dI, L(v0, k) D> (ko_vgrad).

_va_mutation = 0   # deliberate mistakes for the tests of the pins only; 0 = as written


def bin_weights(s) -> np.ndarray:
    """w_b = 1 / (traces in bin b), 0 for bins without traces."""
    b = bins(s)
    n = np.bincount(b[b >= 0], minlength=s.n_bins).astype(np.float64)
    return np.where(n > 0, 1.0 / np.maximum(n, 1.0), 0.0)


def semblance(image, weights):
    """(V, dV/dI) of offset images [n_bins, ...] with bin weights w_b, FP64."""
    img = np.asarray(image, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    used = w > 0
    if _va_mutation == 1:
        w = np.where(used, 1.0, 0.0)                     # weights dropped
    shape = (-1,) + (1,) * (img.ndim - 1)
    wi = img * w.reshape(shape)
    N = int(used.sum())
    m = wi[used].sum(axis=0) / N
    if _va_mutation == 2:
        m = wi[used].sum(axis=0) / (N - 1)               # wrong bin count in the mean
    dev = np.where(used.reshape(shape), wi - m, 0.0)
    D = float(np.sum(dev * dev))
    B = float(np.sum(wi * wi))
    V = D / B
    G = (2.0 * w.reshape(shape) / B) * (dev - V * wi)
    if _va_mutation == 3:
        G = (2.0 * w.reshape(shape) / B) * (dev + V * wi)   # sign of the quotient term
    return V, G


def velocity_objective(s, traces, v0, k):
    """(V, dV/dv0, dV/dk) of the offset images L(v0, k) D: migrate, semblance, and the velocity
    gradient of <dV/dI, L(v0, k) D>."""
    sv_ = s.replace(v0=float(v0), k=float(k))
    img = migrate(sv_, traces)
    V, G = semblance(img, bin_weights(s))
    g = vgrad(sv_, G, traces)
    return V, float(g[0]), float(g[1])


def velocity_analysis(s, traces, v0, k, n_iter: int = 30, scale=(100.0, 0.1), tol: float = 1e-12):
    """Minimises V over (v0, k) from a start: the textbook BFGS iteration on the scaled
    parameters (v0 / scale[0], k / scale[1]) with an Armijo backtracking line search.
    Returns (v0, k, history of (v0, k, V))."""
    sc = np.asarray(scale, dtype=np.float64)
    th = np.array([v0, k], dtype=np.float64)
    V, g0, g1 = velocity_objective(s, traces, *th)
    g = np.array([g0, g1]) * sc
    H = np.eye(2)
    hist = [(th[0], th[1], V)]
    for _ in range(n_iter):
        p = -H @ g
        a = 1.0
        while True:
            tn = th + a * p * sc
            Vn, h0, h1 = velocity_objective(s, traces, *tn)
            if Vn <= V + 1e-4 * a * float(g @ p) or a < 1e-3:
                break
            a *= 0.5
        gn = np.array([h0, h1]) * sc
        step, y = a * p, gn - g
        if float(step @ y) > 1e-300:
            r = 1.0 / float(y @ step)
            I = np.eye(2)
            H = (I - r * np.outer(step, y)) @ H @ (I - r * np.outer(y, step)) + r * np.outer(step, step)
        done = abs(V - Vn) <= tol * max(abs(V), 1e-300)
        th, V, g = tn, Vn, gn
        hist.append((th[0], th[1], V))
        if done:
            break
    return float(th[0]), float(th[1]), hist
