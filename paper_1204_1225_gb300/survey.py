"""Seeded synthetic surveys shaped like the workloads of Sec. 2-3 of the paper.

This module holds geometry, random numbers and wavelet synthesis only: no part of the
migration operator.  Arrival times of the synthetic events are supplied by the caller
(``arrival_fn``), so the same survey can be synthesised from either side of a parity
test without this module computing a traveltime itself.

Survey facts it follows (Sec. 2): each experiment is one surface shot recorded by a
collection of surface receivers; a trace is a receiver recording sampled every few ms;
a survey has N = K*L traces for K shots and L receivers (Sec. 4, Forward PKTM, item 1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional, List

import numpy as np

BASE_SEED = 1204


@dataclasses.dataclass
class Survey:
    """Image grid, offset bins, velocity model, weight, trace sampling and trace headers.

    Image layout is ``[n_bins][ny][nx][nz]`` (z fastest); traces are ``[ntr][nt]``.
    ``vel`` is ``"const"``, ``"linear"`` (v(z) = v0 + k z, z from the surface) or ``"table"``
    (the same v0 + k z model read from a radial traveltime table with node spacing
    ``table_spacing``);
    ``weight`` is ``"one"`` or ``"obliq"``; ``aperture <= 0`` means full aperture; ``taper`` is the
    fraction of the aperture over which the weight falls to 0 (raised cosine; 0: a hard mask);
    ``vel == "pstm"`` reads the depth axis as two-way vertical time (time migration);
    ``vel == "grid"`` (2D) takes each leg from the first-arrival time table of its surface point in
    the gridded model ``grid_v``.
    """

    dim: int
    nx: int
    ny: int
    nz: int
    ox: float
    oy: float
    oz: float
    dx: float
    dy: float
    dz: float
    n_bins: int
    bin_width: float
    vel: str
    v0: float
    k: float
    weight: str
    r0: float
    aperture: float
    nt: int
    t0: float
    dt: float
    sx: np.ndarray
    sy: np.ndarray
    rx: np.ndarray
    ry: np.ndarray
    name: str = ""
    table_spacing: float = 25.0
    taper: float = 0.0
    # vel == "grid" (2D): the model v(x, z) sampled on the square node grid
    # (grid_ox + i grid_h, j grid_h), [nx][nz] float32 m/s, row 0 at the surface
    grid_v: Optional[np.ndarray] = None
    grid_ox: float = 0.0
    grid_h: float = 0.0
    # constant velocity: trace spacing (m) of the operator anti-aliasing; 0 = off
    aa_spacing: float = 0.0

    @property
    def ntr(self) -> int:
        return int(self.sx.shape[0])

    @property
    def image_shape(self):
        return (self.n_bins, self.ny, self.nx, self.nz)

    def replace(self, **kw) -> "Survey":
        return dataclasses.replace(self, **kw)

    def subset(self, idx) -> "Survey":
        idx = np.asarray(idx)
        return self.replace(sx=self.sx[idx], sy=self.sy[idx], rx=self.rx[idx], ry=self.ry[idx])


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


# --------------------------------------------------------------------------------------
# Geometries
# --------------------------------------------------------------------------------------

def survey_2d_const(seed: int = BASE_SEED) -> Survey:
    """2D line, constant velocity 2000 m/s: 16 shots every 80 m, each with a split spread
    of 64 receivers at 10 m (1024 traces, offsets 5-315 m); 512 samples at 4 ms; image
    128 (x) x 128 (z) at 10 m; 8 offset bins of 40 m; W = 1; full aperture."""
    del seed
    i = np.arange(16)
    j = np.arange(64)
    xs = 40.0 + 80.0 * i
    sx = np.repeat(xs, 64)
    rx = sx + np.tile((j - 31.5) * 10.0, 16)
    z = np.zeros_like(sx)
    return Survey(dim=2, nx=128, ny=1, nz=128, ox=0.0, oy=0.0, oz=0.0, dx=10.0, dy=10.0, dz=10.0,
                  n_bins=8, bin_width=40.0, vel="const", v0=2000.0, k=0.0, weight="one", r0=1000.0,
                  aperture=0.0, nt=512, t0=0.0, dt=0.004, sx=_f32(sx), sy=_f32(z), rx=_f32(rx),
                  ry=_f32(z), name="2d-const-1024tr-128x128")


def survey_3d_gradient(ntr: int = 100_000, n: int = 256) -> Survey:
    """3D survey, v(z) = 1500 + 0.5 z: a 10 x 10 shot grid at 50 m centred on
    (1600, 1600) m, each shot recorded by an 8 (y) x 128 (x) receiver patch at 25 m
    centred on the shot; traces in shot-raster order, the first ``ntr`` kept; 1500
    samples at 4 ms; image n^3 at 12.5 m (256^3 at full size); 16 offset bins of 100 m;
    2 km aperture; obliquity x spreading weight."""
    g = np.arange(10)
    shot_x = 1600.0 + (g - 4.5) * 50.0
    sy_s, sx_s = np.meshgrid(shot_x, shot_x, indexing="ij")
    a = np.arange(128)
    b = np.arange(8)
    pb, pa = np.meshgrid(b, a, indexing="ij")
    offx = ((pa - 63.5) * 25.0).ravel()
    offy = ((pb - 3.5) * 25.0).ravel()
    sx = np.repeat(sx_s.ravel(), offx.size)
    sy = np.repeat(sy_s.ravel(), offx.size)
    rx = sx + np.tile(offx, 100)
    ry = sy + np.tile(offy, 100)
    sl = slice(0, ntr)
    h = 12.5 * 256 / n
    return Survey(dim=3, nx=n, ny=n, nz=n, ox=0.0, oy=0.0, oz=0.0, dx=h, dy=h, dz=h,
                  n_bins=16, bin_width=100.0, vel="linear", v0=1500.0, k=0.5, weight="obliq",
                  r0=1000.0, aperture=2000.0, nt=1500, t0=0.0, dt=0.004, sx=_f32(sx[sl]),
                  sy=_f32(sy[sl]), rx=_f32(rx[sl]), ry=_f32(ry[sl]),
                  name=f"3d-vz-{ntr}tr-{n}cube")


def survey_25d_velan(nx: int = 128, nz: int = 100, h: float = 15.0, nt: int = 800, n_shots: int = 48,
                     n_rec: int = 96, n_bins: int = 4, aperture: float = 400.0, v0: float = 1800.0,
                     k: float = 0.6) -> Survey:
    """A shorter 2.5D line of the least-squares geometry for velocity analysis: shots every 25 m
    and split spreads of receivers at 12.5 m (offsets up to ~600 m), centred over an nx x nz
    image at h m; v(z) = v0 + k z (the 2.5D line's model by default); W = 1; a 400 m aperture;
    4 offset bins of 150 m."""
    xs = 25.0 * np.arange(n_shots)
    xs = xs + 0.5 * ((nx - 1) * h - xs[-1])
    sx = np.repeat(xs, n_rec)
    rx = sx + np.tile((np.arange(n_rec) - (n_rec - 1) / 2.0) * 12.5, n_shots)
    z = np.zeros_like(sx)
    wmax = float(np.max(np.abs(rx - sx)))
    return Survey(dim=2, nx=nx, ny=1, nz=nz, ox=0.0, oy=0.0, oz=0.0, dx=h, dy=h, dz=h,
                  n_bins=n_bins, bin_width=wmax * 1.0001 / n_bins, vel="linear", v0=v0, k=k,
                  weight="one", r0=1000.0, aperture=aperture, nt=nt, t0=0.0, dt=0.004,
                  sx=_f32(sx), sy=_f32(z), rx=_f32(rx), ry=_f32(z),
                  name=f"25d-velan-{sx.size}tr-{nx}x{nz}")


def diffractors_2d(rng: np.random.Generator, survey: Survey, n: int = 12, zr=(300.0, 1300.0),
                   amp: float = 1.0) -> np.ndarray:
    """Point diffractors uniform over the middle half of the line and a depth range (y = 0)."""
    w = (survey.nx - 1) * survey.dx
    x = rng.uniform(survey.ox + 0.25 * w, survey.ox + 0.75 * w, n)
    z = rng.uniform(zr[0], zr[1], n)
    return np.stack([x, np.zeros(n), z, np.full(n, amp)], axis=1)


def survey_batch_3d(n_jobs: int = 64, n_range=(64, 192), ntr_range=(1000, 50_000),
                    nt_range=(750, 2000), seed: int = BASE_SEED, h: float = 10.0) -> List[Survey]:
    """Batch of independent 3D migrations of uneven size, each with the physics of the 2D
    constant-velocity survey: v = 2000 m/s, W = 1, full aperture, 8 offset bins, 4 ms
    sampling.  Job j draws, from a generator seeded with seed + j, an n^3 image at ``h`` m with
    n ~ U{n_range}, N_tr ~ U{ntr_range} traces and nt ~ U{nt_range} samples; sources and
    receivers are uniform over the image's surface footprint [0, n h)^2, and the bins split
    [0, largest offset] into 8."""
    out = []
    for j in range(n_jobs):
        rng = np.random.default_rng(seed + j)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        ntr = int(rng.integers(ntr_range[0], ntr_range[1] + 1))
        nt = int(rng.integers(nt_range[0], nt_range[1] + 1))
        w = n * h
        sx, sy, rx, ry = (_f32(rng.uniform(0.0, w, ntr)) for _ in range(4))
        xmax = float(np.max(np.hypot(sx.astype(np.float64) - rx, sy.astype(np.float64) - ry)))
        out.append(Survey(dim=3, nx=n, ny=n, nz=n, ox=0.0, oy=0.0, oz=0.0, dx=h, dy=h, dz=h,
                          n_bins=8, bin_width=xmax / 8.0 * (1.0 + 1e-9), vel="const", v0=2000.0,
                          k=0.0, weight="one", r0=1000.0, aperture=0.0, nt=nt, t0=0.0, dt=0.004,
                          sx=sx, sy=sy, rx=rx, ry=ry, name=f"3d-const-{ntr}tr-{n}cube-{nt}nt"))
    return out


def survey_25d_lsm(nx: int = 512, nz: int = 400, nt: int = 2000, n_shots: int = 100,
                   n_rec: int = 200) -> Survey:
    """2.5D line for least-squares migration: 100 shots every 25 m, 200 receivers at
    12.5 m in a split spread (20 000 traces); 2000 samples at 4 ms; image 512 x 400 at
    5 m; 8 offset bins of 160 m; v(z) = 1800 + 0.6 z; W = 1; full aperture."""
    xs = 25.0 * np.arange(n_shots)
    sx = np.repeat(xs, n_rec)
    rx = sx + np.tile((np.arange(n_rec) - (n_rec - 1) / 2.0) * 12.5, n_shots)
    z = np.zeros_like(sx)
    return Survey(dim=2, nx=nx, ny=1, nz=nz, ox=0.0, oy=0.0, oz=0.0, dx=5.0, dy=5.0, dz=5.0,
                  n_bins=8, bin_width=160.0, vel="linear", v0=1800.0, k=0.6, weight="one",
                  r0=1000.0, aperture=0.0, nt=nt, t0=0.0, dt=0.004, sx=_f32(sx), sy=_f32(z),
                  rx=_f32(rx), ry=_f32(z), name=f"25d-vz-{sx.size}tr-{nx}x{nz}")


def survey_25d_vxz(m: int = 4) -> Survey:
    """The 2.5D line of ``survey_25d_lsm`` (20 000 traces, 512 x 400 image at 5 m) over a laterally
    varying model: v = 1800 + 0.6 z with a Gaussian low-velocity lens (-300 m/s, radius 250 m) at
    (1280 m, 800 m), on 20 m nodes (m = 4) covering every shot and receiver."""
    s = vxz_model(survey_25d_lsm(), m, lens_dv=-300.0, lens_xz=(1280.0, 800.0), lens_r=250.0)
    return s.replace(name=f"25d-vxz-{s.ntr}tr-{s.nx}x{s.nz}")


def grid_layout(survey: Survey, m: int, margin_nodes: int = 1):
    """Node grid for a gridded model of a 2D survey: square cells of side h = m dz (m in 1, 2, 4),
    row 0 at the surface, columns covering the image and every source and receiver with
    ``margin_nodes`` spare nodes each side, and rows down to one node below the image depths
    rounded up to a multiple of 16 samples (the depths a migration tile may evaluate).
    Returns (nx, nz, ox, h)."""
    h = m * survey.dz
    zoff = int(round(survey.oz / h))
    xs = np.concatenate([np.asarray(survey.sx, np.float64), np.asarray(survey.rx, np.float64),
                         [survey.ox, survey.ox + (survey.nx - 1) * survey.dx]])
    i0 = math.floor(float(xs.min()) / h) - margin_nodes
    i1 = math.ceil(float(xs.max()) / h) + margin_nodes
    nz = zoff + (-(-survey.nz // 16) * 16) // m + 1
    return i1 - i0 + 1, nz, i0 * h, h


def vxz_model(survey: Survey, m: int, lens_dv: float = -300.0, lens_xz=None, lens_r: float = 250.0,
              lateral: float = 0.0) -> Survey:
    """The survey with vel "grid" and a laterally varying model on ``grid_layout``'s nodes:
    v = v0 + k z + lateral (x - x_c) + lens_dv exp(-|p - p_lens|^2 / (2 lens_r^2)), a Gaussian lens
    (low velocity for lens_dv < 0) centred at ``lens_xz`` (default: the image centre, 40 % down)
    in the gradient model of the survey (x_c the image centre)."""
    nx, nz, ox, h = grid_layout(survey, m)
    xc = survey.ox + 0.5 * (survey.nx - 1) * survey.dx
    if lens_xz is None:
        lens_xz = (xc, survey.oz + 0.4 * (survey.nz - 1) * survey.dz)
    x = ox + np.arange(nx, dtype=np.float64) * h
    z = np.arange(nz, dtype=np.float64) * h
    X, Z = np.meshgrid(x, z, indexing="ij")
    v = (survey.v0 + survey.k * Z + lateral * (X - xc)
         + lens_dv * np.exp(-((X - lens_xz[0]) ** 2 + (Z - lens_xz[1]) ** 2) / (2.0 * lens_r ** 2)))
    return survey.replace(vel="grid", grid_v=_f32(v), grid_ox=float(ox), grid_h=float(h))


def survey_random(rng: np.random.Generator, dim: int, ntr: int, nx: int, ny: int, nz: int,
                  nt: int, vel: str = "const", weight: str = "one", aperture: float = 0.0,
                  n_bins: int = 4, h: float = 10.0, dt: float = 0.004, t0: float = 0.0,
                  v0: float = 2000.0, k: float = 0.0) -> Survey:
    """Small randomised survey over the image footprint (used for edge cases and tiny
    grids): sources and receivers uniform over the footprint, offsets binned uniformly
    up to the largest offset drawn."""
    wx, wy = nx * h, (ny * h if dim == 3 else 0.0)
    sx = rng.uniform(-0.1 * wx, 1.1 * wx, ntr)
    rx = rng.uniform(-0.1 * wx, 1.1 * wx, ntr)
    if dim == 3:
        sy = rng.uniform(-0.1 * wy, 1.1 * wy, ntr)
        ry = rng.uniform(-0.1 * wy, 1.1 * wy, ntr)
    else:
        sy = np.zeros(ntr)
        ry = np.zeros(ntr)
    sx, sy, rx, ry = _f32(sx), _f32(sy), _f32(rx), _f32(ry)
    off = np.hypot(sx.astype(np.float64) - rx, sy.astype(np.float64) - ry)
    xmax = float(np.max(off)) * 1.0001 + 1.0
    return Survey(dim=dim, nx=nx, ny=ny if dim == 3 else 1, nz=nz, ox=0.0, oy=0.0, oz=0.0,
                  dx=h, dy=h, dz=h, n_bins=n_bins, bin_width=xmax / n_bins, vel=vel, v0=v0,
                  k=k, weight=weight, r0=1000.0, aperture=aperture, nt=nt, t0=t0, dt=dt,
                  sx=sx, sy=sy, rx=rx, ry=ry, name=f"random-{dim}d-{ntr}tr")


# --------------------------------------------------------------------------------------
# Subsurface models: point scatterers and reflector sheets (x, y, z, amplitude)
# --------------------------------------------------------------------------------------

def point_scatterers_2d(rng: np.random.Generator, n: int = 3, xr=(100.0, 1180.0),
                        zr=(200.0, 1200.0), snap: float = 10.0, amp: float = 1.0) -> np.ndarray:
    x = np.round(rng.uniform(*xr, n) / snap) * snap
    z = np.round(rng.uniform(*zr, n) / snap) * snap
    return np.stack([x, np.zeros(n), z, np.full(n, amp)], axis=1)


def reflectors_3d(rng: np.random.Generator, survey: Survey, n_planes: int = 4,
                  n_diffractors: int = 40, spacing: float = 12.5, sheet_amp: float = 0.1,
                  max_dip_deg: float = 20.0, z0_range=(600.0, 2600.0)) -> np.ndarray:
    """Dipping planes z = z0 + a (x - xc) + b (y - yc) sampled as scatterer sheets every
    ``spacing`` m (amplitude scaled by (spacing/12.5)^2 so the reflectivity per unit
    area does not depend on the sampling), plus point diffractors below 300 m."""
    xc = survey.ox + 0.5 * (survey.nx - 1) * survey.dx
    yc = survey.oy + 0.5 * (survey.ny - 1) * survey.dy
    wx = (survey.nx - 1) * survey.dx
    wy = (survey.ny - 1) * survey.dy
    zmax = survey.oz + (survey.nz - 1) * survey.dz
    pts = []
    gx = np.arange(survey.ox, survey.ox + wx + 1e-9, spacing)
    gy = np.arange(survey.oy, survey.oy + wy + 1e-9, spacing)
    GY, GX = np.meshgrid(gy, gx, indexing="ij")
    amp = sheet_amp * (spacing / 12.5) ** 2
    for _ in range(n_planes):
        z0 = rng.uniform(*z0_range)
        dip = math.radians(rng.uniform(0.0, max_dip_deg))
        az = rng.uniform(0.0, 2.0 * math.pi)
        a, b = math.tan(dip) * math.cos(az), math.tan(dip) * math.sin(az)
        Z = z0 + a * (GX - xc) + b * (GY - yc)
        keep = (Z > 0.0) & (Z < zmax)
        pts.append(np.stack([GX[keep], GY[keep], Z[keep], np.full(int(keep.sum()), amp)], 1))
    dx_ = rng.uniform(survey.ox, survey.ox + wx, n_diffractors)
    dy_ = rng.uniform(survey.oy, survey.oy + wy, n_diffractors)
    dz_ = rng.uniform(300.0, zmax, n_diffractors)
    pts.append(np.stack([dx_, dy_, dz_, np.ones(n_diffractors)], 1))
    return np.concatenate(pts, 0)


def reflectors_2d(rng: np.random.Generator, survey: Survey, n_lines: int = 3,
                  n_diffractors: int = 10, spacing: float = 5.0, line_amp: float = 0.1,
                  max_dip_deg: float = 15.0) -> np.ndarray:
    """Flat and dipping reflector lines z = z0 + a (x - xc) sampled every ``spacing`` m, plus
    point diffractors (2D sections; y = 0)."""
    xc = survey.ox + 0.5 * (survey.nx - 1) * survey.dx
    wx = (survey.nx - 1) * survey.dx
    zmax = survey.oz + (survey.nz - 1) * survey.dz
    gx = np.arange(survey.ox, survey.ox + wx + 1e-9, spacing)
    pts = []
    amp = line_amp * spacing / 5.0
    for i in range(n_lines):
        z0 = rng.uniform(0.2 * zmax, 0.9 * zmax)
        a = 0.0 if i == 0 else math.tan(math.radians(rng.uniform(-max_dip_deg, max_dip_deg)))
        Z = z0 + a * (gx - xc)
        keep = (Z > 0.0) & (Z < zmax)
        pts.append(np.stack([gx[keep], np.zeros(int(keep.sum())), Z[keep],
                             np.full(int(keep.sum()), amp)], 1))
    pts.append(np.stack([rng.uniform(survey.ox, survey.ox + wx, n_diffractors), np.zeros(n_diffractors),
                         rng.uniform(0.1 * zmax, zmax, n_diffractors), np.ones(n_diffractors)], 1))
    return np.concatenate(pts, 0)


# --------------------------------------------------------------------------------------
# Trace synthesis
# --------------------------------------------------------------------------------------

def ricker(t, f: float):
    """Ricker wavelet with peak 1 at t = 0: (1 - 2 pi^2 f^2 t^2) exp(-pi^2 f^2 t^2)."""
    a = (math.pi * f * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


ArrivalFn = Callable[[np.ndarray, Survey, np.ndarray], np.ndarray]


def synthesize(survey: Survey, scatterers: np.ndarray, arrival_fn: ArrivalFn, freq: float,
               noise_sigma: float = 0.0, seed: int = BASE_SEED, device: str = "cpu",
               chunk: int = 1 << 22, dtype=np.float32):
    """Traces D_j(t) = sum_s a_s r(t - t_js) + noise, with t_js = arrival_fn(...).

    ``arrival_fn(points[n,3], survey, trace_idx[m]) -> times[n, m]`` (seconds, float64)
    gives the two-way time from the source of each trace, via each scatterer, to its
    receiver.  The wavelet is evaluated exactly at every sample within 1.6/f of the
    arrival.  ``noise_sigma`` is the standard deviation of white Gaussian noise.
    Returns a torch tensor [ntr, nt] on ``device`` (float32 by default).
    """
    import torch

    ntr, nt = survey.ntr, survey.nt
    out = torch.zeros(ntr * nt, dtype=torch.float64, device=device)
    half = int(math.ceil(1.6 / freq / survey.dt)) + 1
    offs = torch.arange(-half, half + 1, device=device, dtype=torch.int64)
    pts = np.asarray(scatterers[:, :3], dtype=np.float64)
    amp_all = torch.as_tensor(np.asarray(scatterers[:, 3], dtype=np.float64), device=device)
    ns = pts.shape[0]
    per = max(1, chunk // max(ns, 1))
    for j0 in range(0, ntr, per):
        jj = np.arange(j0, min(ntr, j0 + per))
        t = arrival_fn(pts, survey, jj)
        t = torch.as_tensor(np.asarray(t, dtype=np.float64) if not torch.is_tensor(t) else t,
                            device=device, dtype=torch.float64)            # [ns, m]
        tau = (t - survey.t0) / survey.dt
        i0 = torch.floor(tau).to(torch.int64)
        idx = i0.unsqueeze(-1) + offs                                       # [ns, m, K]
        tt = idx.to(torch.float64) * survey.dt + survey.t0 - t.unsqueeze(-1)
        a = (math.pi * freq * tt) ** 2
        w = (1.0 - 2.0 * a) * torch.exp(-a) * amp_all.view(-1, 1, 1)
        ok = (idx >= 0) & (idx < nt)
        row = torch.as_tensor(jj, device=device).view(1, -1, 1) * nt
        flat = (row + idx)[ok]
        out.index_add_(0, flat, w[ok])
    out = out.view(ntr, nt)
    if noise_sigma > 0.0:
        rng = np.random.default_rng(seed + 7)
        out += torch.as_tensor(rng.normal(0.0, noise_sigma, (ntr, nt)), device=device)
    if dtype == np.float32:
        return out.to(torch.float32)
    return out


def random_traces(survey: Survey, seed: int, smooth: int = 0) -> np.ndarray:
    """White Gaussian traces (optionally smoothed by a running mean of ``smooth`` samples)."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((survey.ntr, survey.nt))
    if smooth > 1:
        ker = np.ones(smooth) / smooth
        d = np.apply_along_axis(lambda r: np.convolve(r, ker, mode="same"), 1, d)
    return d.astype(np.float32)


def random_image(survey: Survey, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(survey.image_shape).astype(np.float32)


def sample_points(survey: Survey, n: int, seed: int) -> np.ndarray:
    """Flat indices of ``n`` distinct image samples, uniform over the image."""
    rng = np.random.default_rng(seed)
    total = int(np.prod(survey.image_shape))
    return np.sort(rng.choice(total, size=min(n, total), replace=False)).astype(np.int64)
