"""The window slack of the table path (CPU).

With a radial traveltime table the migration kernel samples without the validity test when a
trace's window is not clipped and every lane of the warp lies in the tile box.  That needs every
interpolated two-way time of the box inside the window, which the library builds from the exact
time bounds of the box widened by 2 sqrt(D^2 + Dz^2) / v_min plus 2 samples: an interpolated leg
time is a convex combination of node times, each node within sqrt(D^2 + Dz^2) of the point
(D the horizontal node spacing, Dz = m dz the depth node spacing), and T is Lipschitz with
1 / v_min.  This checks that bound on the table scheme itself (the oracle's table, bilinear in
(h, z) with nodes on image depths, the scheme the kernel interpolates), against the closed-form
time, over random points, for several spacings and gradients."""
import numpy as np
import pytest

import oracle
from paper_1204_1225_gb300 import survey as sv


def _survey(v0, k, dz, nz, D):
    z1 = np.zeros(1, np.float32)
    return sv.Survey(dim=2, nx=1, ny=1, nz=nz, ox=0.0, oy=0.0, oz=0.0, dx=10.0, dy=10.0, dz=dz,
                     n_bins=1, bin_width=1e4, vel="table", v0=v0, k=k, weight="one", r0=1000.0,
                     aperture=0.0, nt=400, t0=0.0, dt=0.004, sx=z1, sy=z1, rx=z1, ry=z1,
                     table_spacing=D)


def _closed_form(h, z, v0, k):
    if k == 0.0:
        return np.hypot(h, z) / v0
    return np.arccosh(1.0 + k * k * (h * h + z * z) / (2.0 * v0 * (v0 + k * z))) / abs(k)


def _depth_stride(D, dz):
    m = 1
    while m < 4 and 2 * m <= D / dz:
        m *= 2
    return m


@pytest.mark.parametrize("v0,k,dz,D", [(1500.0, 0.5, 12.5, 25.0), (1500.0, 0.5, 12.5, 50.0),
                                       (1800.0, 0.6, 5.0, 25.0), (2000.0, 0.0, 10.0, 40.0),
                                       (1500.0, 1.2, 6.25, 30.0)])
def test_interpolated_leg_time_within_the_slack_bound(v0, k, dz, D):
    nz = 160
    s = _survey(v0, k, dz, nz, D)
    rng = np.random.default_rng(11)
    h = rng.uniform(0.0, 3000.0, 20000)
    z = dz * rng.integers(0, nz, 20000).astype(np.float64)    # image depths
    h[:200] = rng.uniform(0.0, 2.0 * D, 200)                    # near the source: most curved
    z[:200] = dz * rng.integers(0, 8, 200)
    Tt = oracle.table_traveltime(s, h, z)
    Te = _closed_form(h, z, v0, k)
    m = _depth_stride(D, dz)
    zmax = dz * (nz - 1) + m * dz
    vmin = min(v0, v0 + k * zmax)
    bound = np.sqrt(D * D + (m * dz) ** 2) / vmin
    err = np.max(np.abs(Tt - Te))
    print(f"v0 {v0} k {k} dz {dz} D {D}: max |T_table - T| = {err * 1e3:.3f} ms, bound {bound * 1e3:.3f} ms")
    assert err <= bound

