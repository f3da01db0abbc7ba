"""Independent brute-force ray tracer for tiny grids (checks the ray lattice).

It walks every long ray of every direction through the box by accumulating the
3-D step vector ds_d * Omega_d from a slab-0 voxel centre, and records which voxel
each ray point falls in (the voxel containing the point is the one with the nearest
centre, §2.1 text after Eq. 10).  Rays start at every slab-0 column of an extended
range, so the rays that enter through side faces are walked too.  The result is the
upwind map "previous point of the same ray", built without the per-slab offset
formula of ``geometry`` and with its own dominant-axis and floor rules (this module
imports nothing from ``geometry``, so a mistake there cannot hide here).  Plain Python
loops: tiny grids only.
"""
import math

import numpy as np

SNAP = 1e-9  # a coordinate this close to a voxel face belongs to the voxel on its + side


def _major_axis(om):
    """Index of the largest |component| of ``om``; on a tie z wins over y, y over x.

    Written as a scan from z down to x that keeps the first strict maximum, so that a
    tie (|Omega_x| = |Omega_y| happens at every N_side) goes to the later axis."""
    best, which = -1.0, -1
    for a in (2, 1, 0):
        c = abs(float(om[a]))
        if c > best + 1e-12:
            best, which = c, a
    return which


def _cell(coord):
    """Voxel index of a coordinate given in voxel units: the integer part, except that a
    value within SNAP of an integer is that integer (the point lies on a voxel face)."""
    k = math.floor(coord)
    if coord - k > 1.0 - SNAP:
        return k + 1
    return k


def traced_upwind(dirs, shape_zyx, h):
    """Upwind flat index per (direction, voxel): -1 inflow face, -2 side entry.

    Also returns the visit count per (direction, voxel), which must be exactly one.
    """
    nz, ny, nx = shape_zyx
    n = (nx, ny, nz)
    na = len(dirs)
    up = np.full((na, nx * ny * nz), -3, dtype=np.int64)
    visits = np.zeros((na, nx * ny * nz), dtype=np.int64)
    for d in range(na):
        om = np.asarray(dirs[d], dtype=np.float64)
        dom = _major_axis(om)
        step = (h / abs(om[dom])) * om
        tr = [a for a in range(3) if a != dom]
        first = 0 if om[dom] > 0 else n[dom] - 1
        rng = [range(-n[dom] - 1, n[a] + n[dom] + 1) for a in tr]
        for c0 in rng[0]:
            for c1 in rng[1]:
                pos = np.zeros(3)
                pos[dom] = (first + 0.5) * h
                pos[tr[0]] = (c0 + 0.5) * h
                pos[tr[1]] = (c1 + 0.5) * h
                prev = -1  # the sample before slab 0 is the inflow ghost
                for k in range(n[dom]):
                    if k > 0:
                        pos = pos + step
                    idx = [_cell(pos[a] / h) for a in range(3)]
                    inside = all(0 <= idx[a] < n[a] for a in range(3))
                    if inside:
                        flat = (idx[2] * ny + idx[1]) * nx + idx[0]
                        visits[d, flat] += 1
                        up[d, flat] = prev
                        prev = flat
                    else:
                        prev = -2
    return up, visits
