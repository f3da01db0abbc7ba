"""Long-characteristic ray lattice on a uniform voxel grid, FP64 decisions.

§2.1 (text after Eq. 9 and Fig. 1) and §2.4 Step 1: rays are laid independently of
the grid and run from one face of the box to the other; the intensity of a grid
point is taken from the nearest ray with a single interpolation, so no numerical
diffusion builds up along the ray.  The paper gives no construction.  Reading used
here ("slab lattice"):

* For direction Omega_d the dominant axis dom(d) is the axis of the largest
  |Omega_d| component (ties prefer z, then y, then x).  The box is cut into slabs
  normal to dom(d), slab k' = 0, 1, ... counted along the direction of travel.
* Every ray passes through the centre of one voxel of slab 0 and advances by
  ds_d = h / |Omega_dom| between slab centre planes, moving t_a = Omega_a / |Omega_dom|
  voxels along each transverse axis a.  At slab k' the ray lies in the voxel column
  c + floor(1/2 + k' t_a) (the voxel whose centre is nearest to the ray point).
* So every voxel holds exactly one sample of one ray per direction; its upwind
  sample is the previous sample of the same ray, in slab k'-1, shifted transversely
  by -Delta_a(k') with Delta_a(k') = floor(1/2 + k' t_a) - floor(1/2 + (k'-1) t_a),
  which is -1, 0 or +1.
* For k' = 0 the upwind sample lies outside the box (inflow through the face normal
  to dom(d)); when the transverse shift leaves the box the ray entered through a side
  face (vacuum: zero inflow).  With periodic boundaries indices wrap, and slab 0 takes
  its upwind sample from slab N-1 with Delta_a(0) = -floor(1/2 - t_a).

Integer decisions are taken in FP64.  A floor argument within 1e-9 of an integer is a
tie (a ray point on a voxel face; it happens for real at N_side = 2, where the
directions (+-2/3, +-2/3, +-1/3) have t = +-1/2).  Such an argument is snapped to that
integer, i.e. a ray point lying on a voxel face belongs to the voxel on its + side.
The snap margin is far above FP64 rounding and far below any genuine distance, so two
independent FP64 implementations take the same decision.
"""
import numpy as np

TIE_EPS = 1e-9
DOM_EPS = 1e-12


def dominant_axis(omega):
    """Axis (0=x, 1=y, 2=z) of the largest |component|; ties prefer z, then y, then x."""
    ax, ay, az = np.abs(omega)
    if az >= max(ax, ay) - DOM_EPS:
        return 2
    if ay >= ax - DOM_EPS:
        return 1
    return 0


def transverse_axes(dom):
    """The two axes other than ``dom``, in increasing order."""
    return [a for a in range(3) if a != dom]


def floor_snapped(y):
    """floor(y), except that y within TIE_EPS of an integer is taken as that integer."""
    y = np.asarray(y, dtype=np.float64)
    r = np.round(y)
    return np.where(np.abs(y - r) < TIE_EPS, r, np.floor(y)).astype(np.int64)


def slab_offsets(t, nslab, periodic):
    """Delta(k') for k' = 0..nslab-1 for one transverse slope ``t`` (|t| <= 1).

    Delta(0) is only meaningful with periodic boundaries (0 otherwise).
    """
    k = np.arange(nslab, dtype=np.float64)
    cur = floor_snapped(0.5 + k * t)
    prev = floor_snapped(0.5 + (k - 1.0) * t)
    off = cur - prev
    if not periodic:
        off[0] = 0
    return off


class RayLattice:
    """Per-direction lattice data for a grid of shape (nz, ny, nx) and spacing h (mm)."""

    def __init__(self, dirs, shape_zyx, h, periodic=False):
        self.dirs = np.asarray(dirs, dtype=np.float64)
        nz, ny, nx = shape_zyx
        self.n_xyz = (nx, ny, nz)
        self.h = float(h)
        self.periodic = bool(periodic)
        na = self.dirs.shape[0]
        self.dom = np.empty(na, dtype=np.int64)
        self.sgn = np.empty(na, dtype=np.int64)
        self.ds = np.empty(na)
        self.slopes = np.zeros((na, 2))
        self.offsets = []  # per direction: int array [2, n_dom]
        for d in range(na):
            om = self.dirs[d]
            dom = dominant_axis(om)
            self.dom[d] = dom
            self.sgn[d] = 1 if om[dom] > 0 else -1
            self.ds[d] = self.h / abs(om[dom])
            tax = transverse_axes(dom)
            offs = []
            for j, a in enumerate(tax):
                t = om[a] / abs(om[dom])
                self.slopes[d, j] = t
                offs.append(slab_offsets(t, self.n_xyz[dom], self.periodic))
            self.offsets.append(np.stack(offs))

    def upwind_index(self, d, voxels=None):
        """Flat upwind voxel index for direction d, for all voxels or the given flat indices.

        -1: the upwind sample is outside the box across the face normal to dom(d)
            (inflow face; k' = 0).
        -2: the ray entered through a side face (vacuum: zero inflow).
        Periodic lattices always return a valid index.
        """
        nx, ny, nz = self.n_xyz
        v = np.arange(nx * ny * nz) if voxels is None else np.asarray(voxels, dtype=np.int64)
        p = [v % nx, (v // nx) % ny, v // (nx * ny)]
        n = [nx, ny, nz]
        dom = int(self.dom[d])
        sgn = int(self.sgn[d])
        kprime = p[dom] if sgn > 0 else n[dom] - 1 - p[dom]
        q = [c.copy() for c in p]
        q[dom] = p[dom] - sgn
        for j, a in enumerate(transverse_axes(dom)):
            q[a] = p[a] - self.offsets[d][j][kprime]
        if self.periodic:
            q = [q[a] % n[a] for a in range(3)]
            return (q[2] * ny + q[1]) * nx + q[0]
        out = (q[2] * ny + q[1]) * nx + q[0]
        side = np.zeros_like(out, dtype=bool)
        for a in transverse_axes(dom):
            side |= (q[a] < 0) | (q[a] >= n[a])
        out = np.where(side, -2, out)
        out = np.where(kprime == 0, -1, out)
        return out

    def upwind_coords(self, d, voxels):
        """Unwrapped (x, y, z) coordinates of the upwind sample of direction d for the given
        flat voxel indices (each may lie one voxel outside the box on any axis)."""
        nx, ny, nz = self.n_xyz
        v = np.asarray(voxels, dtype=np.int64)
        p = [v % nx, (v // nx) % ny, v // (nx * ny)]
        n = [nx, ny, nz]
        dom = int(self.dom[d])
        sgn = int(self.sgn[d])
        kprime = p[dom] if sgn > 0 else n[dom] - 1 - p[dom]
        q = [c.copy() for c in p]
        q[dom] = p[dom] - sgn
        for j, a in enumerate(transverse_axes(dom)):
            q[a] = p[a] - self.offsets[d][j][kprime]
        return q

    def entry_face(self, d):
        """Face (0..5 = -x,+x,-y,+y,-z,+z) through which direction d enters at k' = 0."""
        dom = int(self.dom[d])
        return 2 * dom if self.sgn[d] > 0 else 2 * dom + 1


def face_axes(face):
    """(normal axis, outward sign, (u axis, v axis)) of a face 0..5."""
    ax = face // 2
    sign = -1 if face % 2 == 0 else 1
    return ax, sign, tuple(transverse_axes(ax))
