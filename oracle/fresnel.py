"""Refraction and reflection at refractive-index interfaces, FP64.

Eq. 13 (Snell): n1 sin(theta1) = n2 sin(theta2).
Eq. 14 (Fresnel): R = 1/2 [sin^2(t1 - t2)/sin^2(t1 + t2) + tan^2(t1 - t2)/tan^2(t1 + t2)]
for theta1 below the critical angle, R = 1 beyond it.

§3.3 (air-hole phantom): grid points next to a region of different refractive index are
"boundary grids", and their source function uses a phase function that includes Eqs.
13-14.  The paper does not say how.  Reading used here (and by the GPU library):

* A segment crosses an interface when the upwind sample of voxel v along direction j
  lies in a voxel of different n.  The light that arrives along j at v through the
  interface, Q(v, j), is split: R(theta1) goes to the specular direction and 1 - R to
  the Snell direction, each snapped to the pixel with the largest dot product (lowest
  index among dot products within 1e-12 of the best).  Incident medium n1 = n(upwind),
  transmitted n2 = n(v).
* The interface normal at v is the central-difference gradient of the n map (one-sided
  at the box faces); a voxel where it vanishes is left alone.
* The redistribution acts on Q before the source iteration of the step, and is
  column-stochastic (sum over outputs of each column = 1), so photons are conserved.
  The n^2 scaling of radiance across an index step is not applied (pixel weights are
  equal and the solver carries intensities per pixel).
* R uses the cosine form 1/2 (r_s^2 + r_p^2), which equals Eq. 14 and avoids its 0/0 at
  normal incidence.

Parity status: the optics (R, Snell direction, critical angle) are pinned against Eq. 14
itself and textbook limits, and the whole redistribution table of a plane index step
against directions and weights written out by hand; on curved interfaces the normal of a
stair-stepped boundary has no closed form, and the redistribution there rests on
oracle-GPU agreement ("parity unpinned" beyond its conservation property).
"""
import numpy as np


def fresnel_R(n1, n2, cos1):
    """Unpolarised Fresnel reflectance for incidence cosine ``cos1`` from n1 into n2."""
    cos1 = np.clip(np.asarray(cos1, dtype=np.float64), 0.0, 1.0)
    eta = n1 / n2
    sin2_t = eta * eta * (1.0 - cos1 * cos1)
    tir = sin2_t >= 1.0
    cos2 = np.sqrt(np.clip(1.0 - sin2_t, 0.0, 1.0))
    rs = (n1 * cos1 - n2 * cos2) / (n1 * cos1 + n2 * cos2)
    rp = (n2 * cos1 - n1 * cos2) / (n2 * cos1 + n1 * cos2)
    R = 0.5 * (rs * rs + rp * rp)
    return np.where(tir | (cos1 <= 0.0), 1.0, R)


def fresnel_R_eq14(n1, n2, theta1):
    """Eq. 14 as printed (sin/tan form), for 0 < theta1 < theta_c (test reference)."""
    theta2 = np.arcsin(n1 / n2 * np.sin(theta1))
    a, b = theta1 - theta2, theta1 + theta2
    return 0.5 * (np.sin(a) ** 2 / np.sin(b) ** 2 + np.tan(a) ** 2 / np.tan(b) ** 2)


def reflect_refract(omega, m, n1, n2):
    """Specular and Snell directions of unit vector ``omega`` at a surface with unit normal
    ``m`` (either orientation), travelling from n1 into n2.  Returns (R, omega_r, omega_t);
    omega_t is None under total internal reflection."""
    om = np.asarray(omega, dtype=np.float64)
    dn = float(om @ m)
    u = m if dn >= 0 else -m          # normal along the direction of travel
    cos1 = abs(dn)
    R = float(fresnel_R(n1, n2, cos1))
    om_r = om - 2.0 * dn * m
    eta = n1 / n2
    sin2_t = eta * eta * (1.0 - cos1 * cos1)
    if sin2_t >= 1.0 or cos1 <= 0.0:
        return 1.0, om_r, None
    cos2 = np.sqrt(1.0 - sin2_t)
    om_t = eta * om + (cos2 - eta * cos1) * u
    return R, om_r, om_t


def nearest_direction(dirs, v):
    """Index of the pixel centre with the largest dot product; dot products within 1e-12
    of the best count as ties and the lowest index wins (so that rounding differences of
    two FP64 implementations cannot flip the choice)."""
    dots = dirs @ v
    return int(np.nonzero(dots >= dots.max() - 1e-12)[0][0])


def index_normals(nidx, h=1.0):
    """Central-difference gradient of the refractive-index map [nz, ny, nx] per voxel,
    as (gz, gy, gx) arrays (one-sided differences at the box faces)."""
    return np.gradient(np.asarray(nidx, dtype=np.float64), h)


def interface_operators(model):
    """Per interface voxel v: a dict {direction j -> [(d_out, weight), ...]} for the
    directions whose segment crosses an index step, built as described above."""
    nz, ny, nx = model.shape
    nmap = model.nidx.reshape(nz, ny, nx)
    gz, gy, gx = index_normals(nmap, model.h)
    ops = {}
    for j in range(model.na):
        up = model.lat.upwind_index(j)
        ok = up >= 0
        vs = np.nonzero(ok)[0]
        cross = vs[model.nidx[up[ok]] != model.nidx[vs]]
        for v in cross:
            z, rem = divmod(int(v), nx * ny)
            y, x = divmod(rem, nx)
            g = np.array([gx[z, y, x], gy[z, y, x], gz[z, y, x]])
            gn = np.linalg.norm(g)
            if gn == 0.0:
                continue
            m = g / gn
            n1, n2 = float(model.nidx[up[v]]), float(model.nidx[v])
            R, om_r, om_t = reflect_refract(model.dirs[j], m, n1, n2)
            outs = [(nearest_direction(model.dirs, om_r), R)]
            if om_t is not None:
                outs.append((nearest_direction(model.dirs, om_t), 1.0 - R))
            ops.setdefault(int(v), {})[j] = outs
    return ops


def apply_interfaces(ops, Q):
    """Q' = F Q at every interface voxel (Q is [N_a, N_v], updated in place)."""
    for v, cols in ops.items():
        q = Q[:, v].copy()
        out = q.copy()
        for j, outs in cols.items():
            out[j] -= q[j]
            for d, wgt in outs:
                out[d] += wgt * q[j]
        Q[:, v] = out
    return Q
