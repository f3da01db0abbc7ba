"""Collimated source and detector acceptance cones, FP64.

§3.1: the pulse is injected collimated within a 15-degree cone and the detectors have
the same opening angle.  At N_side = 2 no pixel centre lies within 15 degrees of an
axis, so the cone cannot be a set of whole pixels.  Reading used here: the cone's
solid angle is shared among directions by nearest-centre assignment.  The cap of
half-angle theta_c around the axis n is sampled at K x L equal-area points
(cos theta uniform on [cos theta_c, 1]: mu_k = 1 - (k + 1/2)(1 - cos theta_c)/K;
phi_l = 2 pi (l + 1/2)/L), each point is assigned to the direction with the largest
dot product, and alpha_d is the fraction of points assigned to d (sum_d alpha_d = 1).
A point whose two best dot products differ by less than 1e-12 is a tie and raises.

The cap's local frame is (e_u, e_v, n) with e_u, e_v the face's own u and v axes.
"""
import numpy as np

from .geometry import face_axes

CAP_K = 64
CAP_L = 256
TIE_EPS = 1e-12


def cap_samples(axis_vec, e_u, e_v, half_angle_deg, K=CAP_K, L=CAP_L):
    """Equal-area sample points (unit vectors, [K*L, 3]) of the cap around ``axis_vec``."""
    ct = np.cos(np.radians(half_angle_deg))
    mu = 1.0 - (np.arange(K) + 0.5) * (1.0 - ct) / K
    phi = 2.0 * np.pi * (np.arange(L) + 0.5) / L
    mu, phi = np.meshgrid(mu, phi, indexing="ij")
    st = np.sqrt((1.0 - mu) * (1.0 + mu))
    pts = (mu.ravel()[:, None] * axis_vec[None, :]
           + (st * np.cos(phi)).ravel()[:, None] * e_u[None, :]
           + (st * np.sin(phi)).ravel()[:, None] * e_v[None, :])
    return pts


def cone_fractions(dirs, face, half_angle_deg, inward):
    """alpha_d: fraction of the cone around the face normal that falls nearest to d.

    ``inward`` selects the cone around the inward normal (a source on that face) or the
    outward normal (a detector on that face).
    """
    ax, sign, (ua, va) = face_axes(face)
    nvec = np.zeros(3)
    nvec[ax] = -sign if inward else sign
    e_u = np.zeros(3)
    e_u[ua] = 1.0
    e_v = np.zeros(3)
    e_v[va] = 1.0
    pts = cap_samples(nvec, e_u, e_v, half_angle_deg)
    dots = pts @ np.asarray(dirs).T
    best = np.argmax(dots, axis=1)
    srt = np.sort(dots, axis=1)
    if np.any(srt[:, -1] - srt[:, -2] < TIE_EPS):
        raise ValueError("cone sample equidistant from two directions")
    counts = np.bincount(best, minlength=dirs.shape[0])
    return counts / float(pts.shape[0])


def cap_solid_angle(half_angle_deg):
    """Solid angle of a cap of the given half-angle, 2 pi (1 - cos theta_c)."""
    return 2.0 * np.pi * (1.0 - np.cos(np.radians(half_angle_deg)))
