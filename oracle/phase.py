"""Henyey-Greenstein phase function and the discrete phase matrix, FP64.

Eq. 11 (§2.1): phi(mu) = (1/4pi) (1 - g^2) / (1 + g^2 - 2 g mu)^(3/2), normalised to one
over the sphere (text under Eq. 1) with mean cosine g.

Eq. 12 (§2.1): the source function is a discrete sum S_i = a * sum_j p(Omega_j, Omega_i)
I_j dOmega.  The paper does not say how the discrete weights are normalised.  Reading
used here (and by the GPU library): the raw kernel K_ij = w * phi(Omega_i . Omega_j; g_eff)
is scaled by a diagonal D, P = D K D, so that every row and every column of P sums to one
(scattering neither creates nor destroys photons and keeps an isotropic field isotropic),
and g_eff is chosen so that the mean over i of sum_j P_ij (Omega_i . Omega_j) equals the
physical g.  P is symmetric, so the same matrix serves both orientations of the sum.
"""
import numpy as np

from .healpix import ring_directions, pixel_weight


def henyey_greenstein(mu, g):
    """Eq. 11: HG phase function per steradian at scattering cosine ``mu``."""
    mu = np.asarray(mu, dtype=np.float64)
    return (1.0 - g * g) / (4.0 * np.pi * (1.0 + g * g - 2.0 * g * mu) ** 1.5)


def raw_kernel(dirs, w, g):
    """K_ij = w * phi(Omega_i . Omega_j; g) (the un-normalised weights of Eq. 12)."""
    mu = np.clip(dirs @ dirs.T, -1.0, 1.0)
    return w * henyey_greenstein(mu, g)


def symmetric_sinkhorn(K, tol=1e-14, max_iter=200000):
    """Diagonal scaling P = D K D with unit row (and, by symmetry, column) sums.

    Fixed point d_i * sum_j K_ij d_j = 1, reached by the damped update
    d <- sqrt(d / (K d)).  Stops when every row sum is within ``tol`` of one.
    """
    d = np.ones(K.shape[0])
    for _ in range(max_iter):
        r = d * (K @ d)
        if np.max(np.abs(r - 1.0)) < tol:
            break
        d = np.sqrt(d / (K @ d))
    else:
        raise RuntimeError("Sinkhorn scaling did not converge")
    return d[:, None] * K * d[None, :]


def mean_cosine(P, dirs):
    """Mean over rows i of sum_j P_ij Omega_i . Omega_j."""
    return float(np.mean(np.sum(P * (dirs @ dirs.T), axis=1)))


def phase_matrix(nside, g, return_geff=False):
    """The normalised discrete phase matrix P (N_a x N_a, FP64) of Eq. 12.

    g == 0 gives the isotropic matrix 1/N_a exactly.  Otherwise g_eff is found by
    bisection on [0, 1) (or (-1, 0] for g < 0) so that mean_cosine(P(g_eff)) == g,
    to an interval width below 1e-15.
    """
    dirs = ring_directions(nside)
    w = pixel_weight(nside)
    n = dirs.shape[0]
    if g == 0.0:
        P = np.full((n, n), 1.0 / n)
        return (P, 0.0) if return_geff else P
    if not -1.0 < g < 1.0:
        raise ValueError("g must lie in (-1, 1)")

    def build(ge):
        return symmetric_sinkhorn(raw_kernel(dirs, w, ge))

    lo, hi = (0.0, 1.0 - 1e-12) if g > 0 else (-1.0 + 1e-12, 0.0)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mean_cosine(build(mid), dirs) < g:
            lo = mid
        else:
            hi = mid
        if hi - lo < 1e-15:
            break
    geff = 0.5 * (lo + hi)
    P = build(geff)
    return (P, geff) if return_geff else P
