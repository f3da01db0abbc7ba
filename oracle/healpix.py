"""HEALPix pixel centres in RING order, FP64.

§2.1 (angular discretisation, text around Eq. 12): the paper discretises direction
space with HEALPix equal-area pixels and runs its fiducial model with 3072 bins
(N_side = 16) and a coarse source-function grid of 192 bins (N_side = 4).

The pixel-centre positions follow the published HEALPix construction (Gorski et al.
2005, ApJ 622, 759): 4*N_side - 1 iso-latitude rings; rings in the polar caps carry
4*i pixels, rings in the equatorial belt carry 4*N_side pixels, every pixel has the
same area 4*pi / (12 N_side^2).
"""
import numpy as np


def ring_z_phi(nside):
    """Return (z, phi) of the 12*nside^2 pixel centres, RING order.

    Ring index i runs 1 .. 4*nside-1 from the north pole.
      polar cap (i < nside):        z = 1 - i^2/(3 nside^2), 4i pixels,
                                    phi_j = (pi / (2i)) (j - 1/2),      j = 1..4i
      belt (nside <= i <= 3 nside): z = 4/3 - 2i/(3 nside), 4 nside pixels,
                                    phi_j = (pi / (2 nside)) (j - s/2), s = (i - nside + 1) mod 2
      south cap (i > 3 nside):      mirror image of ring 4 nside - i.
    """
    if nside < 1:
        raise ValueError("nside must be >= 1")
    zs, phis = [], []
    for i in range(1, 4 * nside):
        if i < nside:
            z = 1.0 - i * i / (3.0 * nside * nside)
            j = np.arange(1, 4 * i + 1)
            phi = (np.pi / (2.0 * i)) * (j - 0.5)
        elif i <= 3 * nside:
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * nside)
            s = (i - nside + 1) % 2
            j = np.arange(1, 4 * nside + 1)
            phi = (np.pi / (2.0 * nside)) * (j - 0.5 * s)
        else:
            ii = 4 * nside - i
            z = -(1.0 - ii * ii / (3.0 * nside * nside))
            j = np.arange(1, 4 * ii + 1)
            phi = (np.pi / (2.0 * ii)) * (j - 0.5)
        zs.append(np.full(phi.shape, z))
        phis.append(phi)
    return np.concatenate(zs), np.concatenate(phis)


def ring_directions(nside):
    """Unit vectors Omega_d (shape [12 nside^2, 3]) of the RING-ordered pixel centres."""
    z, phi = ring_z_phi(nside)
    sin_theta = np.sqrt((1.0 - z) * (1.0 + z))
    return np.stack([sin_theta * np.cos(phi), sin_theta * np.sin(phi), z], axis=1)


def pixel_weight(nside):
    """Solid angle of one pixel, 4 pi / N_a (equal-area pixels)."""
    return 4.0 * np.pi / (12 * nside * nside)


def ring_pixel(nside, z, phi):
    """RING index of the pixel containing each direction (z = cos theta, phi), FP64.

    Restated from the pixel boundaries of the HEALPix construction (Gorski et al. 2005):
      belt (|z| <= 2/3): with t = 2 nside phi / pi (one unit per pixel along a ring) and
        w = 3 nside z / 2 (one unit per ring), pixels are the unit squares of the rotated
        lattice a = t + w/2, b = t - w/2, whose centres sit at (N - 1)/2 + integers;
        the centre (a0, b0) gives ring i = 2N - (a0 - b0) and j = (a0 + b0 + s)/2 with
        s = (i - N + 1) mod 2 (j taken modulo 4N);
      caps (|z| > 2/3): with sigma = N sqrt(3 (1 - |z|)) and tp the fraction of phi within
        its quarter, pixel boundaries are the curves x = tp sigma = k and
        y = (1 - tp) sigma = k, so ring i = floor(x) + floor(y) + 1 (counted from the
        pole) and, in quarter q, j = q i + floor(x) + 1.
    """
    z = np.asarray(z, dtype=np.float64)
    phi = np.mod(np.asarray(phi, dtype=np.float64), 2.0 * np.pi)
    N = nside
    npix = 12 * N * N
    out = np.empty(z.shape, dtype=np.int64)
    belt = np.abs(z) <= 2.0 / 3.0
    # belt
    t = 2.0 * N * phi[belt] / np.pi
    w = 1.5 * N * z[belt]
    off = (N - 1) / 2.0
    a0 = np.floor(t + w / 2.0 - off + 0.5) + off
    b0 = np.floor(t - w / 2.0 - off + 0.5) + off
    i = np.rint(2 * N - (a0 - b0)).astype(np.int64)
    s = (i - N + 1) % 2
    j = np.rint((a0 + b0 + s) / 2.0).astype(np.int64)
    j = (j - 1) % (4 * N) + 1
    out[belt] = 2 * N * (N - 1) + 4 * N * (i - N) + (j - 1)
    # caps
    cap = ~belt
    zc, pc = z[cap], phi[cap]
    sigma = N * np.sqrt(3.0 * (1.0 - np.abs(zc)))
    quarter = np.minimum(np.floor(pc / (np.pi / 2.0)), 3.0)
    tp = pc / (np.pi / 2.0) - quarter
    kx = np.floor(tp * sigma)
    ky = np.floor((1.0 - tp) * sigma)
    ic = (kx + ky + 1).astype(np.int64)
    jc = (quarter * ic + kx + 1).astype(np.int64)
    north = zc > 0
    out_c = np.where(north, 2 * ic * (ic - 1) + (jc - 1), npix - 2 * ic * (ic + 1) + (jc - 1))
    out[cap] = out_c
    return out


def parent_map(nside_fine, nside_coarse):
    """Coarse pixel (RING) of every fine pixel: the coarse pixel that contains the fine
    pixel's centre.  HEALPix pixels nest, so every coarse pixel is the union of its
    (nside_fine / nside_coarse)^2 children (the paper's 16 finer angles per source-function
    bin, §2.1, when 3072 transport directions feed 192 source-function directions)."""
    if nside_fine % nside_coarse:
        raise ValueError("nside_fine must be a multiple of nside_coarse")
    z, phi = ring_z_phi(nside_fine)
    return ring_pixel(nside_coarse, z, phi)
