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
