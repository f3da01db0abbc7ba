"""Pins of the two-level angular grid (§2.1: transport on fine HEALPix directions, the
source function on coarse ones from the mean of each coarse bin's children).

Point location is pinned by the round trip through the pixel centres of the published
construction, by equal pixel areas (Monte Carlo counts), and by the nesting of two
resolutions; the two-level step by two reductions that fix it independently: with
isotropic scattering it equals the one-level step on the fine grid (a coarse bin's mean
of the children's intensities sums them all), and a uniform isotropic field in a
non-absorbing periodic box is invariant for any anisotropy.
"""
import numpy as np
import pytest

import workloads as W
from oracle.healpix import parent_map, ring_pixel, ring_z_phi
from oracle.solver import Solver
from oracle.twolevel import TwoLevelSolver


@pytest.mark.parametrize("nside", [1, 2, 3, 4, 8, 16])
def test_pixel_centres_locate_to_themselves(nside):
    z, phi = ring_z_phi(nside)
    assert np.array_equal(ring_pixel(nside, z, phi), np.arange(12 * nside * nside))


@pytest.mark.parametrize("nside", [4, 16])
def test_pixels_have_equal_areas(nside):
    rng = np.random.default_rng(0)
    M = 1_000_000
    z = rng.uniform(-1.0, 1.0, M)  # uniform on the sphere (Archimedes)
    phi = rng.uniform(0.0, 2 * np.pi, M)
    npix = 12 * nside * nside
    c = np.bincount(ring_pixel(nside, z, phi), minlength=npix)
    mean = M / npix
    chi2 = np.sum((c - mean) ** 2 / mean)
    # chi-square with npix - 1 degrees of freedom: mean npix - 1, std sqrt(2 (npix - 1))
    assert abs(chi2 - (npix - 1)) < 6 * np.sqrt(2 * (npix - 1))
    assert np.max(np.abs(c - mean)) < 6 * np.sqrt(mean)


@pytest.mark.parametrize("fine,coarse", [(16, 4), (4, 2), (2, 1), (8, 4)])
def test_resolutions_nest(fine, coarse):
    par = parent_map(fine, coarse)
    assert np.all(np.bincount(par, minlength=12 * coarse ** 2) == (fine // coarse) ** 2)
    rng = np.random.default_rng(1)
    z = rng.uniform(-1.0, 1.0, 200_000)
    phi = rng.uniform(0.0, 2 * np.pi, 200_000)
    assert np.array_equal(par[ring_pixel(fine, z, phi)], ring_pixel(coarse, z, phi))
    # the children's mean direction points at the parent's centre (to O(pixel size^2))
    from oracle.healpix import ring_directions
    df, dc = ring_directions(fine), ring_directions(coarse)
    m = np.zeros_like(dc)
    np.add.at(m, par, df)
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    assert np.min(np.sum(m * dc, axis=1)) > np.cos(0.5 * np.sqrt(4 * np.pi / (12 * coarse ** 2)))


def _small(nside, g, mus, steps=12, n=8):
    p = W.homogeneous(n, n, n, nside, 0.02, mus, g=g, steps=steps, tol=1e-12)
    p["max_iters"] = 10000
    rng = np.random.default_rng(2)
    p["mus"] = mus * (1 + 0.5 * rng.random(p["mus"].shape))
    c = n / 2
    p["source"] = dict(face=4, u_mm=c, v_mm=c, half_angle_deg=20.0, pulse_steps=1, energy=1.0)
    p["detectors"] = [dict(face=4, u_mm=c + 2.5, v_mm=c + 0.5, radius_mm=0.5, half_angle_deg=20.0),
                      dict(face=5, u_mm=c + 0.5, v_mm=c + 0.5, radius_mm=0.5, half_angle_deg=20.0)]
    return W._bins(p)


@pytest.mark.parametrize("fine,coarse", [(2, 1), (4, 2)])
def test_isotropic_scattering_reduces_to_the_fine_grid(fine, coarse):
    p = _small(fine, 0.0, 1.0, steps=10 if fine == 4 else 12, n=6 if fine == 4 else 8)
    a = Solver(dict(p)).run(p["steps"])
    b = TwoLevelSolver(dict(p, nside_scatter=coarse)).run(p["steps"])
    assert np.max(np.abs(a["detectors"] - b["detectors"])) <= 1e-11 * np.max(np.abs(a["detectors"]))
    assert np.allclose(a["energy"], b["energy"], rtol=1e-11, atol=0)


def test_same_resolution_is_the_one_level_step():
    p = _small(2, 0.9, 2.0)
    a = Solver(dict(p)).run(p["steps"])
    b = TwoLevelSolver(dict(p, nside_scatter=2)).run(p["steps"])
    assert np.array_equal(a["detectors"], b["detectors"])


def test_uniform_isotropic_field_is_invariant():
    p = W.homogeneous(5, 4, 6, 2, 0.0, 3.0, g=0.9, steps=6, tol=1e-13, boundary="periodic")
    p["max_iters"] = 10000
    rng = np.random.default_rng(3)
    p["mus"] = 3.0 * (1 + rng.random(p["mus"].shape))
    s = TwoLevelSolver(dict(p, nside_scatter=1))
    s.I[:] = 1.0
    s.S[:] = 1.0
    s.hist_from = -(len(s.I) - 1)
    s.run(6)
    assert np.max(np.abs(s.I - 1.0)) < 1e-11 and np.max(np.abs(s.S - 1.0)) < 1e-11
