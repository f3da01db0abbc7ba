"""Seeded synthetic workloads of the forward model.

This module only builds inputs: grid sizes, optical-property maps, source and
detector placements, iteration controls.  It holds none of the method's arithmetic,
so both the FP64 oracle and the GPU library can take their inputs from here.

A problem is a plain dict:
  nx, ny, nz, h (mm), nside, courant (c0 dt / (n_ref h)), n_ref,
  mua, mus, nidx: float32 arrays [nz, ny, nx] (1/mm, 1/mm, refractive index),
  g, boundary ("vacuum" | "periodic"),
  source: dict(face, u_mm, v_mm, half_angle_deg, pulse_steps, energy) or None,
  detectors: list of dict(face, u_mm, v_mm, radius_mm, half_angle_deg),
  bin_ps, nbins, tol, max_iters, steps, precision ("fp32" | "bf16").
Faces are 0..5 = -x, +x, -y, +y, -z, +z; (u, v) on a face are its two other axes in
increasing order (x face: (y, z); y face: (x, z); z face: (x, y)).

The named workloads follow the sizes and optics of the paper's phantom runs (§3):
a homogeneous tissue-like slab with mu_s ~ 10/mm, g = 0.9, n = 1.4, a 15-degree
collimated delta pulse and surface detectors with 10 ps bins, plus a heterogeneous
variant (air cylinder and absorbing spheres) and random-field optics for the served
stream.  The paper's own phantom measurements are not used (they are not available);
these inputs stand in for them.
"""
import math

import numpy as np


def _uniform(shape_zyx, value):
    return np.full(shape_zyx, value, dtype=np.float32)


def homogeneous(nx, ny, nz, nside, mua, mus, g=0.9, nidx=1.4, h=1.0, steps=100,
                tol=1e-6, max_iters=2000, boundary="vacuum", precision="fp32"):
    shp = (nz, ny, nx)
    return dict(nx=nx, ny=ny, nz=nz, h=h, nside=nside, courant=0.5, n_ref=1.4,
                mua=_uniform(shp, mua), mus=_uniform(shp, mus), nidx=_uniform(shp, nidx),
                g=g, boundary=boundary, source=None, detectors=[], bin_ps=10.0, nbins=1,
                tol=tol, max_iters=max_iters, steps=steps, precision=precision)


def _bins(prob):
    # Room for every bin a run can reach: 10 ps bins hold about four 2.3 ps steps, and
    # bins past the end of the run stay zero.
    prob["nbins"] = prob["steps"] // 4 + 2
    return prob


def config_small(steps=100, precision="fp32", tol=1e-6):
    """16^3 voxels at 1 mm, N_side 2 (48 directions), mu_a 0.01/mm, mu_s 10/mm, g 0.9,
    n 1.4; pulse at the centre of the -z face in a 15-degree cone; three detectors on the
    -z face at 3, 5, 7 mm from the source along +x and one at the centre of the +z face."""
    p = homogeneous(16, 16, 16, 2, 0.01, 10.0, steps=steps, tol=tol, precision=precision)
    c = 8.0  # face centre (voxel index 8 of 16)
    p["source"] = dict(face=4, u_mm=c, v_mm=c, half_angle_deg=15.0, pulse_steps=1, energy=1.0)
    p["detectors"] = [dict(face=4, u_mm=c + 0.5 + s, v_mm=c + 0.5, radius_mm=0.5,
                           half_angle_deg=15.0) for s in (3.0, 5.0, 7.0)]
    p["detectors"].append(dict(face=5, u_mm=c + 0.5, v_mm=c + 0.5, radius_mm=0.5,
                               half_angle_deg=15.0))
    return _bins(p)


def config_slab(steps=1500, precision="fp32", tol=1e-6, nx=96, ny=96, nz=64, nside=4):
    """Phantom-scale homogeneous slab: 96x96x64 voxels at 1 mm, N_side 4 (192 directions),
    mu_a 0.008/mm, mu_s 8/mm, g 0.9, n 1.4; delta pulse at the centre of the -z face in a
    15-degree cone; 8 detectors on the -z face at 10..40 mm from the source along +x."""
    p = homogeneous(nx, ny, nz, nside, 0.008, 8.0, steps=steps, tol=tol, precision=precision)
    cu, cv = float(nx // 2), float(ny // 2)
    p["source"] = dict(face=4, u_mm=cu, v_mm=cv, half_angle_deg=15.0, pulse_steps=1, energy=1.0)
    seps = np.linspace(10.0, 40.0, 8) * (nx / 96.0)
    p["detectors"] = [dict(face=4, u_mm=cu + 0.5 + float(s), v_mm=cv + 0.5, radius_mm=0.5,
                           half_angle_deg=15.0) for s in seps]
    return _bins(p)


def config_hetero(steps=1500, precision="bf16", tol=1e-6, nx=128, ny=128, nz=96, nside=4,
                  scale=1.0, seed=3):
    """Heterogeneous medium: 128x128x96 voxels at 1 mm, 192 directions, slab optics, an air
    cylinder (n 1, mu_a = mu_s = 0) of radius 5 mm along z through (x, y) = (32, 64) mm,
    and three absorbing spheres (radius 4, 6, 8 mm; mu_a x2, x3.5, x5) placed at random
    (seed 3) without touching the cylinder or the box faces.  Source at the centre of the
    -x face; 8 detectors on the -x face at 10..40 mm along +y.  ``scale`` shrinks every
    length (grid and features) for small test cases."""
    p = homogeneous(nx, ny, nz, nside, 0.008, 8.0, steps=steps, tol=tol, precision=precision)
    zz, yy, xx = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                             indexing="ij")
    cx, cy, rc = 32.0 * scale, 64.0 * scale, 5.0 * scale
    cyl = (xx - cx) ** 2 + (yy - cy) ** 2 <= rc * rc
    mua = p["mua"].astype(np.float64)
    mus = p["mus"].astype(np.float64)
    nidx = p["nidx"].astype(np.float64)
    rng = np.random.default_rng(seed)
    spheres = []
    for r, f in ((4.0 * scale, 2.0), (6.0 * scale, 3.5), (8.0 * scale, 5.0)):
        for _ in range(10000):
            c = rng.uniform([r + 1, r + 1, r + 1], [nx - r - 1, ny - r - 1, nz - r - 1])
            if math.hypot(c[0] - cx, c[1] - cy) < rc + r + 1:
                continue
            if any(np.linalg.norm(c - c2) < r + r2 + 1 for c2, r2, _ in spheres):
                continue
            spheres.append((c, r, f))
            break
        else:
            raise RuntimeError("could not place sphere")
    for c, r, f in spheres:
        inside = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= r * r
        mua[inside] *= f
    mua[cyl] = 0.0
    mus[cyl] = 0.0
    nidx[cyl] = 1.0
    p["mua"], p["mus"], p["nidx"] = (a.astype(np.float32) for a in (mua, mus, nidx))
    p["spheres"] = [(tuple(map(float, c)), float(r), float(f)) for c, r, f in spheres]
    p["fresnel"] = True  # refraction and reflection at the cylinder wall
    p["cylinder"] = dict(axis=2, center=(cx, cy), radius=rc)
    cu, cv = float(ny // 2), float(nz // 2)
    p["source"] = dict(face=0, u_mm=cu, v_mm=cv, half_angle_deg=15.0, pulse_steps=1, energy=1.0)
    seps = np.linspace(10.0, 40.0, 8) * scale
    p["detectors"] = [dict(face=0, u_mm=cu + 0.5 + float(s), v_mm=cv + 0.5, radius_mm=0.5,
                           half_angle_deg=15.0) for s in seps]
    return _bins(p)


def gaussian_random_field(shape_zyx, corr_mm, h, rng):
    """Unit-variance Gaussian random field: white noise smoothed by a Gaussian kernel of
    standard deviation ``corr_mm`` (periodic FFT convolution), then rescaled."""
    noise = rng.standard_normal(shape_zyx)
    k = [np.fft.fftfreq(n, d=h) for n in shape_zyx]
    kz, ky, kx = np.meshgrid(*k, indexing="ij")
    filt = np.exp(-2.0 * (math.pi * corr_mm) ** 2 * (kx**2 + ky**2 + kz**2))
    f = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    return (f - f.mean()) / f.std()


def config_served(n_side_len, nside, steps, seed, sigma=0.3, corr_mm=5.0, precision="fp32",
                  tol=1e-6):
    """One request of the served stream: a cubic grid with log-normal random-field optics
    (median mu_a 0.01/mm, mu_s 10/mm, sigma 0.3, correlation length 5 mm), g 0.9, n 1.4;
    source at the centre of the -z face, two detectors on the -z face."""
    n = n_side_len
    p = homogeneous(n, n, n, nside, 0.01, 10.0, steps=steps, tol=tol, precision=precision)
    rng = np.random.default_rng(seed)
    za = gaussian_random_field((n, n, n), corr_mm, 1.0, rng)
    zs = gaussian_random_field((n, n, n), corr_mm, 1.0, rng)
    p["mua"] = (0.01 * np.exp(sigma * za)).astype(np.float32)
    p["mus"] = (10.0 * np.exp(sigma * zs)).astype(np.float32)
    c = float(n // 2)
    p["source"] = dict(face=4, u_mm=c, v_mm=c, half_angle_deg=15.0, pulse_steps=1, energy=1.0)
    p["detectors"] = [dict(face=4, u_mm=c + 0.5 + s, v_mm=c + 0.5, radius_mm=0.5,
                           half_angle_deg=15.0) for s in (5.0, 10.0)]
    return _bins(p)


def config_adjoint(n=64, nside=4, steps=800, seed=11, sigma=0.3, corr_mm=5.0,
                   precision="fp32", tol=1e-6, bump=0.2):
    """Gradient workload: an n^3 grid at 1 mm (64^3), 192 directions, log-normal random-field
    optics (median mu_a 0.01/mm, mu_s 10/mm, sigma 0.3, correlation length 5 mm), g 0.9,
    n 1.4; delta pulse into a 15-degree cone at (n/4, n/2) on the -z face; 8 detectors on
    the -z face at 10..40 mm (scaled by n/64) along +x.  Returns (prob, prob_perturbed):
    the second has mu_a raised by ``bump`` (20 %) inside a Gaussian blob (std 4 mm, scaled)
    at depth n/6 midway between the source and the detectors; its detector curves are the
    observations of the least-squares misfit."""
    p = homogeneous(n, n, n, nside, 0.01, 10.0, steps=steps, tol=tol, precision=precision)
    rng = np.random.default_rng(seed)
    za = gaussian_random_field((n, n, n), corr_mm * n / 64.0, 1.0, rng)
    zs = gaussian_random_field((n, n, n), corr_mm * n / 64.0, 1.0, rng)
    p["mua"] = (0.01 * np.exp(sigma * za)).astype(np.float32)
    p["mus"] = (10.0 * np.exp(sigma * zs)).astype(np.float32)
    su, sv = float(n // 4), float(n // 2)
    p["source"] = dict(face=4, u_mm=su, v_mm=sv, half_angle_deg=15.0, pulse_steps=1, energy=1.0)
    seps = np.linspace(10.0, 40.0, 8) * (n / 64.0)
    p["detectors"] = [dict(face=4, u_mm=su + 0.5 + float(s), v_mm=sv + 0.5, radius_mm=0.5,
                           half_angle_deg=15.0) for s in seps]
    _bins(p)
    zz, yy, xx = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, np.arange(n) + 0.5,
                             indexing="ij")
    cx, cy, cz, r = su + 0.5 + 12.5 * n / 64.0, sv + 0.5, n / 6.0, 4.0 * n / 64.0
    blob = np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2 + (zz - cz) ** 2) / (2 * r * r))
    q = dict(p)
    q["mua"] = (p["mua"] * (1.0 + bump * blob)).astype(np.float32)
    return p, q


def served_stream(n_requests=2000, seed=4, rate_per_s=1.0):
    """Arrival times and shapes of the served stream: Poisson arrivals, cubic N uniform on
    32..96, 48 or 192 directions with probability 1/2, 500..1500 steps."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n_requests)
    out = []
    t = 0.0
    for i in range(n_requests):
        t += gaps[i]
        out.append(dict(arrival_s=t, n=int(rng.integers(32, 97)),
                        nside=2 if rng.random() < 0.5 else 4,
                        steps=int(rng.integers(500, 1501)), seed=int(rng.integers(1 << 31))))
    return out


def developed_history(prob, seed=7, levels=4):
    """A smooth synthetic field history for timing per-voxel work on the CPU: for each
    stored level (oldest first) an intensity that is a broad Gaussian glow around the
    source spot (std 15 mm) times (1 + 0.1 u), u uniform in [-1, 1] per voxel and
    direction, fading by 0.5% per level, with S = 0.9 I.  Returns (I, S), float32 arrays
    [levels, N_a, N_v]."""
    nz, ny, nx = prob["nz"], prob["ny"], prob["nx"]
    na = 12 * prob["nside"] ** 2
    src = prob["source"]
    zz, yy, xx = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                             indexing="ij")
    c = [0.0, 0.0, 0.0]
    ax = src["face"] // 2
    uv = [a for a in range(3) if a != ax]
    c[uv[0]], c[uv[1]] = src["u_mm"], src["v_mm"]
    c[ax] = 0.0 if src["face"] % 2 == 0 else (nx, ny, nz)[ax] * prob["h"]
    r2 = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2
    glow = np.exp(-r2 / (2 * 15.0 ** 2)).ravel()
    rng = np.random.default_rng(seed)
    I = np.empty((levels, na, glow.size), dtype=np.float32)
    for k in range(levels):
        I[k] = glow[None, :] * (1.0 + 0.1 * rng.uniform(-1, 1, (na, glow.size))) * 0.995 ** k
    return I, (0.9 * I).astype(np.float32)
