"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than its own formulas: the
paper's printed numbers, closed forms, quadrature of the defining integrals,
invariants of the physics, a library linear solve, and an independent brute-force
ray tracer.  None needs a GPU.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import workloads as W
from oracle import C0_MM_PER_NS, RING_DEPTH
from oracle.healpix import ring_directions, ring_z_phi, pixel_weight
from oracle.phase import henyey_greenstein, phase_matrix, mean_cosine
from oracle.geometry import RayLattice
from oracle.bruteforce import traced_upwind
from oracle.cones import cone_fractions
from oracle.solver import (Solver, Model, ray_weights, time_step, source_amplitudes,
                           source_iteration, FLOOR)
import oracle.solver as OS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- HEALPix (§2.1)

def test_healpix_base_pixels_nside1():
    """N_side = 1: the 12 HEALPix base pixels (4 at z=2/3, phi=pi/4+k pi/2; 4 at z=0,
    phi=k pi/2; 4 at z=-2/3), the textbook layout of the scheme."""
    z, phi = ring_z_phi(1)
    assert z.size == 12
    np.testing.assert_allclose(z[:4], 2 / 3, atol=1e-15)
    np.testing.assert_allclose(z[4:8], 0.0, atol=1e-15)
    np.testing.assert_allclose(z[8:], -2 / 3, atol=1e-15)
    np.testing.assert_allclose(np.sort(phi[:4]), np.pi / 4 + np.arange(4) * np.pi / 2, atol=1e-14)
    np.testing.assert_allclose(np.sort(np.mod(phi[4:8], 2 * np.pi)), np.arange(4) * np.pi / 2,
                               atol=1e-14)


@pytest.mark.parametrize("nside", [1, 2, 4, 16])
def test_healpix_equal_area_rings(nside):
    """Equal-area property: the cap above ring i's centre, 2 pi (1 - z_i), holds the
    pixels of the rings before it plus half of ring i."""
    z, _ = ring_z_phi(nside)
    assert z.size == 12 * nside * nside
    rings, counts = np.unique(-z, return_counts=True)
    w = pixel_weight(nside)
    above = 0
    for zr, cnt in zip(-rings, counts):
        assert 2 * np.pi * (1 - zr) == pytest.approx(w * (above + cnt / 2), rel=1e-13, abs=1e-13)
        above += cnt
    d = ring_directions(nside)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    # antipodal symmetry of the pixel set
    dots = d @ (-d).T
    assert np.all(np.max(dots, axis=1) > 1 - 1e-12)


def test_fiducial_angle_counts():
    """§2.1: 3072 RT bins (N_side 16) coarse-grained by 16 to 192 (N_side 4)."""
    assert ring_directions(16).shape[0] == 3072
    assert ring_directions(4).shape[0] == 3072 // 16


# ---------------------------------------------------------------- phase function (Eqs. 11-12)

@pytest.mark.parametrize("g", [0.0, 0.5, 0.9, -0.3])
def test_hg_normalisation_and_mean_cosine(g):
    """Eq. 11 is normalised to one over the sphere and has mean cosine g (text under
    Eq. 1 and Eq. 11), checked by 1-D quadrature over mu."""
    norm = 2 * np.pi * integrate.quad(lambda m: henyey_greenstein(m, g), -1, 1, epsabs=1e-14,
                                      epsrel=1e-13, limit=200)[0]
    mcos = 2 * np.pi * integrate.quad(lambda m: m * henyey_greenstein(m, g), -1, 1,
                                      epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    assert norm == pytest.approx(1.0, abs=1e-11)
    assert mcos == pytest.approx(g, abs=1e-11)


@pytest.mark.parametrize("nside", [1, 2, 4])
@pytest.mark.parametrize("g", [0.9, 0.3])
def test_phase_matrix_stochastic_symmetric_meancos(nside, g):
    P = phase_matrix(nside, g)
    d = ring_directions(nside)
    assert np.all(P >= 0)
    np.testing.assert_allclose(P, P.T, atol=1e-15)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-13)
    np.testing.assert_allclose(P.sum(axis=0), 1.0, atol=1e-13)
    assert mean_cosine(P, d) == pytest.approx(g, abs=1e-12)
    # an isotropic field scatters into an isotropic field
    np.testing.assert_allclose(P @ np.ones(P.shape[0]), 1.0, atol=1e-13)


def test_phase_matrix_isotropic_limit():
    """g = 0: every direction scatters equally into all N_a bins."""
    P = phase_matrix(2, 0.0)
    np.testing.assert_array_equal(P, np.full((48, 48), 1.0 / 48))


def test_phase_matrix_forward_peaked():
    """g = 0.9 is forward peaked: every row's largest entry is its own direction."""
    P = phase_matrix(4, 0.9)
    assert np.all(np.argmax(P, axis=1) == np.arange(P.shape[0]))


# ---------------------------------------------------------------- Eq. 9 weights

@pytest.mark.parametrize("tau", [1e-6, 5e-4, 1e-3, 2e-3, 0.05, 0.7, 3.0, 15.0])
def test_eq9_matches_quadrature_of_eq7_eq8(tau):
    """Eq. 9 is Eq. 7 with the linear source of Eq. 8 integrated exactly: compare with
    numerical quadrature of the integral for arbitrary I0, S0, S1."""
    rng = np.random.default_rng(1)
    I0, S0, S1 = rng.uniform(0.1, 2.0, 3)
    integrand = lambda s: ((1 - s / tau) * S0 + (s / tau) * S1) * math.exp(s - tau)
    ref = I0 * math.exp(-tau) + integrate.quad(integrand, 0, tau, epsabs=1e-15, epsrel=1e-13)[0]
    T, b0, b1 = ray_weights(np.array([tau]))
    got = I0 * T[0] + S0 * b0[0] + S1 * b1[0]
    assert got == pytest.approx(ref, rel=1e-11)


def test_eq9_identities():
    """T + b0 + b1 = 1 (a constant source is a fixed point), S0 = S1 reduces to the
    constant-source formal solution, all weights are non-negative."""
    x = np.concatenate([np.logspace(-8, 2, 400), [0.0]])
    T, b0, b1 = ray_weights(x)
    np.testing.assert_allclose(T + b0 + b1, 1.0, atol=2e-15)
    S = 0.37
    np.testing.assert_allclose(S * (b0 + b1), S * (1 - np.exp(-x)), atol=1e-15)
    assert np.all(b0 >= 0) and np.all(b1 >= 0) and np.all(T >= 0)
    assert b0[-1] == 0 and b1[-1] == 0 and T[-1] == 1


# ---------------------------------------------------------------- time step (§2.2, §3.1)

def test_time_step_rule_matches_printed_values():
    cases = json.load(open(os.path.join(GOLDEN, "paper_time_steps.json")))["cases"]
    for c in cases:
        dt = time_step(c["courant"], c["dx_mm"], c["n"])
        assert float("%.*g" % (c["printed_digits"], dt)) == c["printed_dt_ns"], c["what"]
        if "printed_steps" in c:
            assert c["run_ns"] / dt == pytest.approx(c["printed_steps"], rel=3e-3)


# ---------------------------------------------------------------- ray lattice vs brute force

@pytest.mark.parametrize("nside", [1, 2])
@pytest.mark.parametrize("shape", [(3, 4, 5), (5, 4, 3), (2, 7, 3), (4, 4, 4)])
def test_lattice_matches_bruteforce_tracer(nside, shape):
    d = ring_directions(nside)
    up, visits = traced_upwind(d, shape, 1.0)
    lat = RayLattice(d, shape, 1.0)
    ours = np.stack([lat.upwind_index(i) for i in range(len(d))])
    assert np.all(visits == 1), "every voxel holds exactly one ray sample per direction"
    np.testing.assert_array_equal(ours, up)


def test_lattice_periodic_is_a_permutation():
    """With periodic wrap every voxel is the upwind of exactly one voxel."""
    d = ring_directions(2)
    lat = RayLattice(d, (6, 5, 4), 1.0, periodic=True)
    for i in range(len(d)):
        u = lat.upwind_index(i)
        assert np.array_equal(np.sort(u), np.arange(u.size))


# ---------------------------------------------------------------- transport pins

def _beam_problem(delta, mua=0.0, mus=0.0, shape=(8, 4, 4), d0=0):
    """A single-direction beam entering the -z face, with c0 dt chosen so that the
    retarded delay in the medium (n = 1) is ``delta`` steps."""
    nz, ny, nx = shape
    dirs = ring_directions(2)
    ds = 1.0 / dirs[d0, 2]
    p = W.homogeneous(nx, ny, nz, 2, mua, mus, g=0.9, nidx=1.0, steps=0)
    p["n_ref"] = 1.0
    p["courant"] = ds / delta
    amp = np.zeros(48)
    amp[d0] = 3.0
    p["source"] = dict(face=4, u_mm=1.2, v_mm=1.2, pulse_steps=1, amp=amp)
    return p, dirs[d0], ds


def _ray_voxels(omega, ds, shape, start_xy=(1, 1)):
    """Voxels crossed by the beam, by stepping the 3-D point (independent of the lattice)."""
    nz, ny, nx = shape
    pos = np.array([start_xy[0] + 0.5, start_xy[1] + 0.5, 0.5])
    out = []
    for k in range(nz):
        idx = np.floor(pos + 1e-9).astype(int)
        if not (0 <= idx[0] < nx and 0 <= idx[1] < ny):
            break
        out.append((idx[2] * ny + idx[1]) * nx + idx[0])
        pos = pos + ds * omega
    return out


def test_vacuum_pulse_integer_delay_is_exact():
    """§2.2 (1-D pulse): the scheme keeps a pulse's shape in vacuum.  With an integer
    delay the pulse moves one ray sample per delta steps with no loss and no spread."""
    p, om, ds = _beam_problem(2.0)
    s = Solver(p)
    path = _ray_voxels(om, ds, (8, 4, 4))
    assert len(path) >= 4
    for n in range(2 * len(path) + 3):
        s.step()
        I = s.level("I")[0]
        k = n // 2 - 1
        expect = np.zeros_like(I)
        if n % 2 == 0 and 0 <= k < len(path):
            expect[path[k]] = 3.0
        np.testing.assert_allclose(I, expect, atol=1e-12)


def test_vacuum_pulse_fractional_delay_centroid():
    """With a non-integer delay the time interpolation spreads the pulse but keeps its
    arrival-time centroid at (k+1) delta exactly and its integral unchanged."""
    delta = 2.3
    p, om, ds = _beam_problem(delta)
    s = Solver(p)
    path = _ray_voxels(om, ds, (8, 4, 4))
    hist = []
    for n in range(40):
        s.step()
        hist.append(s.level("I")[0][path])
    hist = np.array(hist)
    t = np.arange(40)[:, None]
    tot = hist.sum(axis=0)
    np.testing.assert_allclose(tot, 3.0, rtol=1e-12)
    np.testing.assert_allclose((hist * t).sum(axis=0) / tot, (np.arange(len(path)) + 1) * delta,
                               rtol=1e-12)


def test_beer_lambert_pure_absorber():
    """Pure absorber (mu_s = 0): the transmitted beam is I0 exp(-mu_a L) along the ray."""
    mua = 0.3
    p, om, ds = _beam_problem(2.0, mua=mua)
    s = Solver(p)
    path = _ray_voxels(om, ds, (8, 4, 4))
    acc = np.zeros(len(path))
    for n in range(2 * len(path) + 3):
        s.step()
        acc += s.level("I")[0][path]
    mua_stored = float(np.float32(mua))  # the optics maps are float32 inputs
    np.testing.assert_allclose(acc, 3.0 * np.exp(-mua_stored * ds * (np.arange(len(path)) + 1)),
                               rtol=1e-12)


def test_opaque_voxel_leaves_exact_shadow():
    """§2.2 (absorbing grid in the beam): behind an opaque voxel nothing passes."""
    p, om, ds = _beam_problem(2.0)
    path = _ray_voxels(om, ds, (8, 4, 4))
    mua = p["mua"].ravel()
    mua[path[1]] = 1.0e3
    p["mua"] = mua.reshape(p["mua"].shape)
    s = Solver(p)
    for n in range(2 * len(path) + 3):
        s.step()
        I = s.level("I")[0]
        assert np.all(I[path[2:]] == 0.0)


# ---------------------------------------------------------------- source iteration (Eq. 12)

def test_source_iteration_matches_direct_solve():
    """The iterated source equals the per-voxel fixed point S = (1 - a P B1)^-1 a P Q,
    solved here by a library linear solve, within the stop bound."""
    p = W.config_small(steps=12, tol=1e-12)
    s = Solver(p)
    for _ in range(11):
        s.step()
    m, seg, n = s.m, s.seg, s.n
    Q = OS._retarded(s._hist, seg, n, "I", m) * seg["T"] + OS._retarded(s._hist, seg, n, "S", m) * seg["b0"]
    S_prev = s.S[(n - 1) % RING_DEPTH]
    S, it = source_iteration(m, Q, seg["b1"], S_prev, m.albedo, np.abs(S_prev).max())
    rng = np.random.default_rng(0)
    live = np.nonzero(np.abs(Q).max(axis=0) > 1e-3 * np.abs(Q).max())[0]
    for v in rng.choice(live, 25, replace=False):
        A = np.eye(m.na) - m.albedo[v] * m.P * seg["b1"][None, :, v]
        ref = np.linalg.solve(A, m.albedo[v] * (m.P @ Q[:, v]))
        scale = max(np.abs(ref).max(), FLOOR * np.abs(S_prev).max())
        assert np.abs(S[:, v] - ref).max() <= 1.01e-12 * scale + 1e-15 * np.abs(ref).max() * 100


def test_isotropic_state_is_invariant_without_absorption():
    """a = 1, periodic box, isotropic uniform intensity: scattering only redistributes,
    so the state is a fixed point of the scheme (T + b0 + b1 = 1, P rows sum to 1)."""
    p = W.homogeneous(4, 5, 3, 2, 0.0, 7.0, boundary="periodic", tol=1e-13)
    s = Solver(p, init=(np.ones((48, 1)), np.ones((48, 1))))
    for _ in range(12):
        s.step()
    np.testing.assert_allclose(s.level("I"), 1.0, atol=1e-11)
    np.testing.assert_allclose(s.level("S"), 1.0, atol=1e-11)


# ---------------------------------------------------------------- source and cones (§3.1)

def test_cone_fractions_sum_and_symmetry():
    d = ring_directions(2)
    a = cone_fractions(d, 4, 15.0, inward=True)
    assert a.sum() == pytest.approx(1.0, abs=1e-15)
    nz = np.nonzero(a)[0]
    assert list(nz) == [0, 1, 2, 3]  # the four pixels of the first ring around +z
    np.testing.assert_allclose(a[nz], 0.25, atol=1e-15)
    for face in range(6):
        for inward in (True, False):
            assert cone_fractions(ring_directions(4), face, 15.0, inward).sum() == pytest.approx(1.0)


def test_source_injects_exactly_the_pulse_energy():
    """The inflow through the source voxel carries exactly E over the pulse."""
    d = ring_directions(4)
    w = pixel_weight(4)
    for face in range(6):
        amp = source_amplitudes(d, w, face, 15.0, 1.0, 2.3e-3, 3, 0.7)
        ax = face // 2
        flux = amp * w * np.abs(d[:, ax]) * 1.0 * 2.3e-3 * 3
        assert flux.sum() == pytest.approx(0.7, rel=1e-14)


# ---------------------------------------------------------------- Fresnel / Snell (Eqs. 13-14)

from oracle.fresnel import fresnel_R, fresnel_R_eq14, reflect_refract, apply_interfaces


def test_fresnel_normal_incidence_and_critical_angle():
    """Textbook limits: R(0) = ((n1-n2)/(n1+n2))^2 (0.027778 for 1.4 -> 1.0); total
    reflection from the critical angle asin(n2/n1) = 45.585 deg on."""
    assert fresnel_R(1.4, 1.0, 1.0) == pytest.approx((0.4 / 2.4) ** 2, rel=1e-14)
    assert fresnel_R(1.0, 1.4, 1.0) == pytest.approx((0.4 / 2.4) ** 2, rel=1e-14)
    tc = np.arcsin(1.0 / 1.4)
    assert np.degrees(tc) == pytest.approx(45.585, abs=1e-3)
    assert fresnel_R(1.4, 1.0, np.cos(tc + 1e-6)) == 1.0
    assert fresnel_R(1.4, 1.0, np.cos(tc - 1e-3)) < 1.0
    assert fresnel_R(1.0, 1.4, 1e-9) == pytest.approx(1.0, abs=1e-6)  # grazing


@pytest.mark.parametrize("n1,n2", [(1.4, 1.0), (1.0, 1.4), (1.51, 1.33)])
def test_fresnel_matches_eq14_form(n1, n2):
    """The cosine form used by the solver equals Eq. 14 as printed (sin/tan form)."""
    tmax = np.arcsin(min(1.0, n2 / n1)) - 1e-3 if n1 > n2 else np.pi / 2 - 1e-3
    th = np.linspace(1e-3, tmax, 50)
    np.testing.assert_allclose(fresnel_R(n1, n2, np.cos(th)), fresnel_R_eq14(n1, n2, th), rtol=1e-10)


def test_snell_direction():
    """Transmitted direction: unit length, in the plane of incidence, n1 sin1 = n2 sin2."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        om = rng.normal(size=3); om /= np.linalg.norm(om)
        m = rng.normal(size=3); m /= np.linalg.norm(m)
        n1, n2 = 1.0, 1.4
        R, om_r, om_t = reflect_refract(om, m, n1, n2)
        assert np.linalg.norm(om_r) == pytest.approx(1.0, abs=1e-12)
        assert np.dot(om_r, m) == pytest.approx(-np.dot(om, m), abs=1e-12)
        assert np.linalg.norm(om_t) == pytest.approx(1.0, abs=1e-12)
        assert np.dot(np.cross(om, m), om_t) == pytest.approx(0.0, abs=1e-12)
        s1 = np.linalg.norm(np.cross(om, m))
        s2 = np.linalg.norm(np.cross(om_t, m))
        assert n1 * s1 == pytest.approx(n2 * s2, abs=1e-12)
        assert np.sign(np.dot(om_t, m)) == np.sign(np.dot(om, m))


def test_interface_redistribution_at_a_planar_step():
    """A plane index step (n = 1.0 below z = 4, 1.4 from z = 4 up): every segment whose
    upwind sample lies across the step is split into the mirror image of its direction
    (weight R of Eq. 14 as printed) and the Snell direction written out by hand (weight
    1 - R, none under total internal reflection), each snapped to the pixel with the
    largest dot product by brute force (the reading's tie rule: lowest index within 1e-12);
    no other segment is touched."""
    nx, ny, nz, k0 = 6, 6, 8, 4
    p = W.homogeneous(nx, ny, nz, 2, 0.01, 1.0, steps=1)
    nmap = np.full((nz, ny, nx), 1.0)
    nmap[k0:] = 1.4
    p["nidx"] = nmap.astype(np.float32)
    p["fresnel"] = True
    m = Model(p)
    n = m.nidx
    expected = {}
    for j in range(m.na):
        up = m.lat.upwind_index(j)
        for v in range(m.nv):
            if up[v] < 0 or n[up[v]] == n[v]:
                continue
            n1, n2 = float(n[up[v]]), float(n[v])
            ox, oy, oz = m.dirs[j]
            cos1 = abs(oz)
            th1 = math.acos(cos1)
            eta = n1 / n2
            sin2 = eta * eta * (1.0 - cos1 * cos1)
            refl = np.array([ox, oy, -oz])
            if sin2 >= 1.0:
                R, trans = 1.0, None
            else:
                R = float(fresnel_R_eq14(n1, n2, th1))
                trans = np.array([eta * ox, eta * oy, math.copysign(math.sqrt(1.0 - sin2), oz)])

            def snap(vec):  # ties (mirror-symmetric pixel pairs) go to the lowest index
                dots = m.dirs @ vec
                return min(i for i in range(m.na) if dots[i] >= dots.max() - 1e-12)
            outs = [(snap(refl), R)]
            if trans is not None:
                outs.append((snap(trans), 1.0 - R))
            expected.setdefault(v, {})[j] = outs
    assert expected and set(expected) == set(m.interfaces)
    kinds = {len(outs) for cols in expected.values() for outs in cols.values()}
    assert kinds == {1, 2}  # both total internal reflection and transmission occur
    zs = {v // (nx * ny) for v in expected}
    assert zs <= {k0 - 1, k0}
    for v, cols in expected.items():
        assert set(cols) == set(m.interfaces[v])
        for j, outs in cols.items():
            got = m.interfaces[v][j]
            assert [d for d, _ in got] == [d for d, _ in outs]
            np.testing.assert_allclose([w for _, w in got], [w for _, w in outs], rtol=0, atol=1e-12)


def test_interface_redistribution_conserves_photons():
    """The interface operator is column-stochastic: the sum over directions of Q at every
    interface voxel is unchanged, and it moves intensity only where n changes."""
    p = W.config_hetero(steps=1, precision="fp32", nx=24, ny=24, nz=8, nside=2, scale=0.25)
    m = Model(p)
    assert len(m.interfaces) > 0
    rng = np.random.default_rng(0)
    Q = rng.uniform(0, 1, (m.na, m.nv))
    Q2 = apply_interfaces(m.interfaces, Q.copy())
    np.testing.assert_allclose(Q2.sum(axis=0), Q.sum(axis=0), rtol=1e-13)
    moved = np.nonzero(np.abs(Q2 - Q).max(axis=0) > 0)[0]
    assert set(moved) <= set(m.interfaces.keys())
    n = m.nidx
    for v in m.interfaces:
        z, rem = divmod(v, p["nx"] * p["ny"])
        y, x = divmod(rem, p["nx"])
        nb = [n[v + o] for o, ok in ((1, x + 1 < p["nx"]), (-1, x > 0), (p["nx"], y + 1 < p["ny"]),
                                        (-p["nx"], y > 0)) if ok]
        assert any(b != n[v] for b in nb)
