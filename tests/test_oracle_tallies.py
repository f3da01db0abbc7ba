"""Pins of the oracle's tallies and boundary modes: detector curves, photon accounting,
the closed-box recurrence and the mirror faces.

Each expected value here comes from its own arithmetic: a hand-derived bin table, the
binomial law of a vacuum pulse's arrival on the lattice, a closed-form solid angle, a
0-D recurrence solved with a library linear solve, or an exact shift on a mirror
cavity.  A plausible mistake in a weight, an index, a sign or a time level of the
oracle's tally code fails one of them.  None needs a GPU.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import C0_MM_PER_NS
from oracle.healpix import ring_directions
from oracle.phase import phase_matrix
from oracle.solver import (Solver, Model, step_bin, time_step, detector_weights, disk_voxels,
                           energy_density, reflection_table)

DT_PS = 0.7 / C0_MM_PER_NS * 1e3  # c0 dt / n_ref = 0.5 voxel of 1 mm at n_ref = 1.4


# ---------------------------------------------------------------- detector bins (§3.1)

# First step of each 10 ps bin at dt = 0.7 mm / c0 = 2.334949 ps, derived by hand: step n
# covers [n dt, (n+1) dt) and is binned at its midpoint, so bin k starts at the first n
# with (n + 1/2) * 2.334949 >= 10 k, i.e. n >= 10 k / 2.334949 - 1/2:
#   k:      1      2      3      4      5      6      7      8      9     10     11     12
#   bound: 3.78   8.07  12.35  16.63  20.91  25.20  29.48  33.76  38.04  42.33  46.61  50.89
BIN_STARTS = [0, 4, 9, 13, 17, 21, 26, 30, 34, 39, 43, 47, 51]
# the last step of a 1500-step run lands in bin 350 (1499.5 * 2.334949 / 10 = 350.13)
LAST_STEP_BIN = (1499, 350)


def test_step_bin_matches_hand_table():
    dt = time_step(0.5, 1.0, 1.4)
    assert dt * 1e3 == pytest.approx(2.334949, abs=1e-6)
    for k in range(len(BIN_STARTS) - 1):
        for n in range(BIN_STARTS[k], BIN_STARTS[k + 1]):
            assert step_bin(n, dt, 10e-3) == k, (n, k)
    assert step_bin(LAST_STEP_BIN[0], dt, 10e-3) == LAST_STEP_BIN[1]


def test_detector_weight_of_a_single_ring():
    """N_side 2, 15-degree cap around +z: the four pixels of the first ring (z = 11/12)
    share the cap equally, so each weight is (1/4) * 2 pi (1 - cos 15 deg) * 11/12 (the
    acceptance fraction, the cap's solid angle and Omega . n_out), and no other
    direction counts."""
    d = ring_directions(2)
    wgt = detector_weights(d, 5, 15.0)
    expect = 0.25 * 2 * math.pi * (1 - math.cos(math.radians(15.0))) * 11.0 / 12.0
    np.testing.assert_allclose(wgt[:4], expect, rtol=1e-14)
    assert np.all(wgt[4:] == 0)


@pytest.mark.parametrize("half_angle", [15.0, 45.0, 80.0])
def test_detector_weights_project_the_cap(half_angle):
    """Summed over directions the weights approximate the cap's projected solid angle
    int_cap cos dOmega = pi sin^2(theta_c) (the flux an isotropic unit radiance sends
    through unit area into the cap).  The nearest-centre shares of 3072 directions
    reproduce it to 5e-4 (bar 1e-3); a missing cosine, a wrong cap solid angle or an inward cone
    is off by 3-50%."""
    d = ring_directions(16)
    total = detector_weights(d, 1, half_angle).sum()
    assert total == pytest.approx(math.pi * math.sin(math.radians(half_angle)) ** 2, rel=1e-3)


def test_disk_voxels_lie_on_the_face_and_in_the_disk():
    """Every voxel of a disk is on the named face, its centre is within the radius, and
    the count is the number of voxel centres (i + 1/2, j + 1/2) in the disk, counted
    here by brute force."""
    shape = (6, 7, 9)  # nz, ny, nx
    nz, ny, nx = shape
    for face, (u, v, r) in enumerate([(3.2, 2.0, 1.6), (4.5, 1.5, 2.1), (2.0, 3.0, 1.0),
                                      (5.5, 2.5, 2.5), (3.0, 4.0, 2.2), (7.5, 6.5, 0.5)]):
        vox = disk_voxels(shape, 1.0, face, u, v, r)
        ax = face // 2
        n_uv = [m for a, m in enumerate((nx, ny, nz)) if a != ax]
        want = sum(1 for i in range(n_uv[0]) for j in range(n_uv[1])
                   if (i + 0.5 - u) ** 2 + (j + 0.5 - v) ** 2 <= r * r + 1e-12)
        assert len(vox) == want > 0
        for f in vox:
            x, y, z = f % nx, (f // nx) % ny, f // (nx * ny)
            c = (x, y, z)
            assert c[ax] == (0 if face % 2 == 0 else (nx, ny, nz)[ax] - 1)
            cu, cv = [c[a] for a in range(3) if a != ax]
            assert (cu + 0.5 - u) ** 2 + (cv + 0.5 - v) ** 2 <= r * r + 1e-12


def _vacuum_beam(detectors, steps=52):
    """16^3 box with n = 1.4 and no interaction; a one-step pulse into the 15-degree cone
    at the -z face voxel (5, 9); N_side 2."""
    p = W.homogeneous(16, 16, 16, 2, 0.0, 0.0, steps=steps)
    p["source"] = dict(face=4, u_mm=5.0, v_mm=9.0, half_angle_deg=15.0, pulse_steps=1,
                       energy=1.0)
    p["detectors"] = detectors
    p["nbins"] = 14
    return Solver(p).run(steps)


def test_detector_curves_of_a_vacuum_beam():
    """The cone's four directions (the first ring, 23.56 degrees from +z, t = +-0.3083
    voxels per slab) cross 16 slabs with delay 24/11 = 2 + 2/11 steps each, so a beam's
    exit sample at the +z face carries the pulse at step 32 + B, B ~ Binomial(16, 2/11)
    (each segment's linear interpolation in time splits what it passes on between
    delays 2 and 3).  A one-voxel detector on the exit spot of direction
    (+x, +y), at (5 + 5, 9 + 5), sees E0 * (1/4 of the source) * (1/4 of the detector
    cap) * Omega_cap / w in total, binned by the hand table; the u/v-swapped voxel
    (14, 10) sees nothing; a detector over the whole face sees all four beams."""
    omega_cap = 2 * math.pi * (1 - math.cos(math.radians(15.0)))
    w = 4 * math.pi / 48
    dets = [dict(face=5, u_mm=10.5, v_mm=14.5, radius_mm=0.5, half_angle_deg=15.0),
            dict(face=5, u_mm=14.5, v_mm=10.5, radius_mm=0.5, half_angle_deg=15.0),
            dict(face=5, u_mm=8.0, v_mm=8.0, radius_mm=100.0, half_angle_deg=15.0)]
    r = _vacuum_beam(dets)
    E = r["detectors"]
    one = omega_cap / (16 * w)
    # the map holds n in FP32 (1.39999998), so the delay is 12/11 * n / 0.7 = 24/11 - 2e-7
    f = 12.0 / 11.0 * float(np.float32(1.4)) / 0.7 - 2.0
    assert f == pytest.approx(2.0 / 11.0, abs=1e-6)
    expect = np.zeros(14)
    for b in range(17):
        n = 32 + b
        k = max(i for i, s in enumerate(BIN_STARTS) if s <= n)
        expect[k] += one * math.comb(16, b) * f**b * (1 - f) ** (16 - b)
    np.testing.assert_allclose(E[0], expect, rtol=1e-12, atol=1e-15 * one)
    assert np.all(E[1] == 0)
    assert E[2].sum() == pytest.approx(4 * one, rel=1e-12)
    assert one == pytest.approx(1.5 * (1 - math.cos(math.radians(15.0))), rel=1e-14)


# ---------------------------------------------------------------- photon accounting

def test_vacuum_budget_closes_exactly():
    """With no interaction every injected photon leaves: after the pulse has crossed the
    box the escaped energy sums to the pulse energy, the residual is zero and nothing was
    absorbed (time integrals of the flux along a ray are conserved exactly, since the
    interpolation weights of each segment sum to one, and all rays of the cone leave
    through the +z face, where the face flux w (Omega . n) I h^2 dt is the ray's flux)."""
    p = W.config_small(steps=60)
    p["mus"][:] = 0.0
    p["mua"][:] = 0.0
    r = Solver(p).run(60)
    assert r["injected"].sum() == pytest.approx(1.0, rel=1e-14)
    assert r["injected"][0] == r["injected"].sum()
    assert r["escaped"].sum() == pytest.approx(1.0, rel=1e-12)
    assert np.all(r["absorbed"] == 0)
    assert r["energy"][-1] == 0
    assert abs(r["residual"][-1]) < 1e-12


def test_energy_density_of_isotropic_unit_radiance():
    """u = (n / c0) * 4 pi for a unit isotropic radiance, and h^3 sum_v u = N."""
    p = W.homogeneous(3, 4, 2, 2, 0.01, 1.0)
    p["nidx"][0] = 1.2
    m = Model(p)
    I = np.ones((m.na, m.nv))
    u = energy_density(m, I)
    np.testing.assert_allclose(u, m.nidx * 4 * math.pi / C0_MM_PER_NS, rtol=1e-14)


def _recurrence(nside, g, mua, mus, nidx, I0, steps, h=1.0, courant=0.5, n_ref=1.4):
    """The closed box reduced to one voxel.  In a spatially uniform periodic (or
    reflection-symmetric mirror) box every voxel holds the same state, so each upwind
    sample is a copy of the voxel itself and Eq. 10 becomes a recurrence over the stored
    levels of one N_a-vector.  Solved here with its own arithmetic: weights from the
    closed forms of Eq. 9, the delay ds n / (c0 dt) split into floor and fraction, the
    levels before 0 held at (I0, a P I0), and a library linear solve of
    (1 - a P diag b1) S = a P Q per step (no iteration).  Returns I per step."""
    d = ring_directions(nside)
    P = phase_matrix(nside, g)
    na = d.shape[0]
    mut = mua + mus
    a = mus / mut
    dt = courant * h * n_ref / C0_MM_PER_NS
    ds = h / np.max(np.abs(d), axis=1)
    x = mut * ds
    T = np.exp(-x)
    b0 = (1.0 - (1.0 + x) * T) / x
    b1 = (x - 1.0 + T) / x
    delay = ds * nidx / (C0_MM_PER_NS * dt)
    m = np.floor(delay).astype(int)
    f = delay - m
    S0 = a * (P @ I0)
    lev = {k: (I0.copy(), S0.copy()) for k in range(-6, 0)}
    A = np.eye(na) - a * P * b1[None, :]
    out = []
    for n in range(steps):
        DI = np.array([(1 - f[j]) * lev[n - m[j]][0][j] + f[j] * lev[n - m[j] - 1][0][j]
                       for j in range(na)])
        DS = np.array([(1 - f[j]) * lev[n - m[j]][1][j] + f[j] * lev[n - m[j] - 1][1][j]
                       for j in range(na)])
        Q = T * DI + b0 * DS
        S = np.linalg.solve(A, a * (P @ Q))
        I = Q + b1 * S
        lev[n] = (I, S)
        out.append(I)
    return np.array(out), dt


@pytest.mark.parametrize("boundary", ["periodic", "mirror"])
def test_closed_box_matches_zero_d_recurrence(boundary):
    """Closed box (exact discrete pin of the photon decay): the 3-D oracle in a uniform
    box, started from a uniform but anisotropic state, equals the one-voxel recurrence
    step by step to 1e-12 in every field value, in N(t), in the absorbed energy and in the
    residual.  The state is symmetric under reflection in each face, so the mirror box
    stays uniform too.  A swapped interpolation weight, a wrong delay, a dropped b0 or b1
    term or a wrong energy or absorption formula fails it; the residual is the scheme's
    own departure from photon balance (T, b0, b1 make the per-step factor differ slightly
    from exp(-mu_a c dt / n)), identical in both."""
    mua, mus, nidx, g = 0.02, 5.0, 1.4, 0.8
    d = ring_directions(2)
    if boundary == "periodic":
        I0 = 1.0 + 0.3 * d[:, 2] + 0.2 * d[:, 0] * d[:, 1] + 0.1 * d[:, 0]
    else:
        I0 = 1.0 + 0.3 * d[:, 2] ** 2 + 0.2 * d[:, 0] ** 2 * d[:, 1] ** 2
    steps = 40
    # the maps hold FP32 values; the recurrence takes the same numbers
    mua32, mus32, n32 = (float(np.float32(v)) for v in (mua, mus, nidx))
    ref, dt = _recurrence(2, g, mua32, mus32, n32, I0, steps)
    p = W.homogeneous(3, 4, 5, 2, mua, mus, g=g, nidx=nidx, boundary=boundary, tol=1e-14)
    a = mus32 / (mua32 + mus32)
    P = phase_matrix(2, g)
    s = Solver(p, init=(I0[:, None], (a * (P @ I0))[:, None]))
    hist = []
    for _ in range(steps):
        s.step()
        hist.append(s.level("I"))
    r = s.result()
    nv = 60
    w = 4 * math.pi / 48
    for n in range(steps):
        np.testing.assert_allclose(hist[n], np.broadcast_to(ref[n][:, None], hist[n].shape),
                                   rtol=1e-12, atol=0)
    N_ref = nv * n32 / C0_MM_PER_NS * w * ref.sum(axis=1)
    ab_ref = nv * dt * mua32 * w * ref.sum(axis=1)
    N_init = nv * n32 / C0_MM_PER_NS * w * I0.sum()
    res_ref = N_init - np.cumsum(ab_ref) - N_ref
    np.testing.assert_allclose(r["energy"], N_ref, rtol=1e-12)
    np.testing.assert_allclose(r["absorbed"], ab_ref, rtol=1e-12)
    assert np.all(r["escaped"] == 0)
    np.testing.assert_allclose(r["residual"], res_ref, rtol=1e-9, atol=1e-12 * N_init)
    # the decay follows mu_a c / n only to the scheme's accuracy: 1e-2 here, not exactly
    rate = -np.log(N_ref[-1] / N_ref[-11]) / (10 * dt)
    assert rate == pytest.approx(mua * C0_MM_PER_NS / nidx, rel=2e-2)


def test_isotropic_state_is_invariant_in_a_mirror_box():
    """a = 1 and a unit isotropic state: every image is the same unit state, so the mirror
    box keeps it exactly (any photon leaking at a face would lower it)."""
    p = W.homogeneous(4, 3, 5, 2, 0.0, 7.0, boundary="mirror", tol=1e-13)
    s = Solver(p, init=(np.ones((48, 1)), np.ones((48, 1))))
    for _ in range(12):
        s.step()
    np.testing.assert_allclose(s.level("I"), 1.0, atol=1e-11)
    assert np.all(np.array(s.escaped) == 0)


def test_mirror_cavity_shifts_a_beam_exactly():
    """A 1-D mirror cavity: N_side 1 has directions exactly along +-x (no transverse
    offsets; n = 1 and c0 dt = h / 2 give a delay of 2 steps per voxel).  With no interaction and the +x beam
    filling the box before step 0, light runs around the loop +x cells (x = 0..N-1) ->
    reflected at the +x face into -x cells -> reflected at the -x face back into +x, one
    cell per two steps: loop position p (+x cell x: p = x; -x cell x: p = 2N - 1 - x)
    holds at step n the initial pattern shifted by floor(n / 2) + 1.  Taking the wrong
    reflected direction or the wrong image voxel breaks the loop; the photon number stays
    exactly constant and nothing escapes."""
    N = 6
    p = W.homogeneous(N, 2, 3, 1, 0.0, 0.0, nidx=1.0, boundary="mirror")
    p["n_ref"] = 1.0  # with courant 0.5: c0 dt = h / 2, a delay of 2 steps per voxel
    d = ring_directions(1)
    px = int(np.argmax(d[:, 0]))
    mx = int(np.argmin(d[:, 0]))
    assert d[px, 0] == pytest.approx(1.0) and d[mx, 0] == pytest.approx(-1.0)
    I0 = np.zeros((12, 1))
    I0[px] = 1.0
    s = Solver(p, init=(I0, np.zeros((12, 1))))
    init = np.r_[np.ones(N), np.zeros(N)]
    nv = N * 6
    for n in range(4 * N):
        s.step()
        I = s.level("I").reshape(12, 3, 2, N)
        k = n // 2 + 1
        loop = np.roll(init, k)
        np.testing.assert_allclose(I[px], np.broadcast_to(loop[:N], (3, 2, N)), atol=1e-13)
        np.testing.assert_allclose(I[mx], np.broadcast_to(loop[N:][::-1], (3, 2, N)), atol=1e-13)
        others = [j for j in range(12) if j not in (px, mx)]
        assert np.all(I[others] == 0)
    E = np.array(s.energy)
    np.testing.assert_allclose(E, E[0], rtol=1e-13)
    # N of the 2N loop positions hold 1 in each of the 6 (y, z) columns
    assert E[0] == pytest.approx(nv / C0_MM_PER_NS * (4 * math.pi / 12), rel=1e-13)
    assert np.all(np.array(s.escaped) == 0)


def test_reflection_table_is_an_involution():
    for nside in (1, 2, 4):
        d = ring_directions(nside)
        R = reflection_table(d)
        for mask in range(8):
            s = np.array([-1.0 if (mask >> a) & 1 else 1.0 for a in range(3)])
            np.testing.assert_allclose(d[R[:, mask]], d * s[None, :], atol=1e-14)
            np.testing.assert_array_equal(R[R[:, mask], mask], np.arange(d.shape[0]))
