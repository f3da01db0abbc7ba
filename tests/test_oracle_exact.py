"""Pins of the exact per-voxel source function (S = M Q per optics class).

The operator is pinned to its defining fixed-point equation, and the solver to the
converged source iteration (itself pinned in test_oracle_pins.py) on a small phantom of
uniform regions with index interfaces.
"""
import numpy as np

import workloads as W
from oracle.exact import ExactSolver, exact_operator, optics_classes
from oracle.phase import phase_matrix
from oracle.solver import Model, Solver, ray_weights


def test_operator_solves_the_fixed_point():
    P = phase_matrix(2, 0.9)
    rng = np.random.default_rng(0)
    ds = 1.0 + 0.7 * rng.random(48)
    for mut, a in ((10.0, 0.999), (2.0, 0.5), (0.3, 0.9), (5.0, 0.0)):
        _, _, b1 = ray_weights(mut * ds)
        M = exact_operator(P, a, b1)
        Q = rng.random((48, 7))
        S = M @ Q
        assert np.max(np.abs(S - a * P @ (Q + b1[:, None] * S))) <= 1e-13 * max(1.0, np.max(np.abs(S)))
    assert not np.any(exact_operator(P, 0.0, b1))  # no scattering, no source


def test_isotropic_scattering_has_a_closed_form():
    """g = 0: every row of P is 1/N_a, so S is the same in every direction and the fixed
    point reduces to the scalar S = a mean(Q) / (1 - a mean(b1)) (b1 still varies with the
    ray spacing of each direction)."""
    P = phase_matrix(2, 0.0)
    np.testing.assert_allclose(P, np.full((48, 48), 1.0 / 48), rtol=1e-12)
    rng = np.random.default_rng(1)
    ds = 1.0 + 0.7 * rng.random(48)
    for mut, a in ((10.0, 0.999), (1.0, 0.6)):
        _, _, b1 = ray_weights(mut * ds)
        Q = rng.random((48, 5))
        S = exact_operator(P, a, b1) @ Q
        closed = a * Q.mean(axis=0) / (1.0 - a * b1.mean())
        np.testing.assert_allclose(S, np.broadcast_to(closed, S.shape), rtol=1e-11)


def phantom(nside=2, steps=12, tol=1e-13):
    """10 x 10 x 8 voxels: background mu_a 0.02, mu_s 2 /mm, n 1.4; an absorbing sphere
    (mu_a x 4, radius 2 mm); an air block (mu_a = mu_s = 0, n 1) with interfaces."""
    p = W.homogeneous(10, 10, 8, nside, 0.02, 2.0, g=0.9, steps=steps, tol=tol)
    p["max_iters"] = 20000
    zz, yy, xx = np.meshgrid(np.arange(8) + 0.5, np.arange(10) + 0.5, np.arange(10) + 0.5, indexing="ij")
    mua, mus, nid = (np.array(p[k], np.float32) for k in ("mua", "mus", "nidx"))
    sph = (xx - 6.5) ** 2 + (yy - 4.5) ** 2 + (zz - 3.5) ** 2 <= 4.0
    mua[sph] *= 4.0
    air = (xx > 2) & (xx < 4) & (yy > 5) & (yy < 8) & (zz > 2) & (zz < 5)
    mua[air] = 0.0
    mus[air] = 0.0
    nid[air] = 1.0
    p["mua"], p["mus"], p["nidx"], p["fresnel"] = mua, mus, nid, True
    p["source"] = dict(face=4, u_mm=5.0, v_mm=5.0, half_angle_deg=20.0, pulse_steps=2, energy=1.0)
    p["detectors"] = [dict(face=4, u_mm=5.5 + s, v_mm=5.5, radius_mm=0.5, half_angle_deg=20.0)
                      for s in (1.0, 3.0)]
    return W._bins(p)


def test_classes_of_the_phantom():
    m = Model(phantom())
    cls, pairs = optics_classes(m)
    assert len(pairs) == 3 and cls.shape == (m.nv,)
    for c, (mut, a) in enumerate(pairs):
        assert np.all(m.mut[cls == c] == mut) and np.all(m.albedo[cls == c] == a)


def test_exact_solver_equals_converged_iteration():
    p = phantom()
    assert Model(p).interfaces
    a = Solver(dict(p)).run(p["steps"])
    b = ExactSolver(dict(p)).run(p["steps"])
    scale = np.max(np.abs(a["detectors"]))
    assert scale > 0
    assert np.max(np.abs(a["detectors"] - b["detectors"])) <= 1e-10 * scale
    assert np.allclose(a["energy"], b["energy"], rtol=1e-10, atol=0)
