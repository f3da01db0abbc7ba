"""Pins of the oracle's discrete adjoint (gradient of a detector misfit w.r.t. mu_a, mu_s).

The paper has no adjoint (§4 names inverse problems as future work).  The gradient is
pinned to central finite differences of the forward oracle, which shares none of its
backward arithmetic, and the derivatives of the Eq. 9 weights to differences of the
weights themselves across the series / closed-form switch.
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint
from oracle.solver import Solver, ray_weights

NSTEPS = 24


def _problem(fresnel):
    """6^3 voxels, 48 directions, +-25 % random optics, a 2-step pulse, three detectors;
    with ``fresnel`` a 2^3 block of n = 1 inside n = 1.4 adds index interfaces."""
    p = W.homogeneous(6, 6, 6, 2, 0.05, 2.0, steps=NSTEPS, tol=1e-13)
    rng = np.random.default_rng(1)
    p["mua"] = 0.05 * (1 + 0.5 * rng.random(p["mua"].shape))
    p["mus"] = 2.0 * (1 + 0.5 * rng.random(p["mus"].shape))
    p["max_iters"] = 5000
    c = 3.0
    p["source"] = dict(face=4, u_mm=c, v_mm=c, half_angle_deg=30.0, pulse_steps=2, energy=1.0)
    p["detectors"] = [dict(face=4, u_mm=c + 0.5 + s, v_mm=c + 0.5, radius_mm=0.5,
                           half_angle_deg=30.0) for s in (1.0, 2.0)]
    p["detectors"].append(dict(face=5, u_mm=c + 0.5, v_mm=c + 0.5, radius_mm=0.5,
                               half_angle_deg=30.0))
    if fresnel:
        nid = np.full(p["mua"].shape, 1.4)
        nid[2:4, 2:4, 2:4] = 1.0
        p["nidx"] = nid
        p["fresnel"] = True
    return W._bins(p)


def _misfit(p, obs):
    d = Solver(p).run(NSTEPS)["detectors"]
    return 0.5 * float(np.sum((d - obs) ** 2))


@pytest.mark.parametrize("fresnel", [False, True])
def test_gradient_matches_central_differences(fresnel):
    p = _problem(fresnel)
    obs = 0.8 * Solver(p).run(NSTEPS)["detectors"]
    L, g_a, g_s, det = adjoint.gradient(p, NSTEPS, obs)
    assert L == pytest.approx(_misfit(p, obs), rel=1e-12)
    # voxels on the source column, beside the detectors, in the low-index block and far off
    voxels = [100, 170, 141, 4] + ([int(np.ravel_multi_index((2, 2, 3), (6, 6, 6)))]
                                   if fresnel else [])
    for name, g in (("mua", g_a), ("mus", g_s)):
        for v in voxels:
            base = p[name].ravel()[v]
            e = 1e-5 * base
            vals = []
            for sgn in (1.0, -1.0):
                q = dict(p)
                arr = np.array(p[name], dtype=np.float64)
                arr.ravel()[v] = base + sgn * e
                q[name] = arr
                vals.append(_misfit(q, obs))
            fd = (vals[0] - vals[1]) / (2 * e)
            # FD noise ~ 1e-16 L / e; the gradient is exact up to the iteration tolerance
            noise = 1e-15 * L / e
            assert abs(g[v] - fd) <= 1e-6 * abs(fd) + 10 * noise, (name, v, g[v], fd)


def test_zero_misfit_has_zero_gradient():
    p = _problem(False)
    obs = Solver(p).run(NSTEPS)["detectors"]
    L, g_a, g_s, _ = adjoint.gradient(p, NSTEPS, obs)
    assert L == 0.0 and not np.any(g_a) and not np.any(g_s)


def test_ray_weight_derivatives_match_differences():
    x = np.concatenate([np.geomspace(1e-5, 30.0, 400), [9.9e-3, 1e-2, 1.01e-2]])
    dT, db0, db1 = adjoint.ray_weight_derivatives(x)
    h = np.maximum(1e-4 * x, 1e-6)   # above the cancellation noise of the closed forms
    hi, lo = ray_weights(x + h), ray_weights(x - h)
    for k, got in enumerate((dT, db0, db1)):
        fd = (hi[k] - lo[k]) / (2 * h)
        assert np.max(np.abs(got - fd) / np.maximum(np.abs(fd), 1e-3)) < 2e-6, k
    # limits: db0/dx, db1/dx -> 1/2 at x = 0
    d0 = adjoint.ray_weight_derivatives(np.array([0.0]))
    assert d0[1][0] == 0.5 and d0[2][0] == 0.5 and d0[0][0] == -1.0


def test_transposed_interfaces_are_the_adjoint_of_the_split():
    from oracle.fresnel import apply_interfaces
    from oracle.solver import Model
    m = Model(_problem(True))
    assert m.interfaces
    rng = np.random.default_rng(2)
    q = rng.random((m.na, m.nv))
    r = rng.random((m.na, m.nv))
    Fq = apply_interfaces(m.interfaces, q.copy())
    assert np.sum(Fq * r) == pytest.approx(np.sum(q * adjoint.transpose_interfaces(m.interfaces, r)),
                                           rel=1e-13)
