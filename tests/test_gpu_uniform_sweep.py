"""The sweeps' uniform-optics forms against their per-voxel forms, bit for bit.

When mu_t or n is the same in every voxel the sweeps take the direction's attenuation,
b0, b1 and the retarded delay's split once per block instead of once per voxel, by the
same FP32 operations on the same values.  The check: change mu_s (or n) in one corner
voxel that light cannot reach within the run (light moves at most one slab per step,
Section 2.1), which sends every voxel through the per-voxel form, and ask for identical
fields (detector curves and energy tallies to 1e-12: FP64 atomics add them in
scheduling order).  The per-voxel forms themselves are held to
the oracle by the parity tests on heterogeneous media.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

STEPS = 12  # light moves at most one slab per step: the corner, 15 slabs away, stays dark


def _lib():
    import paper_2105_01028_gb300 as P
    return P


def _slab(precision, nside_scatter=0):
    p = W.config_slab(steps=STEPS, precision=precision, nx=24, ny=24, nz=16)
    if nside_scatter:
        p["nside_scatter"] = nside_scatter
    return p


def _run(p):
    P = _lib()
    fw = P.Forward(p)
    fw.step(STEPS)
    out = dict(det=fw.detectors(), N=fw.energy(), I=fw.field(P.FIELD_I), S=fw.field(P.FIELD_S),
               I1=fw.field(P.FIELD_I, 1))
    fw.close()
    return out


def _perturbed(p, mu, n):
    q = dict(p, mus=p["mus"].copy(), nidx=p["nidx"].copy())
    corner = (q["nz"] - 1, 0, 0)  # >= 15 slabs from the source on the -z face
    if mu:
        q["mus"][corner] *= 1.25
    if n:
        q["nidx"][corner] = np.float32(1.45)
    return q


@pytest.mark.parametrize("precision,nside_scatter", [("fp32", 0), ("bf16", 0), ("fp32", 2)])
def test_uniform_forms_match_per_voxel_forms(precision, nside_scatter):
    p = _slab(precision, nside_scatter)
    base = _run(p)
    assert np.max(base["det"]) > 0 and np.max(np.abs(base["I"])) > 0
    for mu, n in ((True, False), (False, True), (True, True)):
        got = _run(_perturbed(p, mu, n))
        for k in ("I", "S", "I1"):
            assert np.array_equal(got[k], base[k]), (precision, nside_scatter, mu, n, k)
        for k in ("det", "N"):
            np.testing.assert_allclose(got[k], base[k], rtol=1e-12, atol=0)


@pytest.mark.parametrize("face,grid", [(0, (20, 12, 16)), (3, (20, 12, 16)), (4, (20, 12, 16)),
                                       (1, (44, 10, 9)), (5, (44, 10, 9))])
def test_tma_sweep_matches_plain_sweep(face, grid):
    """With a uniform refractive index, vacuum faces and nx a multiple of 4 the sweep stages
    its upwind planes through the TMA (one kernel per dominant-axis class).  Against the
    plain-load sweep of the same description, and with n changed in one unreachable corner
    voxel (which sends the step through the plain sweep's per-voxel delays), fields must
    agree bit for bit.  The pulse enters through an x, y or z face so that each class sees the source
    face's inflow; nx = 44 gives the x-dominant items a full 32-voxel chunk and a ragged one."""
    P = _lib()
    n = grid
    p = W.homogeneous(n[0], n[1], n[2], 4, 0.01, 2.0, steps=STEPS, tol=1e-6)
    axis = face // 2
    uv = [a for a in range(3) if a != axis]
    p["source"] = dict(face=face, u_mm=n[uv[0]] / 2, v_mm=n[uv[1]] / 2, half_angle_deg=15.0,
                       pulse_steps=2, energy=1.0)
    fw = P.Forward(p)
    launches = fw.kernels_per_step()
    form = fw.sweep_form()
    fw.close()
    assert launches == 6 and form == "tma"  # three sweep classes, scatter, tallies, step counter
    base = _run(p)
    assert np.max(np.abs(base["I"])) > 0
    plain = dict(p, sweep_tma=False)
    fw = P.Forward(plain)
    assert fw.kernels_per_step() == 4 and fw.sweep_form() == "plain"
    fw.close()
    got = _run(plain)
    for k in ("I", "S", "I1"):
        assert np.array_equal(got[k], base[k]), k
    q = dict(p)
    q["nidx"] = p["nidx"].copy()
    q["nidx"][-1, -1, -1 if face % 2 == 0 else 0] = 1.3
    fw = P.Forward(q)
    assert fw.kernels_per_step() == 4 and fw.sweep_form() == "plain"
    fw.close()
    got = _run(q)
    for k in ("I", "S", "I1"):
        assert np.array_equal(got[k], base[k]), k
