"""Exact per-voxel source function (trinity_set_exact_solve) on the GPU against the
oracle's ExactSolver, which is pinned to the fixed-point equation and to the converged
iteration on the CPU (test_oracle_exact.py).

Bars are the FP32 bar of the iteration (test_gpu_parity.py): 1e-5 of the peak for
detector curves, energy and whole fields.  The exact path replaces the iteration's
stopping error by one product with an operator that the host builds in FP64: on the
tensor cores at 192 directions (three TF32 products, ~22 significant bits per operand,
FP32 accumulation), else FP32 on the SIMT cores; both are held to the same bar.
"""
import numpy as np
import pytest

import workloads as W
from oracle.exact import ExactSolver
from test_oracle_exact import phantom

pytestmark = pytest.mark.gpu

DET_TOL = 1e-5
FIELD_TOL = 1e-5


def _lib():
    import paper_2105_01028_gb300 as P
    return P


def _run(p, steps):
    P = _lib()
    fw = P.Forward(p)
    fw.step(steps)
    out = dict(det=fw.detectors(), N=fw.energy()[0], I=fw.field(P.FIELD_I), S=fw.field(P.FIELD_S),
               classes=fw.exact_classes(), form=fw.exact_form(), absorbed=fw.balance()["absorbed"])
    fw.close()
    return out


@pytest.mark.parametrize("nside", [2, 4])
def test_exact_matches_oracle(nside):
    steps = 12 if nside == 2 else 8
    p = phantom(nside=nside, steps=steps, tol=1e-6)
    p["exact"] = True
    s = ExactSolver(dict(p, mua=np.asarray(p["mua"], np.float64), mus=np.asarray(p["mus"], np.float64)))
    ref = s.run(steps)
    g = _run(p, steps)
    assert g["classes"] == 3
    assert g["form"] == ("tc" if nside == 4 else "simt")  # 800 voxels: six tiles and a ragged one
    assert np.max(np.abs(g["det"] - ref["detectors"])) <= DET_TOL * np.max(np.abs(ref["detectors"]))
    assert np.max(np.abs(g["N"] - ref["energy"])) <= DET_TOL * np.max(ref["energy"])
    I_ref, S_ref = s.level("I"), s.level("S")
    assert np.max(np.abs(g["I"] - I_ref)) <= FIELD_TOL * np.max(np.abs(I_ref))
    assert np.max(np.abs(g["S"] - S_ref)) <= FIELD_TOL * np.max(np.abs(S_ref))


def test_exact_agrees_with_the_converged_gpu_iteration():
    p = phantom(nside=2, steps=16, tol=1e-8)
    it = _run(dict(p), 16)
    ex = _run(dict(p, exact=True), 16)
    assert it["classes"] == 0 and ex["classes"] == 3
    assert np.max(np.abs(it["det"] - ex["det"])) <= DET_TOL * np.max(np.abs(ex["det"]))
    assert np.max(np.abs(it["I"] - ex["I"])) <= FIELD_TOL * np.max(np.abs(ex["I"]))


def test_tensor_core_and_simt_forms_agree():
    """The two forms of the exact solve on the phantom (three classes, tiles that mix
    them, a ragged last tile), after enough steps for light to cross the interfaces."""
    p = phantom(nside=4, steps=10, tol=1e-6)
    tc = _run(dict(p, exact=True), 10)
    simt = _run(dict(p, exact="simt"), 10)
    assert tc["form"] == "tc" and simt["form"] == "simt"
    for k in ("det", "N", "I", "S", "absorbed"):
        assert np.max(np.abs(tc[k] - simt[k])) <= FIELD_TOL * np.max(np.abs(simt[k])), k


def test_tensor_core_form_with_eight_classes():
    """Eight optics classes (the most the exact solve takes) in stripes along x, so every
    128-voxel tile holds several of them: against the oracle."""
    steps = 8
    p = W.homogeneous(16, 8, 6, 4, 0.02, 2.0, g=0.9, steps=steps, tol=1e-6)
    p["max_iters"] = 20000
    mua, mus = np.array(p["mua"], np.float32), np.array(p["mus"], np.float32)
    x = np.arange(16)
    for c in range(8):
        sel = (x // 2) == c
        mua[:, :, sel] = np.float32(0.01 + 0.01 * c)
        mus[:, :, sel] = np.float32(1.0 + 0.25 * c)
    p["mua"], p["mus"] = mua, mus
    p["source"] = dict(face=4, u_mm=8.0, v_mm=4.0, half_angle_deg=20.0, pulse_steps=2, energy=1.0)
    p["detectors"] = [dict(face=4, u_mm=10.5, v_mm=4.5, radius_mm=1.0, half_angle_deg=20.0)]
    p = W._bins(p)
    g = _run(dict(p, exact=True), steps)
    assert g["classes"] == 8 and g["form"] == "tc"
    s = ExactSolver(dict(p, mua=np.asarray(p["mua"], np.float64), mus=np.asarray(p["mus"], np.float64)))
    ref = s.run(steps)
    assert np.max(np.abs(g["det"] - ref["detectors"])) <= DET_TOL * np.max(np.abs(ref["detectors"]))
    I_ref, S_ref = s.level("I"), s.level("S")
    assert np.max(np.abs(g["I"] - I_ref)) <= FIELD_TOL * np.max(np.abs(I_ref))
    assert np.max(np.abs(g["S"] - S_ref)) <= FIELD_TOL * np.max(np.abs(S_ref))


def test_voxel_count_not_a_multiple_of_four_takes_the_simt_form():
    p = W.config_slab(steps=4, nx=9, ny=9, nz=7)
    p["exact"] = True
    g = _run(p, 4)
    assert g["classes"] == 1 and g["form"] == "simt"


def test_bf16_context_takes_the_same_exact_path():
    p = phantom(nside=4, steps=6, tol=1e-6)
    a = _run(dict(p, exact=True, precision="fp32"), 6)
    b = _run(dict(p, exact=True, precision="bf16"), 6)
    assert np.array_equal(a["I"], b["I"]) and np.array_equal(a["S"], b["S"])


def test_homogeneous_slab_is_one_class():
    p = W.config_slab(steps=8, nx=24, ny=24, nz=16)
    p["exact"] = True
    g = _run(p, 8)
    assert g["classes"] == 1 and np.max(g["det"]) > 0


def test_exact_rejects_continuous_optics_and_two_level_grids():
    P = _lib()
    p, _ = W.config_adjoint(n=8, nside=2, steps=4)  # log-normal random field: 512 classes
    with pytest.raises(P.TrinityError, match="E_UNSUPPORTED"):
        P.Forward(dict(p, exact=True))
    fw = P.Forward(p)
    assert fw.L.trinity_set_exact_solve(fw.h, 1) != 0 and fw.exact_classes() == 0
    fw.step(2)  # still steps with the iteration
    q = W.homogeneous(6, 6, 6, 4, 0.02, 2.0, steps=4)
    q["nside_scatter"] = 2
    with pytest.raises(P.TrinityError, match="E_UNSUPPORTED"):
        P.Forward(dict(q, exact=True))


def _sampled_one_step(prob, steps, vox, tol_scale=DET_TOL):
    """Run ``steps`` steps on the GPU and recompute level steps-1 at ``vox`` with the oracle
    from the GPU's own stored history (one step of Eq. 10, the interface split and the
    source function converged to 1e-10, i.e. the fixed point the exact solve reaches)."""
    P = _lib()
    from oracle.solver import Model, one_step_at
    fw = P.Forward(prob)
    fw.step(steps)
    n = steps - 1
    hist = {}
    for back in range(1, 5):
        if n - back >= 0:
            hist[n - back] = (fw.field(P.FIELD_I, back), fw.field(P.FIELD_S, back))
    I_n, S_n = fw.field(P.FIELD_I, 0), fw.field(P.FIELD_S, 0)
    fw.close()

    def h(which, lev, d, u):
        out = np.zeros(np.shape(lev))
        for L, (Ia, Sa) in hist.items():
            m = lev == L
            if np.any(m):
                out[m] = (Ia if which == "I" else Sa)[d[m], u[m]]
        return out

    s_glob = float(np.abs(hist[n - 1][1]).max())
    p = dict(prob, tol=1e-10, max_iters=20000)
    I_ref, S_ref, _ = one_step_at(Model(p), n, h, np.asarray(vox), s_glob)
    assert np.abs(I_n[:, vox] - I_ref).max() <= tol_scale * np.abs(I_n).max()
    assert np.abs(S_n[:, vox] - S_ref).max() <= tol_scale * np.abs(S_n).max()


def test_full_size_slab_exact_sampled_one_step():
    """The bench's exact-solve workload at full size (96x96x64, 192 directions)."""
    prob = W.config_slab(steps=24)
    prob["exact"] = True
    nz, ny, nx = prob["nz"], prob["ny"], prob["nx"]
    rng = np.random.default_rng(5)
    cx, cy = nx // 2, ny // 2
    vox = sorted({(z * ny + y) * nx + x for z, y, x in zip(rng.integers(0, 12, 64), rng.integers(cy - 8, cy + 8, 64),
                                                           rng.integers(cx - 8, cx + 8, 64))} | {cy * nx + cx})
    _sampled_one_step(prob, 24, vox)


def test_full_size_phantom_exact_sampled_one_step():
    """The heterogeneous phantom at full size (128x128x96, 192 directions, five optics
    classes, refraction at the air cylinder): voxels near the source, in and beside the
    cylinder and in the spheres, some in tiles that mix classes."""
    prob = W.config_hetero(steps=20, precision="fp32")
    prob["exact"] = True
    nz, ny, nx = prob["nz"], prob["ny"], prob["nx"]
    rng = np.random.default_rng(6)
    zc, yc = nz // 2, ny // 2
    vox = {(zc * ny + yc) * nx + 0}
    vox |= {(z * ny + y) * nx + x for z, y, x in zip(rng.integers(zc - 6, zc + 6, 48),
                                                      rng.integers(yc - 6, yc + 6, 48), rng.integers(0, 10, 48))}
    cyl = prob["cylinder"]
    for k in range(16):  # along the cylinder wall
        x = int(cyl["center"][0] + (cyl["radius"] + 0.5) * np.cos(k)) % nx
        y = int(cyl["center"][1] + (cyl["radius"] + 0.5) * np.sin(k)) % ny
        vox.add((int(rng.integers(0, nz)) * ny + y) * nx + x)
    for c, r, _ in prob["spheres"]:
        vox.add((int(c[2]) * ny + int(c[1])) * nx + int(c[0]))
    _sampled_one_step(prob, 20, sorted(vox))
