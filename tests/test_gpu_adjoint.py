"""GPU adjoint (trinity_run_checkpointed + trinity_adjoint) against the FP64 oracle adjoint.

The oracle's gradient is pinned to central differences of the forward oracle on the CPU
(test_oracle_adjoint.py); here the library's FP32 reverse sweep is compared with it
element by element, and its exact properties are checked: the checkpoint interval does
not change a bit of the result, the forward state survives the reverse sweep, a zero
misfit gives a zero gradient.  At the gradient workload's optics, directions and detector
layout, the gradient is checked against central differences of the library's own
forward model.

Tolerance.  The FP32 forward fields of slowly converging workloads carry errors of up
to 2e-4 of their peak (the forward parity bar, test_gpu_parity.py); the adjoint fields
are computed with the same arithmetic, and every gradient term is a product of a forward
and an adjoint field summed over steps and directions, so its error relative to max |g|
is bounded by about the sum of the two.  The bar is 3e-4 of max |g| element by element
(measured: 1.5e-5 to 1.1e-4, the largest at 192 directions with interfaces).  Detector
curves are held to the FP32 forward's bar for slow workloads, 2e-5 of their peak.

Finite differences.  The least-squares misfit is a poor subject for them here: its
gradient is concentrated at the source voxel, where the light that enters the medium goes
as exp(-mu_t ds) with mu_t ds of 10-17, while the residual is small compared with the
curves, so the misfit's curvature (the sum of (dE)^2) swamps a central difference of any
step that FP32 resolves.  The checks therefore difference the linear functional
sum G E(mu) with the residual G frozen at the base point: its gradient is the same J^T G.
Detector curves are compared to 1e-12 where FP64 atomics sum them in a different order.
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as OA
from oracle.solver import Solver as OSolver

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4
DET_TOL = 1e-5


def _lib():
    import paper_2105_01028_gb300 as P
    return P


def _problem(nx, ny, nz, nside, steps, fresnel, seed=1):
    """Random optics (+-25 %), a 2-step pulse, two -z detectors and one +z detector; with
    ``fresnel`` a block of n = 1 inside n = 1.4 adds index interfaces."""
    p = W.homogeneous(nx, ny, nz, nside, 0.05, 2.0, steps=steps, tol=1e-6)
    rng = np.random.default_rng(seed)
    p["mua"] = (0.05 * (1 + 0.5 * rng.random(p["mua"].shape))).astype(np.float32)
    p["mus"] = (2.0 * (1 + 0.5 * rng.random(p["mus"].shape))).astype(np.float32)
    p["max_iters"] = 5000
    cu, cv = float(nx // 2), float(ny // 2)
    p["source"] = dict(face=4, u_mm=cu, v_mm=cv, half_angle_deg=30.0, pulse_steps=2, energy=1.0)
    p["detectors"] = [dict(face=4, u_mm=cu + 0.5 + s, v_mm=cv + 0.5, radius_mm=0.5,
                           half_angle_deg=30.0) for s in (1.0, 2.0)]
    p["detectors"].append(dict(face=5, u_mm=cu + 0.5, v_mm=cv + 0.5, radius_mm=0.5,
                               half_angle_deg=30.0))
    if fresnel:
        nid = np.full(p["mua"].shape, 1.4, dtype=np.float32)
        nid[nz // 3: nz // 3 + 2, 2:4, 2:4] = 1.0
        p["nidx"] = nid
        p["fresnel"] = True
    return W._bins(p)


def _gpu_gradient(p, steps, every, G):
    P = _lib()
    fw = P.Forward(p)
    fw.run_checkpointed(steps, every)
    det = fw.detectors()
    ga, gs = fw.adjoint(G)
    fw.close()
    return det, ga, gs


def _oracle_gradient(p, steps, obs):
    q = dict(p, tol=1e-13, mua=np.asarray(p["mua"], np.float64), mus=np.asarray(p["mus"], np.float64))
    return OA.gradient(q, steps, obs)


def _compare(g_gpu, g_ref):
    scale = np.max(np.abs(g_ref))
    assert scale > 0
    err = np.max(np.abs(g_gpu - g_ref)) / scale
    assert err <= GRAD_TOL, err
    return err


@pytest.mark.parametrize("shape,nside,steps,every,fresnel", [
    ((6, 6, 6), 2, 24, 7, False),      # several segments and a ragged last one
    ((7, 6, 5), 2, 24, 24, True),      # index interfaces, one segment, odd grid
    ((8, 8, 6), 4, 16, 5, False),      # 192 directions
    ((8, 7, 6), 4, 14, 4, True),       # 192 directions with interfaces
])
def test_adjoint_matches_oracle(shape, nside, steps, every, fresnel):
    p = _problem(*shape, nside, steps, fresnel)
    obs = 0.8 * OSolver(dict(p, tol=1e-13)).run(steps)["detectors"]
    L, ga_ref, gs_ref, det_ref = _oracle_gradient(p, steps, obs)
    det, _, _ = _gpu_gradient(p, steps, every, np.zeros_like(obs))
    G = det - obs  # the GPU's own residual, as a user computes it
    det, ga, gs = _gpu_gradient(p, steps, every, G)
    assert np.max(np.abs(det - det_ref)) <= DET_TOL * np.max(np.abs(det_ref))
    _compare(ga, ga_ref)
    _compare(gs, gs_ref)


def test_gradient_workload_optics_match_oracle():
    """The gradient workload's optics (random field, mu_s ~ 10/mm) at 8^3, 48 directions."""
    p, q = W.config_adjoint(n=8, nside=2, steps=30)
    p["max_iters"] = 20000
    P = _lib()
    fq = P.Forward(q)
    fq.step(30)
    obs = fq.detectors()
    fq.close()
    det, _, _ = _gpu_gradient(p, 30, 10, np.zeros_like(obs))
    G = det - obs
    _, ga, gs = _gpu_gradient(p, 30, 10, G)
    po = dict(p, tol=1e-13, mua=p["mua"].astype(np.float64), mus=p["mus"].astype(np.float64))
    det_o = OSolver(po).run(30)["detectors"]
    _, ga_ref, gs_ref, _ = OA.gradient(po, 30, det_o - G)  # the oracle at the same residual
    _compare(ga, ga_ref)
    _compare(gs, gs_ref)


def test_checkpoint_interval_changes_nothing():
    p = _problem(6, 6, 6, 2, 24, True)
    G = np.random.default_rng(3).standard_normal((len(p["detectors"]), p["nbins"]))
    _, ga1, gs1 = _gpu_gradient(p, 24, 3, G)
    _, ga2, gs2 = _gpu_gradient(p, 24, 24, G)
    _, ga3, gs3 = _gpu_gradient(p, 24, 10, G)
    assert np.array_equal(ga1, ga2) and np.array_equal(gs1, gs2)
    assert np.array_equal(ga1, ga3) and np.array_equal(gs1, gs3)


def test_forward_state_survives_the_reverse_sweep():
    P = _lib()
    p = _problem(6, 6, 6, 2, 30, False)
    G = np.ones((len(p["detectors"]), p["nbins"]))
    a = P.Forward(p)
    a.run_checkpointed(20, 6)
    a.adjoint(G)
    ga, gs = a.adjoint(G)  # a second reverse sweep from the same checkpoints
    a.step(10)
    b = P.Forward(p)
    b.step(30)
    np.testing.assert_allclose(a.detectors(), b.detectors(), rtol=1e-12, atol=0)
    assert np.array_equal(a.field(0), b.field(0)) and np.array_equal(a.field(1, 3), b.field(1, 3))
    c = P.Forward(p)
    c.run_checkpointed(20, 20)
    ga2, gs2 = c.adjoint(G)
    assert np.array_equal(ga, ga2) and np.array_equal(gs, gs2)


def test_zero_misfit_gives_zero_gradient():
    p = _problem(6, 6, 6, 2, 12, True)
    _, ga, gs = _gpu_gradient(p, 12, 5, np.zeros((len(p["detectors"]), p["nbins"])))
    assert not np.any(ga) and not np.any(gs)


def test_adjoint_call_order_is_checked():
    P = _lib()
    p = _problem(6, 6, 6, 2, 12, False)
    G = np.zeros((len(p["detectors"]), p["nbins"]))
    fw = P.Forward(p)
    with pytest.raises(P.TrinityError, match="E_STATE"):
        fw.adjoint(G)
    fw.run_checkpointed(8, 4)
    with pytest.raises(ValueError):
        fw.adjoint(np.zeros(3))
    fw.step(1)
    with pytest.raises(P.TrinityError, match="E_STATE"):
        fw.adjoint(G)
    with pytest.raises(P.TrinityError, match="E_STATE"):
        fw.run_checkpointed(8, 4)
    fw.reset()
    fw.run_checkpointed(8, 4)
    fw.adjoint(G)


def test_device_pointers_and_autograd():
    torch = pytest.importorskip("torch")
    from paper_2105_01028_gb300.autograd import detector_curves
    P = _lib()
    p = _problem(6, 6, 6, 2, 16, False)
    obs = 0.8 * OSolver(dict(p, tol=1e-13)).run(16)["detectors"]
    fw = P.Forward(p)
    fw.run_checkpointed(16, 5)
    G = fw.detectors() - obs
    ga, gs = fw.adjoint(G)
    dev = torch.device("cuda:0")
    Gd = torch.as_tensor(G, device=dev)
    oa = torch.zeros(ga.size, dtype=torch.float64, device=dev)
    os_ = torch.zeros_like(oa)
    fw.adjoint(Gd, out=(oa, os_))
    assert np.array_equal(oa.cpu().numpy(), ga) and np.array_equal(os_.cpu().numpy(), gs)
    mua = torch.tensor(p["mua"], device=dev, requires_grad=True)
    mus = torch.tensor(p["mus"], device=dev, requires_grad=True)
    E = detector_curves(mua, mus, p, 16, every=5)
    loss = 0.5 * torch.sum((E - torch.as_tensor(obs, device=dev)) ** 2)
    loss.backward()
    # the curves (hence dL/dE) agree to FP64 atomics' order, the gradients to float32
    np.testing.assert_allclose(mua.grad.double().cpu().numpy().ravel(), ga, rtol=1e-6,
                               atol=1e-9 * np.max(np.abs(ga)))
    np.testing.assert_allclose(mus.grad.double().cpu().numpy().ravel(), gs, rtol=1e-6,
                               atol=1e-9 * np.max(np.abs(gs)))


def _functional(P, p, steps, G):
    fw = P.Forward(p)
    fw.step(steps)
    d = fw.detectors()
    fw.close()
    return float(np.sum(G * d))


def test_central_differences_on_gradient_workload_layout():
    """The gradient workload's optics, directions and detector layout on a 24^3 grid
    (100 steps): the library's gradient for the frozen least-squares residual G against
    central differences of sum G E(mu) computed with its own FP32 forward model, on 20
    random voxels with |g| above 1e-3 of the maximum (steps of +-1 %), and along one
    random smooth direction through every voxel (+-0.3 %)."""
    P = _lib()
    steps = 100
    p, q = W.config_adjoint(n=24, steps=steps)
    fw = P.Forward(q)
    fw.step(steps)
    obs = fw.detectors()
    fw.close()
    fw = P.Forward(p)
    fw.run_checkpointed(steps, 50)
    G = fw.detectors() - obs
    ga, gs = fw.adjoint(G)
    fw.close()
    # resolution of sum G E: the curves carry the iteration tolerance (1e-6) relative
    fw = P.Forward(p)
    fw.step(steps)
    F_abs = float(np.sum(np.abs(G * fw.detectors())))
    fw.close()
    rng = np.random.default_rng(8)
    for name, g in (("mua", ga), ("mus", gs)):
        gmax = np.max(np.abs(g))
        cand = np.nonzero(np.abs(g) > 1e-3 * gmax)[0]
        vox = rng.choice(cand, size=min(10, cand.size), replace=False)
        for v in vox:
            base = float(p[name].ravel()[v])
            vals = []
            for sgn in (1.0, -1.0):
                arr = np.array(p[name], dtype=np.float32)
                arr.ravel()[v] = base * (1.0 + sgn * 0.01)
                vals.append((_functional(P, dict(p, **{name: arr}), steps, G), float(arr.ravel()[v])))
            dmu = vals[0][1] - vals[1][1]
            fd = (vals[0][0] - vals[1][0]) / dmu
            noise = 3.0 * 1e-6 * F_abs / dmu
            assert abs(fd - g[v]) <= 2e-2 * abs(g[v]) + noise, (name, v, fd, g[v], noise)
    da = W.gaussian_random_field(p["mua"].shape, 3.0, 1.0, rng).astype(np.float32)
    ds = W.gaussian_random_field(p["mus"].shape, 3.0, 1.0, rng).astype(np.float32)
    t = 3e-3
    Fp = _functional(P, dict(p, mua=(p["mua"] * (1 + t * da)).astype(np.float32),
                             mus=(p["mus"] * (1 + t * ds)).astype(np.float32)), steps, G)
    Fm = _functional(P, dict(p, mua=(p["mua"] * (1 - t * da)).astype(np.float32),
                             mus=(p["mus"] * (1 - t * ds)).astype(np.float32)), steps, G)
    fd = (Fp - Fm) / (2 * t)
    ad = float(np.sum(ga * (p["mua"] * da).ravel()) + np.sum(gs * (p["mus"] * ds).ravel()))
    assert abs(fd - ad) <= 1e-2 * abs(ad), (fd, ad)
