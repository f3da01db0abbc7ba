"""The source-iteration entry point that allocates nothing (trinity_source_iteration_noalloc).

Some callers cannot call cudaMalloc when they need a solve (their framework's pool owns
the device memory, or the code runs where allocation is forbidden).  This entry point
keeps its scratch in a static device array instead.  The test feeds it the inputs of
real time steps taken by the context API (Q recovered as I - b1 S from the context's
own output, b1 and eps from the optics) and checks its S and I against the context's,
on two calls in a row (the second call reuses the scratch the first one left behind).
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-5  # the FP32 parity bar of the other GPU tests (relative to the field peak)


def test_noalloc_source_iteration_matches_context_steps():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2105_01028_gb300 as T
    prob = W.homogeneous(20, 18, 16, 4, 0.02, 3.0, steps=40, tol=1e-6)
    prob["source"] = dict(face=4, u_mm=10.0, v_mm=9.0, half_angle_deg=15.0, pulse_steps=1, energy=1.0)
    na, nv = 192, 20 * 18 * 16
    fwd = T.Forward(prob)
    fwd.step(30)
    # b1 and eps from the optics, in FP64 (Eq. 9 weight of S(n); eps = mu_a / mu_t)
    dom_sgn, ds, _ = T.lattice_tables(4, 20, 18, 16)
    mua = prob["mua"].ravel().astype(np.float64)
    mus = prob["mus"].ravel().astype(np.float64)
    mut = mua + mus
    x = mut[None, :] * ds[:, None]
    b1 = ((x - 1.0 + np.exp(-x)) / x).astype(np.float32)
    eps = (mua / mut).astype(np.float32)
    P, _ = T.phase_matrix(4, prob["g"])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    dP, db1, deps = dev(P), dev(b1), dev(eps)
    lib = T.lib()
    fn = lib.trinity_source_iteration_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 7 + [ctypes.c_double, ctypes.c_int,
                                                                          ctypes.POINTER(ctypes.c_int),
                                                                          ctypes.c_void_p]
    stream = torch.cuda.current_stream()
    for call in range(2):
        fwd.step(1)
        I_n, S_n = fwd.field(T.FIELD_I), fwd.field(T.FIELD_S)
        S_prev = fwd.field(T.FIELD_S, back=1)
        Q = I_n.astype(np.float64) - b1.astype(np.float64) * S_n.astype(np.float64)
        dQ, dSp = dev(Q), dev(S_prev)
        dS = torch.empty((na, nv), dtype=torch.float32, device="cuda")
        dI = torch.empty((na, nv), dtype=torch.float32, device="cuda")
        iters = ctypes.c_int(-1)
        rc = fn(na, nv, dP.data_ptr(), dQ.data_ptr(), db1.data_ptr(), deps.data_ptr(), dSp.data_ptr(),
                dS.data_ptr(), dI.data_ptr(), 1e-6, 2000, ctypes.byref(iters), stream.cuda_stream)
        assert rc == 0, rc
        assert iters.value >= 1
        S_out, I_out = dS.cpu().numpy(), dI.cpu().numpy()
        assert np.abs(S_out - S_n).max() <= TOL * np.abs(S_n).max(), call
        assert np.abs(I_out - I_n).max() <= TOL * np.abs(I_n).max(), call
    # sizes beyond the static scratch are refused, not run
    big = fn(na, (1 << 20) + 1, dP.data_ptr(), dQ.data_ptr(), db1.data_ptr(), deps.data_ptr(),
             dSp.data_ptr(), dS.data_ptr(), dI.data_ptr(), 1e-6, 10, None, stream.cuda_stream)
    assert big == -1
    fwd.close()
