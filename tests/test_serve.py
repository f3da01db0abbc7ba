"""Serving: admission by device footprint, overlapping solves, per-request results."""
import numpy as np
import pytest

import paper_2105_01028_gb300 as T
import workloads as W


def _req(n=12, nside=2, steps=40, seed=1):
    return W.config_served(n, nside, steps, seed)


def test_submit_rejects_malformed_and_oversized():
    srv = T.Server(hbm_budget_bytes=1 << 20, max_slots=2)
    with pytest.raises(T.TrinityError):
        srv.submit(_req())  # footprint of a 12^3 x 48 grid exceeds 1 MiB
    bad = _req()
    bad["steps"] = 0
    srv2 = T.Server(hbm_budget_bytes=1 << 34, max_slots=2)
    with pytest.raises(T.TrinityError):
        srv2.submit(bad)
    srv.close()
    srv2.close()


def test_failure_is_reported_without_a_gpu():
    """Where no device is usable, an accepted request ends FAILED with a CUDA status
    instead of hanging or crashing the process."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    srv = T.Server(hbm_budget_bytes=1 << 34, max_slots=2)
    rid = srv.submit(_req())
    state, status, det, lat = srv.wait(rid, timeout_s=60)
    assert state == T.REQ_FAILED and status < 0
    assert srv.stats()["failed"] == 1
    srv.close()


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_result_is_the_same_alone_and_in_the_mix(precision):
    _gpu()
    target = W.config_served(24, 2, 60, seed=11, precision=precision)
    alone = T.Server(hbm_budget_bytes=8 << 30, max_slots=1)
    rid = alone.submit(target)
    st, rc, det_alone, _ = alone.wait(rid)
    assert st == T.REQ_DONE and rc == 0
    alone.close()
    # a mix of grid sizes and angular resolutions, the target in the middle
    mix = T.Server(hbm_budget_bytes=8 << 30, max_slots=4, steps_per_slice=16)
    ids = []
    for k, (n, ns, steps) in enumerate([(32, 2, 80), (20, 4, 50), (28, 2, 40), (16, 4, 70)]):
        ids.append(mix.submit(W.config_served(n, ns, steps, seed=100 + k, precision=precision)))
        if k == 1:
            tid = mix.submit(target)
    st, rc, det_mix, lat = mix.wait(tid)
    for r in ids:
        assert mix.wait(r)[0] == T.REQ_DONE
    assert st == T.REQ_DONE and lat > 0
    assert mix.stats()["max_concurrent"] >= 2
    np.testing.assert_allclose(det_mix, det_alone, rtol=1e-12, atol=0)
    # and the same as a direct run through the context API
    fwd = T.Forward(target)
    fwd.step(target["steps"])
    np.testing.assert_allclose(det_mix, fwd.detectors(), rtol=1e-12, atol=0)
    fwd.close()
    mix.close()


@pytest.mark.gpu
def test_budget_limits_concurrency_and_cancel():
    _gpu()
    p = W.config_served(24, 2, 400, seed=5)
    fp = T.footprint_bytes(p)
    srv = T.Server(hbm_budget_bytes=2 * fp + fp // 2, max_slots=8, steps_per_slice=8)
    ids = [srv.submit(W.config_served(24, 2, 400, seed=20 + k)) for k in range(5)]
    srv.cancel(ids[-1])
    for r in ids[:-1]:
        assert srv.wait(r)[0] == T.REQ_DONE
    assert srv.wait(ids[-1])[0] == T.REQ_CANCELLED
    s = srv.stats()
    assert s["max_concurrent"] == 2 and s["completed"] == 4 and s["bytes_in_use"] == 0
    srv.close()
