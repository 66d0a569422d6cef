"""Serving engine (step a11): continuous batching on one GPU.

  * each result of a mixed stream (exhaustive and tree potentials, exhaustive
    and tree forces, uneven N, resident systems) equals the same request
    solved alone through
    the direct API: the arithmetic of a request does not depend on what runs
    beside it (Philox draws are keyed by particle and node ids), so only the
    order of FP64 atomic additions differs: |difference| <= 1e-10 max|result|;
  * a request larger than the budget is rejected; a stream whose total
    exceeds the budget is admitted as memory frees up and completes;
  * poll without waiting reports a request still running as pending.
"""
import time

import numpy as np
import pytest
import torch

from paper_1105_2769_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu


def _alone(X, kind, mode, eps, alpha):
    Xd = torch.from_numpy(X).cuda()
    if kind == "forces":
        return api.forces(Xd, mode=mode, eps=eps, alpha=alpha).cpu().numpy()
    return api.potential(Xd, eps=eps, alpha=alpha, mode=mode).cpu().numpy()


def _mix(seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for q in range(18):
        n = int(np.exp(rng.uniform(np.log(256), np.log(3000))))
        if q % 2:
            X = inputs.uniform_cube(n, (n / 1.0) ** (1 / 3), 0.5, 1000 + q)
        else:
            X = inputs.gaussian_mixture(n, 4, 6.0, 0.5, 1.5, 0.05, 1000 + q)
        r = q % 3
        if r == 0:
            reqs.append(dict(X=X, kind="potential", mode="fp32", eps=0.0, alpha=0.0))
        elif r == 1:
            reqs.append(dict(X=X, kind="potential", mode="tree", eps=1e-2, alpha=0.05,
                             system_id=q if q % 4 == 1 else 0))
        elif q % 2:
            reqs.append(dict(X=X, kind="forces", mode="fp32", eps=0.0, alpha=0.0))
        else:  # tree forces, resident for some
            reqs.append(dict(X=X, kind="forces", mode="tree", eps=1e-2, alpha=0.05,
                             system_id=q if q % 4 == 0 else 0))
    return reqs


def test_mixed_stream_equals_alone():
    reqs = _mix(5)
    srv = api.Server(0, hbm_budget_bytes=8 << 30, slots=4)
    tickets = []
    for r in reqs:
        tickets.append(srv.submit(**r))
        time.sleep(0.002)  # arrivals while earlier requests run
    lat = []
    for t, r in zip(tickets, reqs):
        st, res, out = srv.poll(t)
        assert st == 0, res
        lat.append(res["latency_ms"])
        ref = _alone(r["X"], r["kind"], r["mode"], r["eps"], r["alpha"])
        assert np.all(np.abs(out - ref) <= 1e-10 * np.abs(ref).max())
    s = srv.stats()
    assert s["completed"] == len(reqs) and s["pending"] == 0
    print(f"p50 {np.percentile(lat, 50):.1f} ms  p99 {np.percentile(lat, 99):.1f} ms")
    srv.close()


def test_budget_admission_and_rejection():
    X = inputs.uniform_cube(2000, 12.6, 0.5, 7)
    srv = api.Server(0, hbm_budget_bytes=200 << 10, slots=2)  # one request fits at a time
    with pytest.raises(_lib.MbmError) as e:
        srv.submit(inputs.uniform_cube(50000, 36.0, 0.5, 8))
    assert e.value.status == -3
    assert srv.stats()["rejected"] == 1
    # each of these fits alone but not all at once: they run as memory frees up
    tickets = [srv.submit(X[: 1500 + 100 * q]) for q in range(4)]
    for q, t in enumerate(tickets):
        st, res, out = srv.poll(t)
        assert st == 0
        ref = _alone(X[: 1500 + 100 * q], "potential", "fp32", 0.0, 0.0)
        assert np.all(np.abs(out - ref) <= 1e-10 * np.abs(ref).max())
    srv.close()


def test_poll_pending_and_resident_system():
    X = inputs.uniform_cube(6000, 18.2, 0.5, 11)
    srv = api.Server(0, hbm_budget_bytes=4 << 30, slots=1)
    t = srv.submit(X, kind="forces", mode="fp32")
    st, _, _ = srv.poll(t, timeout_us=0)
    assert st == _lib.MBM_PENDING
    st, res, F = srv.poll(t)
    assert st == 0 and res["compute_ms"] > 0
    # the same system twice: the second reuses the resident copy and tree
    a = srv.poll(srv.submit(X, mode="tree", eps=1e-2, alpha=0.0, system_id=42))[2]
    b = srv.poll(srv.submit(X, mode="tree", eps=1e-2, alpha=0.0, system_id=42))[2]
    assert np.all(np.abs(a - b) <= 1e-10 * np.abs(a).max())
    srv.close()


def test_concurrent_first_requests_for_one_system():
    """Several requests for the same new system arrive at once on four slots:
    whichever slot publishes the resident copy, the others either wait for its
    upload and tree build (event) or solve privately; every result equals the
    request solved alone."""
    X = inputs.gaussian_mixture(3000, 4, 8.0, 0.5, 1.5, 0.05, 77)
    ref = _alone(X, "potential", "tree", 1e-2, 0.05)
    srv = api.Server(0, hbm_budget_bytes=4 << 30, slots=4)
    for rep in range(3):
        sid = 900 + rep
        tickets = [srv.submit(X, mode="tree", eps=1e-2, alpha=0.05, system_id=sid)
                   for _ in range(6)]
        for t in tickets:
            st, res, out = srv.poll(t)
            assert st == 0
            assert np.all(np.abs(out - ref) <= 1e-10 * np.abs(ref).max())
    srv.close()


def test_admitted_requests_overlap_on_the_device():
    """Requests admitted together run at once: their device-clock intervals
    (first kernel start to last kernel end, %globaltimer) overlap."""
    srv = api.Server(0, hbm_budget_bytes=8 << 30, slots=4)
    Xs = [inputs.uniform_cube(4096, 16.0, 0.5, 300 + q) for q in range(4)]
    tickets = [srv.submit(X, kind="forces", mode="fp32") for X in Xs]
    iv = []
    for t in tickets:
        st, res, _ = srv.poll(t)
        assert st == 0 and res["dev_end_ns"] > res["dev_start_ns"] > 0
        iv.append((res["dev_start_ns"], res["dev_end_ns"], res["slot"]))
    srv.close()
    iv.sort()
    overlaps = sum(1 for a, b in zip(iv, iv[1:]) if b[0] < a[1])
    print("device intervals (ms from first start):",
          [((s - iv[0][0]) / 1e6, (e - iv[0][0]) / 1e6, sl) for s, e, sl in iv])
    assert overlaps >= 1
    assert len({sl for _, _, sl in iv}) >= 2
