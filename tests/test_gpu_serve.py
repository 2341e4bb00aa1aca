"""GPU tests of the continuous-batching server (pid_serve_*).

A request's results must be the same alone and mixed with other requests (they are
bitwise identical here), requests submitted while others run must be batched into later
steps, and admission (HBM budget, queue length) and shutdown must answer with the
documented status codes.
"""
import threading
import time

import numpy as np
import pytest

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth
from tests.helpers import FP32_TOL, GRAM_TOL, assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2512_15187_gb300 import binding, build
    build.build()
    return binding


def _ensembles():
    rng = np.random.default_rng(17)
    out = []
    for k, (N, M) in enumerate([(16, 256 * 256), (40, 128 * 128), (64, 200 * 200), (100, 9000),
                                (7, 50000), (128, 64 * 64 * 4), (33, 70000), (200, 3000)]):
        if k % 3 == 2:
            F = rng.normal(0, 1, (N, M)).astype(np.float32)
            out.append(dict(data=F, iso=(0.2, 0.4, 0), U=O.iso_soft_mask(F, 0.2, 0.4), w=None))
        else:
            U = synth.random_soft(N, M, seed=300 + k)
            w = rng.uniform(0.5, 2, M).astype(np.float32) if k % 2 else None
            out.append(dict(data=U, iso=None, U=U, w=w))
    return out


REQ_KINDS = [("mean", "fp32"), ("linear", "fp32"), ("full", "bf16"), ("full", "fp8")]


def _kind_ok(ens, kind):
    return not (kind[0] == "full" and ens["data"].shape[0] > 256)


def test_results_same_alone_and_in_the_mix(B):
    ens = _ensembles()
    srv = B.Server(max_inflight=3, max_batch=16)
    ids = [srv.register(e["data"], w=e["w"], iso=e["iso"]) for e in ens]
    # alone: one request at a time
    alone = {}
    for k, (e, i) in enumerate(zip(ens, ids)):
        for kind in REQ_KINDS:
            if not _kind_ok(e, kind):
                continue
            t = srv.submit(i, *kind)
            alone[(k, kind)] = srv.wait(t, e["data"].shape[0])
    # parity of the alone results with the oracle
    for (k, kind), o in alone.items():
        e = ens[k]
        ref = O.pid_mean(e["U"], e["w"]) if kind[0] == "mean" else O.pid(e["U"], e["w"])
        assert_close(o["depth"], ref[2], FP32_TOL if kind[1] == "fp32" else GRAM_TOL, f"{kind}")
    # mixed: all requests, three times each, from four threads in random order
    jobs = [key for key in alone for _ in range(3)]
    np.random.default_rng(0).shuffle(jobs)
    results, errors = [], []

    def worker(part):
        try:
            tickets = [(key, srv.submit(ids[key[0]], *key[1])) for key in part]
            for key, t in tickets:
                results.append((key, srv.wait(t, ens[key[0]]["data"].shape[0])))
        except Exception as ex:  # pragma: no cover
            errors.append(ex)

    th = [threading.Thread(target=worker, args=(jobs[i::4],)) for i in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    assert len(results) == len(jobs)
    for key, o in results:
        for f in ("depth", "in_in", "in_out", "rank", "mean_depth"):
            assert np.array_equal(o[f], alone[key][f]), f"{key} {f} differs in the mix"
    st = srv.stats()
    assert st["failed"] == 0
    assert st["mean_batch"] > 1.0, st      # requests were batched together
    srv.stop()


def test_requests_arriving_during_steps_join_later_steps(B):
    import time
    srv = B.Server(max_inflight=2, max_batch=64)
    U = synth.random_soft(64, 1 << 20, seed=5)       # ~0.27 GB: each step takes a while
    i = srv.register(U)
    srv.reset_stats()
    tickets = []
    for k in range(120):
        tickets.append(srv.submit(i, "mean"))
        if k % 10 == 0:
            time.sleep(0.0005)
    outs = [srv.wait(t, 64) for t in tickets]
    ref = O.pid_mean(U)[2]
    assert_close(outs[-1]["depth"], ref, FP32_TOL, "served")
    st = srv.stats()
    assert st["completed"] == 120 and st["steps"] < 120 and st["mean_batch"] > 1.0, st
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    srv.stop()


def test_admission_budget_and_queue(B):
    from paper_2512_15187_gb300.binding import PID_ERR_BUSY, PID_ERR_OOM, PidError
    U = synth.random_soft(32, 1 << 16, seed=1)       # 8 MiB
    srv = B.Server(max_inflight=1, max_batch=1, max_queue=4, hbm_budget_bytes=20 << 20)
    a = srv.register(U)
    srv.register(U)
    with pytest.raises(PidError) as e:
        srv.register(U)                               # 24 MiB > 20 MiB budget
    assert e.value.status == PID_ERR_OOM
    srv.unregister(a)
    srv.register(U)                                   # room again
    srv.stop()

    big = synth.random_soft(128, 1 << 21, seed=2)    # 1 GiB per request
    srv = B.Server(max_inflight=1, max_batch=1, max_queue=4)
    i = srv.register(big)
    busy = 0
    tickets = []
    for _ in range(64):
        try:
            tickets.append(srv.submit(i, "linear"))
        except PidError as ex:
            assert ex.status == PID_ERR_BUSY
            busy += 1
    assert busy > 0
    for t in tickets:
        srv.wait(t, 128)
    srv.stop()


def test_cancel_releases_waiters_before_the_server_is_freed(B):
    """Waiters blocked on their tickets get PID_OK or PID_ERR_CANCELLED from the cancel, are
    joined, and only then is the server freed: no wait runs on freed memory."""
    from paper_2512_15187_gb300.binding import PID_ERR_CANCELLED, PID_OK, load
    big = synth.random_soft(128, 1 << 21, seed=3)
    srv = B.Server(max_inflight=1, max_batch=1, max_queue=64)
    i = srv.register(big)
    tickets = [srv.submit(i, "linear") for _ in range(20)]
    handle = srv.s
    statuses = {}

    def waiter(ts):
        for t in ts:
            statuses[t] = load().pid_serve_wait(handle, t, -1, None, None, None, None, None)

    threads = [threading.Thread(target=waiter, args=(tickets[k::4],)) for k in range(4)]
    for th in threads:
        th.start()
    srv.cancel()                       # returns once every request is done
    for th in threads:
        th.join()
    assert sorted(statuses) == sorted(tickets)
    assert all(s in (PID_OK, PID_ERR_CANCELLED) for s in statuses.values()), statuses
    assert any(s == PID_ERR_CANCELLED for s in statuses.values())
    # after the cancel the server refuses new work but stays valid until stop
    with pytest.raises(B.PidError) as e:
        srv.submit(i, "mean")
    assert e.value.status == PID_ERR_CANCELLED
    assert srv.stats()["submitted"] == 20
    srv.stop()


def test_stop_waits_for_blocked_waiters(B):
    """pid_serve_stop entered while threads are still blocked in pid_serve_wait: they return
    (OK or CANCELLED) before the server is freed, and stop returns after them."""
    from paper_2512_15187_gb300.binding import PID_ERR_CANCELLED, PID_OK, load
    big = synth.random_soft(128, 1 << 21, seed=4)
    srv = B.Server(max_inflight=1, max_batch=1, max_queue=64)
    i = srv.register(big)
    tickets = [srv.submit(i, "linear") for _ in range(12)]
    handle = srv.s
    statuses = {}
    entered = threading.Barrier(4)

    def waiter(t):
        entered.wait()
        statuses[t] = load().pid_serve_wait(handle, t, -1, None, None, None, None, None)

    # three threads wait on the last tickets (still queued when stop begins)
    threads = [threading.Thread(target=waiter, args=(t,)) for t in tickets[-3:]]
    for th in threads:
        th.start()
    entered.wait()
    time.sleep(0.05)                   # let them block inside the wait
    assert load().pid_serve_stop(handle) == PID_OK
    srv.s = None
    for th in threads:
        th.join()
    assert sorted(statuses) == sorted(tickets[-3:])
    assert all(s in (PID_OK, PID_ERR_CANCELLED) for s in statuses.values()), statuses


def test_time_step_update_of_resident_ensemble(B):
    srv = B.Server(max_inflight=2, max_batch=8)
    U0 = synth.random_soft(20, 5000, seed=10)
    U1 = synth.random_soft(20, 5000, seed=11)
    i = srv.register(U0)
    o0 = srv.wait(srv.submit(i, "linear"), 20)
    srv.update(i, U1)
    o1 = srv.wait(srv.submit(i, "linear"), 20)
    assert_close(o0["depth"], O.pid(U0)[2], FP32_TOL, "t0")
    assert_close(o1["depth"], O.pid(U1)[2], FP32_TOL, "t1")
    srv.stop()
