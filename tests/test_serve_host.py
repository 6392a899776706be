"""Host-side checks of the serving loop (queue, admission by memory budget, bounded
waits, statistics) with the library's host-only executor: no GPU is touched."""
import os
import threading
import time

import numpy as np
import pytest

from paper_2411_16392_gb300.scenes import Camera


@pytest.fixture(scope="module")
def lib():
    from paper_2411_16392_gb300 import _lib as L
    from paper_2411_16392_gb300 import build as B
    if not os.path.exists(L.LIB_PATH):
        B.build()
    return L.load()


def _server(**kw):
    from paper_2411_16392_gb300.serve import Server
    return Server(device=-1, **kw)


CAM = Camera(256, 256, 200.0, 200.0, 128.0, 128.0)   # 65,536 px


def test_requests_complete_and_results_are_returned(lib):
    from paper_2411_16392_gb300.serve import host_planes
    s = _server(budget_bytes=1 << 34, slots=2, fake_us_per_mpix=20_000.0)
    sid = s.load_scene(n=1000)
    tickets = [s.submit(sid, CAM) for _ in range(6)]
    for t in tickets:
        out = host_planes(CAM)
        out["rgb"][:] = 5
        s.wait(t, out=out)
        assert np.all(out["rgb"] == 0)          # host executor returns zero planes
    st = s.stats()
    assert st["submitted"] == 6 and st["completed"] == 6 and st["failed"] == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0 and st["frames_per_s"] > 0
    s.close()


def test_queue_full_is_rejected_with_ebusy(lib):
    from paper_2411_16392_gb300._lib import QGSError
    s = _server(budget_bytes=1 << 34, slots=1, queue=3, fake_us_per_mpix=3_000_000.0)  # ~0.2 s each
    sid = s.load_scene(n=10)
    tickets = [s.submit(sid, CAM)]
    time.sleep(0.05)                       # the first one is running, the queue is empty
    tickets += [s.submit(sid, CAM) for _ in range(3)]
    with pytest.raises(QGSError) as e:
        s.submit(sid, CAM)
    assert e.value.status == 6             # QGS_EBUSY
    assert s.stats()["rejected"] == 1
    s.close()                              # drops the queued requests, joins the workers


def test_bounded_wait_times_out_then_succeeds(lib):
    from paper_2411_16392_gb300._lib import QGSError
    s = _server(budget_bytes=1 << 34, slots=1, fake_us_per_mpix=4_000_000.0)  # ~0.26 s
    sid = s.load_scene(n=10)
    t = s.submit(sid, CAM)
    with pytest.raises(QGSError) as e:
        s.wait(t, timeout_ms=20)
    assert e.value.status == 5             # QGS_ETIMEDOUT, ticket still valid
    s.wait(t, timeout_ms=5000)
    with pytest.raises(QGSError) as e:
        s.wait(t, timeout_ms=10)
    assert e.value.status == 7             # QGS_ENOTFOUND: released
    s.close()


def test_admission_respects_the_memory_budget(lib):
    """With 8 slots but a budget for about two requests, at most two run at once."""
    s = _server(budget_bytes=1 << 34, slots=8, fake_us_per_mpix=500_000.0)
    sid = s.load_scene(n=10)
    t = s.submit(sid, CAM)
    s.wait(t)
    s.close()
    # estimated bytes of one 256x256 request with the default instance estimate
    per = (10 * 168 + 64 * 65536 * 16 + 64 * 65536 / 16 + 65536 * 40) + (1 << 20)
    s = _server(budget_bytes=int(2.5 * per), slots=8, fake_us_per_mpix=500_000.0)
    sid = s.load_scene(n=10)
    ts = [s.submit(sid, CAM) for _ in range(8)]
    for t in ts:
        s.wait(t)
    st = s.stats()
    assert st["max_in_flight"] == 2, st
    assert st["bytes_reserved_peak"] <= st["bytes_budget"]
    s.close()


def test_slots_overlap_requests(lib):
    """Continuous batching: 4 slots finish 8 equal requests about 4x sooner than 1 slot."""
    def run(slots):
        s = _server(budget_bytes=1 << 40, slots=slots, fake_us_per_mpix=1_000_000.0)  # ~65 ms each
        sid = s.load_scene(n=10)
        t0 = time.perf_counter()
        ts = [s.submit(sid, CAM) for _ in range(8)]
        for t in ts:
            s.wait(t)
        dt = time.perf_counter() - t0
        st = s.stats()
        s.close()
        return dt, st
    d1, s1 = run(1)
    d4, s4 = run(4)
    assert s1["max_in_flight"] == 1 and s4["max_in_flight"] == 4
    assert d4 < 0.5 * d1
    assert s4["p99_ms"] < s1["p99_ms"]


def test_concurrent_submitters_are_safe(lib):
    s = _server(budget_bytes=1 << 40, slots=3, queue=4096, fake_us_per_mpix=1000.0)
    sid = s.load_scene(n=10)
    got = []
    lock = threading.Lock()

    def client():
        for _ in range(50):
            t = s.submit(sid, CAM)
            s.wait(t)
            with lock:
                got.append(t)

    ths = [threading.Thread(target=client) for _ in range(6)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    assert len(set(got)) == 300
    assert s.stats()["completed"] == 300
    s.close()


def test_invalid_arguments(lib):
    from paper_2411_16392_gb300._lib import QGSError
    s = _server(budget_bytes=1 << 30, slots=1)
    with pytest.raises(QGSError) as e:
        s.submit(3, CAM)                   # no such scene
    assert e.value.status == 7
    sid = s.load_scene(n=10)
    with pytest.raises(QGSError) as e:
        s.submit(sid, Camera(0, 10, 1.0, 1.0, 0.0, 0.0))
    assert e.value.status == 1
    huge = Camera(30000, 30000, 1e4, 1e4, 1.5e4, 1.5e4)
    with pytest.raises(QGSError) as e:
        s.submit(sid, huge)                # alone larger than the budget
    assert e.value.status == 3
    s.close()


def test_queued_views_of_one_scene_are_batched(lib):
    """One slot, batches of up to 4: while the first request runs, 8 more queue up and
    are taken 4 at a time; views of another scene never join them."""
    s = _server(budget_bytes=1 << 40, slots=1, batch=4, fake_us_per_mpix=1_000_000.0)  # ~65 ms per view
    a = s.load_scene(n=10)
    b = s.load_scene(n=10)
    ts = [s.submit(a, CAM)]
    time.sleep(0.02)
    ts += [s.submit(a, CAM) for _ in range(8)] + [s.submit(b, CAM)]
    for t in ts:
        s.wait(t)
    st = s.stats()
    assert st["completed"] == 10 and st["failed"] == 0
    assert st["max_batch"] == 4
    assert st["batches"] == 4          # [a], [a a a a], [a a a a], [b]
    assert st["max_in_flight"] == 4
    s.close()


def test_only_single_slot_servers_batch(lib):
    """Batching saves a view its launches and host round trip, which the other slots already
    hide: with two slots the queued views run as single renders in both slots; frames
    larger than 512x384 never batch, not even on one slot."""
    s = _server(budget_bytes=1 << 40, slots=2, batch=4, fake_us_per_mpix=1_000_000.0)
    a = s.load_scene(n=10)
    ts = [s.submit(a, CAM) for _ in range(8)]
    for t in ts:
        s.wait(t)
    st = s.stats()
    assert st["completed"] == 8 and st["max_batch"] == 1 and st["batches"] == 8
    assert st["max_in_flight"] == 2
    s.close()
    big = Camera(640, 480, 500.0, 500.0, 320.0, 240.0)
    s = _server(budget_bytes=1 << 40, slots=1, batch=4, fake_us_per_mpix=100_000.0)
    a = s.load_scene(n=10)
    ts = [s.submit(a, big) for _ in range(5)]
    for t in ts:
        s.wait(t)
    st = s.stats()
    assert st["completed"] == 5 and st["max_batch"] == 1
    s.close()


def test_batch_size_is_bounded_by_the_budget(lib):
    per = (10 * 168 + 64 * 65536 * 16 + 64 * 65536 / 16 + 65536 * 40) + (1 << 20)
    s = _server(budget_bytes=int(2.5 * per), slots=1, batch=8, fake_us_per_mpix=500_000.0)
    sid = s.load_scene(n=10)
    ts = [s.submit(sid, CAM)]
    time.sleep(0.01)
    ts += [s.submit(sid, CAM) for _ in range(6)]
    for t in ts:
        s.wait(t)
    st = s.stats()
    assert st["max_batch"] == 2 and st["max_in_flight"] == 2, st
    assert st["bytes_reserved_peak"] <= st["bytes_budget"]
    s.close()


def test_backward_requests_return_gradients_and_run_alone(lib):
    from paper_2411_16392_gb300._lib import QGSError
    s = _server(budget_bytes=1 << 40, slots=1, batch=8, fake_us_per_mpix=2_000_000.0)  # ~130 ms a view
    sid = s.load_scene(n=100)
    first = s.submit(sid, CAM)
    time.sleep(0.02)
    fwd = [s.submit(sid, CAM) for _ in range(3)]
    bwd = s.submit(sid, CAM, backward=True, grad_out={"rgb": np.ones((3, 256, 256), np.float32)})
    fwd += [s.submit(sid, CAM) for _ in range(2)]
    with pytest.raises(QGSError) as e:        # a forward ticket has no gradients
        s.wait(fwd[0], grads={"mean": np.zeros((100, 3), np.float32)})
    assert e.value.status == 1
    grads = {k: np.full(shape, 7.0, np.float32) for k, shape in
             (("mean", (100, 3)), ("quat", (100, 4)), ("scale", (100, 2)), ("curv", (100, 2)),
              ("opacity", (100,)), ("sh", (100, 48)))}
    s.wait(bwd, grads=grads)
    assert all(np.all(v == 0) for v in grads.values())   # host executor: zero gradients
    for t in [first] + fwd:
        s.wait(t)
    st = s.stats()
    assert st["completed"] == 7 and st["failed"] == 0
    assert st["batches"] == 3, st                          # [f], [f f f f f], [b]
    s.close()
