"""Serving: requests of mixed sizes and dimensions submitted together to the
request loop run concurrently on several slots, and each result must be
exactly the oracle's labels -- the same result the request gets when it runs
alone through ms_segment.  Admission must keep what the server holds on the
device -- the slots' resident scratch and the running requests -- within the
budget, measured with cudaMemGetInfo."""
import threading
import time

import numpy as np
import pytest

import oracle
import paper_2303_15491_gb300 as ms
import synthfields as sf
from gpu_util import assert_same_labels

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = ms.ms_create(0)
    yield h
    ms.ms_destroy(h)


def mixed_fields(n, seed):
    """Small 2D squares and 3D boxes, float32 and float16, noise and quantised."""
    out = []
    for i, (dims, sub) in enumerate(sf.serve_specs(n, seed=seed, two_d=(24, 180), three_d=(10, 44))):
        f = sf.smoothed_noise(dims, sub, sigma=2.5)
        if dims[2] == 1:
            f = f[0]
        if i % 3 == 1:
            f = sf.quantize_levels(f, 12)
        if i % 4 == 2:
            f = f.astype(np.float16)
        out.append(np.ascontiguousarray(f))
    return out


def submit_all(srv, fields):
    bufs = []
    for f in fields:
        dev = torch.from_numpy(f).cuda()
        outs = [torch.full((f.size,), -7, dtype=torch.int32, device="cuda") for _ in range(3)]
        bufs.append((dev, outs))
    torch.cuda.synchronize()  # the server's streams do not wait on torch's
    reqs = []
    for f, (dev, outs) in zip(fields, bufs):
        t = ms.ms_server_submit(srv, dev, ms.dims_of(f), ms.dtype_code(f), *outs)
        reqs.append((t, dev, outs))
    return reqs


def collect(srv, reqs):
    got = []
    for t, _, outs in reqs:
        st, k, lat = ms.ms_server_wait(srv, t, 60000)
        assert lat >= 0.0
        got.append((st, tuple(o.cpu().numpy() for o in outs), k))
    return got


@pytest.mark.parametrize("slots", [1, 3])
def test_served_results_match_oracle_and_alone(ctx, slots):
    fields = mixed_fields(16, seed=slots)
    assert any(f.ndim == 2 for f in fields) and any(f.ndim == 3 for f in fields)
    srv = ms.ms_server_create(0, 8 << 30, slots)
    try:
        got = collect(srv, submit_all(srv, fields))
        stats = ms.ms_server_stats(srv)
    finally:
        ms.ms_server_destroy(srv)
    assert stats["admitted"] == stats["completed"] == len(fields)
    assert stats["queued"] == 0 and stats["bytes_in_use"] == stats["resident_bytes"]
    for i, (f, (st, labels, k)) in enumerate(zip(fields, got)):
        assert st == 0, ms.STATUS[st]
        assert_same_labels((*labels, k), oracle.segment(f), f"served request {i} {f.shape} {f.dtype}")
        alone = ms.segment(ctx, torch.from_numpy(f).cuda())
        for a, b in zip(labels, alone[:3]):
            assert np.array_equal(a, b.cpu().numpy())
        assert k == alone[3]


def test_admission_keeps_within_budget(ctx):
    # each 48^3 float32 request is charged 16 bytes a vertex for its field and
    # labels plus its slot's scratch growth (estimated at 10 bytes a vertex plus
    # 64 MiB): a 100 MiB budget runs one at a time although three slots are idle
    fields = [sf.smoothed_noise((48, 48, 48), 70 + i, sigma=3.0) for i in range(5)]
    srv = ms.ms_server_create(0, 100 << 20, 3)
    try:
        got = collect(srv, submit_all(srv, fields))
        stats = ms.ms_server_stats(srv)
    finally:
        ms.ms_server_destroy(srv)
    one = 48 ** 3 * 26 + (64 << 20)
    assert one <= stats["peak_bytes"] <= stats["budget_bytes"]
    for f, (st, labels, k) in zip(fields, got):
        assert st == 0
        assert_same_labels((*labels, k), oracle.segment(f), "budgeted request")


def test_device_memory_stays_within_budget(ctx):
    """A mixed stream through three slots under a 320 MiB budget: the device
    memory the server allocates (cudaMemGetInfo, sampled while it runs, less
    what was in use before it started) never exceeds the budget, and the
    resident bytes it reports match what it holds at the end."""
    fields = mixed_fields(10, seed=21) + [sf.smoothed_noise((64, 60, 56), 400 + i, sigma=3.0)
                                          for i in range(4)]
    bufs = []
    for f in fields:
        dev = torch.from_numpy(f).cuda()
        bufs.append((dev, [torch.full((f.size,), -7, dtype=torch.int32, device="cuda")
                           for _ in range(3)]))
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    used0 = total - free0
    budget = 320 << 20
    peak = [0]
    stop = threading.Event()

    def sample():
        while not stop.is_set():
            free, tot = torch.cuda.mem_get_info()
            peak[0] = max(peak[0], tot - free - used0)
            time.sleep(0.002)

    th = threading.Thread(target=sample)
    srv = ms.ms_server_create(0, budget, 3)
    th.start()
    try:
        reqs = [(ms.ms_server_submit(srv, dev, ms.dims_of(f), ms.dtype_code(f), *outs), dev, outs)
                for f, (dev, outs) in zip(fields, bufs)]
        got = collect(srv, reqs)
        stats = ms.ms_server_stats(srv)
        free, tot = torch.cuda.mem_get_info()
        held = tot - free - used0
    finally:
        stop.set()
        th.join()
        ms.ms_server_destroy(srv)
    slack = 3 * (4 << 20)  # driver allocation granularity per slot
    assert stats["peak_bytes"] <= budget
    assert peak[0] <= budget + slack, (peak[0], budget)
    assert abs(held - stats["resident_bytes"]) <= slack, (held, stats["resident_bytes"])
    for i, (f, (st, labels, k)) in enumerate(zip(fields, got)):
        assert st == 0
        assert_same_labels((*labels, k), oracle.segment(f), f"request {i} {f.shape}")


def test_two_waiters_on_one_ticket(ctx):
    """Two threads wait on the same ticket: one receives the result, the
    other learns that the ticket is gone; neither hangs."""
    fields = mixed_fields(3, seed=31)
    srv = ms.ms_server_create(0, 8 << 30, 1)
    try:
        reqs = submit_all(srv, fields)
        t = reqs[-1][0]
        out = []

        def waiter():
            try:
                out.append(("ok", ms.ms_server_wait(srv, t, 60000)[0]))
            except ms.MSError as e:
                out.append(("err", e.name))

        ths = [threading.Thread(target=waiter) for _ in range(2)]
        for th in ths:
            th.start()
        for th in ths:
            th.join(timeout=120)
        assert not any(th.is_alive() for th in ths)
        for tk, _, _ in reqs[:-1]:
            assert ms.ms_server_wait(srv, tk, -1)[0] == 0
    finally:
        ms.ms_server_destroy(srv)
    assert sorted(out) == [("err", "MS_ERR_INVALID_ARG"), ("ok", 0)], out


def test_large_requests_are_not_starved(ctx):
    # one large request among many small ones: with room for the large one only
    # when nothing else runs, it must still complete (small ones may pass it a
    # bounded number of times)
    big = sf.smoothed_noise((64, 64, 64), 81, sigma=3.0)
    small = [sf.smoothed_noise((20, 24, 16), 90 + i, sigma=2.0) for i in range(30)]
    est_big = big.size * 26 + (64 << 20)
    est_small = small[0].size * 26 + (64 << 20)
    srv = ms.ms_server_create(0, est_big + est_small, 2)
    try:
        reqs = submit_all(srv, small[:3] + [big] + small[3:])
        got = collect(srv, reqs)
    finally:
        ms.ms_server_destroy(srv)
    for f, (st, labels, k) in zip(small[:3] + [big] + small[3:], got):
        assert st == 0
        assert_same_labels((*labels, k), oracle.segment(f), f"request {f.shape}")


def test_failed_request_leaves_the_others_intact(ctx):
    fields = mixed_fields(6, seed=9)
    bad = fields[3].copy()
    bad.flat[bad.size // 2] = np.nan
    fields[3] = bad
    srv = ms.ms_server_create(0, 8 << 30, 2)
    try:
        got = collect(srv, submit_all(srv, fields))
    finally:
        ms.ms_server_destroy(srv)
    for i, (f, (st, labels, k)) in enumerate(zip(fields, got)):
        if i == 3:
            assert ms.STATUS[st] == "MS_ERR_NAN_INPUT"
        else:
            assert st == 0
            assert_same_labels((*labels, k), oracle.segment(f), f"request {i}")


def test_server_argument_errors(ctx):
    srv = ms.ms_server_create(0, 1 << 20, 1)
    try:
        f = torch.zeros(64 * 64 * 64, device="cuda")
        o = [torch.empty(64 ** 3, dtype=torch.int32, device="cuda") for _ in range(3)]
        with pytest.raises(ms.MSError) as e:  # estimate above the whole budget
            ms.ms_server_submit(srv, f, (64, 64, 64), 0, *o)
        assert e.value.name == "MS_ERR_TOO_LARGE"
        with pytest.raises(ms.MSError) as e:
            ms.ms_server_wait(srv, 12345, 0)
        assert e.value.name == "MS_ERR_INVALID_ARG"
        with pytest.raises(ms.MSError) as e:
            ms.ms_server_submit(srv, f, (0, 64, 64), 0, *o)
        assert e.value.name == "MS_ERR_INVALID_ARG"
    finally:
        ms.ms_server_destroy(srv)
    for bad in [(-1, 1 << 30, 1), (0, 0, 1), (0, 1 << 30, 0), (0, 1 << 30, 65)]:
        with pytest.raises(ms.MSError):
            ms.ms_server_create(*bad)


def test_wait_with_timeout_then_release(ctx):
    fields = mixed_fields(4, seed=13)
    srv = ms.ms_server_create(0, 8 << 30, 1)
    try:
        reqs = submit_all(srv, fields)
        t_last = reqs[-1][0]
        try:  # may already be done; either answer is valid
            ms.ms_server_wait(srv, t_last, 0)
            released = True
        except ms.MSError as e:
            assert e.name == "MS_ERR_TIMEOUT"
            released = False
        for t, _, _ in reqs[:-1]:
            assert ms.ms_server_wait(srv, t, -1)[0] == 0
        if not released:
            assert ms.ms_server_wait(srv, t_last, -1)[0] == 0
        with pytest.raises(ms.MSError) as e:  # a ticket is released by its wait
            ms.ms_server_wait(srv, t_last, 0)
        assert e.value.name == "MS_ERR_INVALID_ARG"
    finally:
        ms.ms_server_destroy(srv)


def test_large_requests_run_one_at_a_time_with_small_ones_beside(ctx):
    """Two requests of at least 2^25 vertices (run one at a time) among small
    ones: every result equals the request run alone."""
    big = [torch.randn(6000 * 6000, device="cuda").view(6000, 6000) for _ in range(2)]
    small = [torch.from_numpy(sf.smoothed_noise((40, 30, 20), 300 + i, sigma=2.0)).cuda()
             for i in range(6)]
    fields = [big[0], small[0], small[1], big[1]] + small[2:]
    outs = [[torch.full((f.numel(),), -3, dtype=torch.int32, device="cuda") for _ in range(3)]
            for f in fields]
    torch.cuda.synchronize()
    srv = ms.ms_server_create(0, 64 << 30, 4)
    try:
        tickets = [ms.ms_server_submit(srv, f, ms.dims_of(f), 0, *o) for f, o in zip(fields, outs)]
        res = [ms.ms_server_wait(srv, t, 120000) for t in tickets]
        stats = ms.ms_server_stats(srv)
    finally:
        ms.ms_server_destroy(srv)
    assert stats["completed"] == len(fields)
    for f, o, (st, k, _) in zip(fields, outs, res):
        assert st == 0
        alone = ms.segment(ctx, f)
        for a, b in zip(o, alone[:3]):
            assert torch.equal(a, b)
        assert k == alone[3]
