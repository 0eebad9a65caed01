"""Continuous-batching server (sre_server_*) and bounded device waits, on the GPU.

* requests of mixed N submitted while others run all complete, and each
  result equals the state's M2 evaluated alone (same tolerance as the
  single-state path; in practice bit for bit) and the oracle;
* admission by HBM bytes rejects what does not fit (SRE_EBUSY);
* a bad state comes back as NaN, an unknown ticket as SRE_ENOTFOUND;
* a device wait that nothing satisfies ends with SRE_ETIMEDOUT and leaves
  the context usable;
* a merged batch whose device wait expired reports SRE_ETIMEDOUT for its
  requests.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2512_24685_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def sre():
    from paper_2512_24685_gb300 import binding
    binding.load_library()
    return binding


def test_wait_timeout_is_reported(sre, torch_cuda):
    t0 = time.perf_counter()
    st = sre.selftest_wait_timeout(200_000_000)  # 0.2 s
    dt = time.perf_counter() - t0
    assert st == 7  # SRE_ETIMEDOUT
    assert 0.1 < dt < 30
    # the context is still usable
    psi = W.haar_state(10, 1, np.complex64)
    with sre.Plan(10) as p:
        assert abs(p.m2(torch_cuda.from_numpy(psi).cuda()) - oracle.m2(psi)) <= 1e-6


def test_server_mixed_requests(sre, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(5)
    Ns = [10, 14, 12, 17, 11, 13, 15, 10, 16, 12, 18, 11, 13, 14, 10, 12]
    states = []
    for k, n in enumerate(Ns):
        fam = k % 4
        if fam == 0:
            v = W.haar_state(n, 500 + k, np.complex64)
        elif fam == 1:
            v = W.product_state(n, 500 + k, np.complex64)[0]
        elif fam == 2:
            v = W.stabilizer_state(n, 500 + k, depth=6, dtype=np.complex64)
        else:
            v = W.brickwork_state(n, 4, 500 + k, np.complex64)
        states.append(v)
    # alone values through the single-state path (default tuning, like the server)
    alone = []
    for v in states:
        with sre.Plan(v.size.bit_length() - 1, "c64") as p:
            alone.append(p.m2(torch.from_numpy(v).cuda()))
    with sre.Server(max_inflight=3, max_N=18, hbm_budget_bytes=8 << 30) as srv:
        tickets = []
        for k, v in enumerate(states):
            src = torch.from_numpy(v).cuda() if k % 2 else v  # device and host submissions
            tickets.append(srv.submit(src))
            if k % 5 == 4:
                time.sleep(0.002)  # arrivals while earlier requests run
        got = [srv.wait(t, 60000) for t in tickets]
        st = srv.stats()
    for v, g, a in zip(states, got, alone):
        assert abs(g - a) <= 1e-12, (v.size, g, a)
        if v.size <= 1 << 14:
            assert abs(g - oracle.m2(v)) <= 1e-6
    assert st["completed"] == len(Ns) and st["failed"] == 0
    assert st["p99_latency_ms"] >= st["p50_latency_ms"] > 0
    assert st["admitted"] == len(Ns)


def test_server_poll_errors_and_admission(sre, torch_cuda):
    with sre.Server(max_inflight=2, max_N=14, hbm_budget_bytes=1 << 30) as srv:
        good = W.haar_state(12, 9, np.complex64)
        t_good = srv.submit(good)
        t_zero = srv.submit(np.zeros(1 << 11, dtype=np.complex64))
        with pytest.raises(sre.SreError) as e:
            srv.submit(np.ones(1 << 15, dtype=np.complex64))  # N above max_N
        assert e.value.status == 1
        while not srv.poll(t_good)[0]:
            time.sleep(0.001)
        z = srv.wait(t_zero, 60000)
        assert np.isnan(z)
        with pytest.raises(sre.SreError) as e:
            srv.poll(t_good)  # a done ticket is forgotten after it was polled done
        assert e.value.status == 9  # SRE_ENOTFOUND
    with pytest.raises(sre.SreError):
        sre.Server(max_inflight=2, max_N=20, hbm_budget_bytes=1 << 20)  # scratch exceeds budget


def test_server_admission_by_hbm_bytes(sre, torch_cuda):
    with sre.Server(max_inflight=1, max_N=16, hbm_budget_bytes=1 << 32) as srv:
        slot_bytes = srv.stats()["resident_bytes"]
    small = W.haar_state(14, 4, np.complex64)           # 128 KiB
    big = W.haar_state(16, 5, np.complex64)             # 512 KiB
    with sre.Server(max_inflight=1, max_N=16, hbm_budget_bytes=slot_bytes + (300 << 10)) as srv:
        with pytest.raises(sre.SreError) as e:
            srv.submit(big)
        assert e.value.status == 6  # SRE_EBUSY: does not fit the budget
        t = srv.submit(small)
        assert abs(srv.wait(t, 60000) - oracle.m2(small)) <= 1e-6
        st = srv.stats()
        assert st["rejected"] == 1 and st["completed"] == 1
        assert st["peak_resident_bytes"] <= slot_bytes + (300 << 10)


def _poll_status(sre, srv, ticket, timeout_s=60.0):
    """(status, m2) of a finished ticket through sre_server_poll."""
    end = time.perf_counter() + timeout_s
    while time.perf_counter() < end:
        try:
            done, m = srv.poll(ticket)
        except sre.SreError as e:
            return e.status, float("nan")
        if done:
            return 0, m
        time.sleep(0.001)
    raise AssertionError("request did not finish")


def test_server_merged_batch_reports_device_timeout(sre, torch_cuda):
    """A merged batch of N = 16 requests (two-pass kernel, bounded device
    waits) under a 1 ns wait limit: a request whose batch had a wait expire
    comes back from poll as SRE_ETIMEDOUT, not as SRE_OK with a NaN, and one
    whose batch finished has the correct M2."""
    states = [W.haar_state(16, 900 + k, np.complex64) for k in range(8)]
    with sre.Server(max_inflight=1, max_N=16, hbm_budget_bytes=4 << 30, wait_limit_ns=1) as srv:
        tickets = [srv.submit(v) for v in states]
        res = [_poll_status(sre, srv, t) for t in tickets]
        st = srv.stats()
    statuses = [s for s, _ in res]
    assert set(statuses) <= {0, 7}, statuses
    assert 7 in statuses, statuses
    assert st["failed"] == statuses.count(7)
    for (s, m), v in zip(res, states):
        if s == 0:
            assert abs(m - oracle.m2(v)) <= 1e-6
    # the server stays usable with an ordinary limit afterwards
    with sre.Server(max_inflight=1, max_N=16) as srv:
        assert abs(srv.wait(srv.submit(states[0]), 60000) - oracle.m2(states[0])) <= 1e-6


def test_server_chunked_requests_and_tuning(sre, torch_cuda):
    """Requests with N > 16 split into shift ranges (chunk_terms) come back
    with the M2 of the whole state (partial sums added in range order), and
    a tuning set for an N applies to its units; a ring larger than the
    slot scratch is refused."""
    torch = torch_cuda
    Ns = [18, 12, 17, 10, 18, 14, 17]
    states = [W.haar_state(n, 700 + k, np.complex64) for k, n in enumerate(Ns)]
    alone = []
    for v in states:
        with sre.Plan(v.size.bit_length() - 1, "c64") as p:
            alone.append(p.m2(torch.from_numpy(v).cuda()))
    with sre.Plan(18, "c64") as p:
        tun18, _ = p.autotune(18)
    with sre.Server(max_inflight=3, max_N=18, chunk_terms=1 << 33,
                    slot_scratch_bytes=256 << 20) as srv:
        srv.set_tuning(18, tun18)
        with pytest.raises(sre.SreError) as e:
            srv.set_tuning(18, {"x_batch_log": 3, "ring_slots": 47, "lag": 5})  # 394 MB ring
        assert e.value.status == 1
        tickets = [srv.submit(v) for v in states]
        got = [srv.wait(t, 120000) for t in tickets]
        st = srv.stats()
    for n, g, a, v in zip(Ns, got, alone, states):
        assert abs(g - a) <= 1e-9, (n, g, a)
        if n <= 14:
            assert abs(g - oracle.m2(v)) <= 1e-6
    assert st["completed"] == len(Ns) and st["failed"] == 0 and st["admitted"] == len(Ns)


def test_server_split_mode(sre, torch_cuda):
    """A server in the FP16 split mode: N = 17 requests take the tensor-core
    kernel (bitwise the plan's result in that mode), small ones the merged
    FP32 launches."""
    torch = torch_cuda
    states = [W.haar_state(17, 811, np.complex64), W.haar_state(11, 812, np.complex64),
              W.haar_state(17, 813, np.complex64)]
    want = []
    for v in states:
        n = v.size.bit_length() - 1
        with sre.Plan(n, "c64", "fp16_split" if n == 17 else "fp32") as p:
            want.append(p.m2(torch.from_numpy(v).cuda()))
    with sre.Server(max_inflight=2, max_N=17, mode="fp16_split") as srv:
        got = [srv.wait(srv.submit(v), 120000) for v in states]
    for g, w in zip(got, want):
        assert abs(g - w) <= 1e-12, (g, w)
    assert abs(got[1] - oracle.m2(states[1])) <= 1e-6


def test_server_split_mode_chunked(sre, torch_cuda):
    """The bench's serving configuration: FP16 split server, requests with
    N > 16 split into shift ranges; each result matches the state's single
    evaluation in that mode (range partial sums added in order: 1e-9)."""
    torch = torch_cuda
    states = [W.haar_state(18, 821, np.complex64), W.haar_state(12, 822, np.complex64),
              W.brickwork_state(17, 10, 823, np.complex64), W.haar_state(18, 824, np.complex64)]
    want = []
    for v in states:
        n = v.size.bit_length() - 1
        with sre.Plan(n, "c64", "fp16_split" if n > 16 else "fp32") as p:
            want.append(p.m2(torch.from_numpy(v).cuda()))
    with sre.Server(max_inflight=3, max_N=18, mode="fp16_split", chunk_terms=1 << 33) as srv:
        got = [srv.wait(t, 120000) for t in [srv.submit(v) for v in states]]
        st = srv.stats()
    for g, w in zip(got, want):
        assert abs(g - w) <= 1e-9, (g, w)
    assert st["completed"] == len(states) and st["failed"] == 0
