"""Batched uneven-N evaluation (sre_m2_batched) on the GPU.

* every result equals the single-state evaluation bit for bit (same
  per-tile / per-chunk partials, same fixed-order finalize);
* a state gives the same M2 alone and inside a mixed batch;
* results match the FP64 oracle within the FP32 / FP64 tolerances;
* a repeated submission replays the captured CUDA graph with identical
  results; a bad state yields NaN without disturbing the others.
"""
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


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def mixed_states(spec, dtype=np.complex64):
    return [W.brickwork_state(n, depth, seed).astype(dtype) for n, depth, seed in spec]


SPEC = [(3, 2, 1), (12, 4, 2), (9, 3, 3), (14, 6, 4), (13, 2, 5), (1, 1, 6), (16, 8, 7),
        (14, 3, 8), (12, 5, 9), (5, 2, 10), (13, 7, 11), (15, 4, 12)]


def test_batch_equals_single_bitwise_and_oracle(sre, torch_cuda):
    torch = torch_cuda
    states = mixed_states(SPEC)
    ts = [dev(torch, v) for v in states]
    with sre.Plan(16, "c64") as p:
        out = p.m2_batched(ts)
        torch.cuda.synchronize()
        singles = [p.m2(t) for t in ts]
    got = out.cpu().numpy()
    for v, g, s in zip(states, got, singles):
        assert g == s, (v.size, g, s)  # bitwise
        assert abs(g - oracle.m2(v)) <= 1e-6


def test_alone_equals_in_mix(sre, torch_cuda):
    torch = torch_cuda
    states = mixed_states(SPEC)
    ts = [dev(torch, v) for v in states]
    with sre.Plan(16, "c64") as p:
        mix = p.m2_batched(ts).cpu().numpy()
        for k in (0, 3, 6, 11):
            alone = p.m2_batched([ts[k]]).cpu().numpy()[0]
            assert alone == mix[k]
        # a different mix (reordered, with duplicates)
        order = [6, 6, 3, 0, 11, 2, 3]
        mix2 = p.m2_batched([ts[k] for k in order]).cpu().numpy()
        for j, k in enumerate(order):
            assert mix2[j] == mix[k]


def test_graph_replay_and_launch_count(sre, torch_cuda):
    torch = torch_cuda
    states = mixed_states(SPEC[:6])
    ts = [dev(torch, v) for v in states]
    out = torch.empty(len(ts), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()  # capturable stream: replays come from the CUDA graph
    torch.cuda.synchronize()
    with sre.Plan(16, "c64") as p, torch.cuda.stream(side):
        p.m2_batched(ts, out=out)
        side.synchronize()
        first = out.clone()
        c0 = p.launch_count()
        for _ in range(3):
            out.fill_(float("nan"))
            p.m2_batched(ts, out=out)
            side.synchronize()
            assert torch.equal(out, first)
        assert p.launch_count() > c0
        singles = [p.m2(t) for t in ts]
    assert first.cpu().tolist() == singles


def test_fp64_batch(sre, torch_cuda):
    torch = torch_cuda
    spec = [(6, 2, 20), (13, 3, 21), (11, 4, 22), (14, 2, 23)]
    states = mixed_states(spec, np.complex128)
    ts = [dev(torch, v) for v in states]
    with sre.Plan(14, "c128", "fp64") as p:
        got = p.m2_batched(ts).cpu().numpy()
        singles = [p.m2(t) for t in ts]
    for v, g, s in zip(states, got, singles):
        assert g == s
        assert abs(g - oracle.m2(v)) <= 1e-10


def test_converted_batch(sre, torch_cuda):
    """complex128 states evaluated in FP32 mode (converted on the device)."""
    torch = torch_cuda
    spec = [(8, 2, 30), (13, 3, 31), (12, 2, 32)]
    states = mixed_states(spec, np.complex128)
    with sre.Plan(13, "c128", "fp32") as p:
        got = p.m2_batched([dev(torch, v) for v in states]).cpu().numpy()
    for v, g in zip(states, got):
        assert abs(g - oracle.m2(v)) <= 1e-6


def test_bad_state_in_batch(sre, torch_cuda):
    torch = torch_cuda
    good = mixed_states([(10, 3, 40), (13, 2, 41)])
    ts = [dev(torch, v) for v in good]
    zero = torch.zeros(1 << 12, dtype=torch.complex64, device="cuda")
    nan = dev(torch, W.haar_state(13, 42, np.complex64))
    nan[7] = float("nan")
    with sre.Plan(13, "c64") as p:
        got = p.m2_batched([ts[0], zero, ts[1], nan]).cpu().numpy()
    assert np.isnan(got[1]) and np.isnan(got[3])
    assert abs(got[0] - oracle.m2(good[0])) <= 1e-6
    assert abs(got[2] - oracle.m2(good[1])) <= 1e-6


def test_uneven_batch_workload_sample(sre, torch_cuda):
    """A reduced instance of the uneven batched workload (brickwork Haar
    circuits, N ~ U{12..16}, depth ~ U{1..32}); oracle on a sample."""
    torch = torch_cuda
    spec = W.uneven_batch_spec(count=40, n_lo=12, n_hi=16)
    states = [W.brickwork_state(n, t, s).astype(np.complex64) for n, t, s in spec]
    with sre.Plan(16, "c64") as p:
        got = p.m2_batched([dev(torch, v) for v in states]).cpu().numpy()
    for k in range(0, 40, 7):
        assert abs(got[k] - oracle.m2(states[k])) <= 1e-6
    assert np.all(np.isfinite(got)) and np.all(got >= -1e-6)


@pytest.mark.parametrize("mode", ["fp16_split", "bf16_split"])
def test_split_mode_batch(sre, torch_cuda, mode):
    """Split modes in a batch: the N = 16..18 classes take the tensor-core
    kernel with per-state scale tables; every result equals the state's
    single evaluation in the same mode bit for bit, and the oracle within
    1e-6; a replay from the captured graph gives the same values."""
    torch = torch_cuda
    spec = [(17, 12, 21), (12, 4, 22), (16, 9, 23), (18, 14, 24), (16, 3, 25), (14, 5, 26), (17, 2, 27),
            (16, 16, 28)]
    states = mixed_states(spec)
    ts = [dev(torch, v) for v in states]
    with sre.Plan(18, "c64", mode) as p:
        out = p.m2_batched(ts)
        torch.cuda.synchronize()
        first = out.cpu().numpy().copy()
        again = p.m2_batched(ts).cpu().numpy()
        singles = [p.m2(t) for t in ts]
    for v, g, s, r in zip(states, first, singles, again):
        assert g == s, (v.size, g, s)
        assert r == g
        if v.size <= 1 << 16:
            assert abs(g - oracle.m2(v)) <= 1e-6, (v.size, g)


def test_split_mode_batch_converted(sre, torch_cuda):
    """complex128 states batched in the FP16 split mode (converted to
    complex64 on the device, then the tensor-core kernel for N = 16, 17):
    each equals its single evaluation in that mode bit for bit."""
    torch = torch_cuda
    spec = [(16, 6, 41), (13, 3, 42), (17, 9, 43)]
    states = mixed_states(spec, np.complex128)
    ts = [dev(torch, v) for v in states]
    with sre.Plan(17, "c128", "fp16_split") as p:
        got = p.m2_batched(ts).cpu().numpy()
        singles = [p.m2(t) for t in ts]
    for v, g, s in zip(states, got, singles):
        assert g == s, (v.size, g, s)
        if v.size <= 1 << 13:
            assert abs(g - oracle.m2(v)) <= 1e-6
