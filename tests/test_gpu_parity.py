"""GPU parity: libsre (through the C ABI) against the FP64 oracle on the same
seeded inputs.

Tolerances (|Delta M2|): 1e-10 for the FP64 path, 1e-6 for the FP32 path.
Per-shift sums sum_z |A_x(z)|^4 are compared relative to the largest one:
the FP32 arithmetic carries ~1e-7 relative error per stage.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2512_24685_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "fp64": 1e-10}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.fixture(scope="module")
def sre():
    from paper_2512_24685_gb300 import binding
    binding.load_library()
    return binding


def dev(torch, psi):
    return torch.from_numpy(np.ascontiguousarray(psi)).cuda()


def rand_state(N, seed, normalise=True, dtype=np.complex128):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << N) + 1j * rng.standard_normal(1 << N)
    if normalise:
        v /= np.linalg.norm(v)
    return v.astype(dtype)


def gpu_m2(sre, torch, psi, mode):
    dt = "c64" if psi.dtype == np.complex64 else "c128"
    N = psi.size.bit_length() - 1
    with sre.Plan(N, dt, mode) as p:
        return p.m2(dev(torch, psi))


# ------------------------------------------------------------------ parity

@pytest.mark.parametrize("N", list(range(1, 13)))
@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_small_n_random_states(sre, torch_cuda, N, mode):
    """Single-tile path (N <= 12): every N, normalised and unnormalised."""
    for seed, norm in ((10 * N + 1, True), (10 * N + 2, False)):
        psi = rand_state(N, seed, norm, np.complex64 if mode == "fp32" else np.complex128)
        ref = oracle.m2(psi, "direct" if N <= 6 else "xorfwht")
        got = gpu_m2(sre, torch_cuda, psi, mode)
        assert abs(got - ref) <= TOL[mode], (N, mode, got, ref, got - ref)


@pytest.mark.parametrize("N", [13, 14, 15])
@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_two_pass_path(sre, torch_cuda, N, mode):
    """Persistent two-pass path (N > 12): Haar and unnormalised states."""
    for psi in (W.haar_state(N, 100 + N), rand_state(N, 200 + N, normalise=False)):
        psi = psi.astype(np.complex64 if mode == "fp32" else np.complex128)
        ref = oracle.m2(psi, "xorfwht")
        got = gpu_m2(sre, torch_cuda, psi, mode)
        assert abs(got - ref) <= TOL[mode], (N, mode, got - ref)


@pytest.mark.parametrize("N", [4, 12, 13])
def test_cross_dtype_modes(sre, torch_cuda, N):
    """complex128 state in FP32 mode (rounded on device) and complex64 state
    in FP64 mode (widened exactly) both match the oracle."""
    psi128 = W.haar_state(N, 7 * N)
    psi64 = psi128.astype(np.complex64)
    with sre.Plan(N, "c128", "fp32") as p:
        got = p.m2(dev(torch_cuda, psi128))
    assert abs(got - oracle.m2(psi128)) <= TOL["fp32"]
    with sre.Plan(N, "c64", "fp64") as p:
        got = p.m2(dev(torch_cuda, psi64))
    assert abs(got - oracle.m2(psi64)) <= TOL["fp64"]


@pytest.mark.parametrize("N", [8, 13, 16])
def test_product_states_closed_form(sre, torch_cuda, N):
    """Product states: M2 = -sum_q log2((1 + x^4 + y^4 + z^4)/2) (additivity)."""
    for j in range(2):
        psi, bloch = W.product_state(N, W.config_seed(1, 16 + j), np.complex64)
        expect = float(-np.sum(np.log2((1 + np.sum(bloch ** 4, axis=1)) / 2)))
        assert abs(gpu_m2(sre, torch_cuda, psi, "fp32") - expect) <= TOL["fp32"]


@pytest.mark.parametrize("N", [10, 13, 16])
def test_stabilizer_states_zero(sre, torch_cuda, N):
    psi = W.stabilizer_state(N, W.config_seed(1, 32))
    assert abs(gpu_m2(sre, torch_cuda, psi.astype(np.complex64), "fp32")) <= TOL["fp32"]
    assert abs(gpu_m2(sre, torch_cuda, psi, "fp64")) <= TOL["fp64"]


@pytest.mark.parametrize("N", [13, 14, 15])
def test_per_shift_sums(sre, torch_cuda, N):
    """sum_z |A_x(z)|^4 for every shift x equals the oracle's Algorithm-1 loop."""
    psi = W.haar_state(N, 31 * N)
    _, ref = oracle.sum4_xorfwht(psi, per_x=True)
    for mode, rtol in (("fp64", 1e-12), ("fp32", 2e-6)):
        with sre.Plan(N, "c128", mode) as p:
            out, px = p.sum4_range(dev(torch_cuda, psi), 0, 1 << N, per_x=True)
            torch_cuda.cuda.synchronize()
        np.testing.assert_allclose(px.cpu().numpy(), ref, rtol=0, atol=rtol * ref.max())
        # FP32 mode evaluates the state rounded to complex64
        n2 = oracle.norm2(psi if mode == "fp64" else psi.astype(np.complex64))
        assert out[1].item() == pytest.approx(n2, rel=1e-12)


@pytest.mark.parametrize("N,ranges", [(9, [(0, 5), (5, 300), (300, 512)]),
                                      (13, [(0, 1), (1, 4099), (4099, 8000), (8000, 8192)])])
def test_shift_ranges_partition(sre, torch_cuda, N, ranges):
    """Shift-range shards (ragged, unaligned) add up to the full sum and match
    the oracle's sums over the same ranges."""
    psi = W.haar_state(N, 55)
    t = dev(torch_cuda, psi)
    with sre.Plan(N, "c128", "fp64") as p:
        tot = 0.0
        for a, b in ranges:
            s = p.sum4_range(t, a, b)[0].item()
            assert s == pytest.approx(oracle.sum4_xorfwht(psi, a, b), rel=1e-12)
            tot += s
        full = p.sum4_range(t, 0, 1 << N)[0].item()
    assert tot == pytest.approx(full, rel=1e-13)


def test_deterministic_bitwise(sre, torch_cuda):
    """Fixed-order reductions: repeated evaluations agree bit for bit."""
    for N in (11, 14):
        psi = W.haar_state(N, 3).astype(np.complex64)
        t = dev(torch_cuda, psi)
        with sre.Plan(N, "c64") as p:
            vals = {p.m2(t) for _ in range(3)}
        assert len(vals) == 1


@pytest.mark.parametrize("N,tuning,xr", [
    (14, (0, 9, 4, 1, 1), (0, 1 << 14)),
    (17, (0, 15, 7, 2, 2), (0, 1 << 17)),
    (20, (0, 23, 11, 2, 2), (4096 - 64, 4096 + 2048)),
])
def test_staged_and_register_pass1_agree(sre, torch_cuda, N, tuning, xr):
    """One shift per chunk: a 16-byte aligned state takes its pass-1 block
    pairs by bulk copy into shared memory, the same state at an 8-byte offset
    by per-thread loads.  Both paths do the same arithmetic in the same
    order, so the per-shift sums agree bit for bit."""
    torch = torch_cuda
    psi = torch.from_numpy(W.haar_state(N, 77, np.complex64)).cuda()
    pad = torch.zeros((1 << N) + 1, dtype=torch.complex64, device="cuda")
    pad[1:] = psi
    shifted = pad[1:]
    assert psi.data_ptr() % 16 == 0 and shifted.data_ptr() % 16 == 8
    with sre.Plan(N, "c64") as p:
        p.set_tuning(*tuning)
        out_a, px_a = p.sum4_range(psi, xr[0], xr[1], per_x=True)
        out_b, px_b = p.sum4_range(shifted, xr[0], xr[1], per_x=True)
        torch.cuda.synchronize()
    assert torch.equal(px_a, px_b)
    assert torch.equal(out_a, out_b)
    ref = oracle.sum4_xorfwht(psi.cpu().numpy(), xr[1] - 1, xr[1])
    assert abs(px_a[-1].item() - ref) <= 1e-5 * ref


@pytest.mark.parametrize("N,tuning", [
    (18, (2, 23, 11, 2, 0)),
    (20, (0, 23, 11, 3, 2)),
])
def test_copy_paths_agree(sre, torch_cuda, N, tuning):
    """Pass-2 tiles by TMA copy or by per-thread loads, and pass-1 blocks by
    bulk copy or by per-thread loads: every combination gives per-shift sums
    within FP32 rounding of each other and of the FP64 oracle; the two
    pass-1 paths alone give identical sums."""
    torch = torch_cuda
    psi_np = W.haar_state(N, 91, np.complex64)
    psi = torch.from_numpy(psi_np).cuda()
    xr = (4096 - 32, 4096 + 1024)
    res = {}
    with sre.Plan(N, "c64") as p:
        for s1 in (0, 1):
            for s2 in (0, 1):
                p.set_tuning(*tuning, s1, s2)
                _, px = p.sum4_range(psi, xr[0], xr[1], per_x=True)
                res[(s1, s2)] = px.cpu().numpy()
    for s2 in (0, 1):
        assert np.array_equal(res[(0, s2)], res[(1, s2)])
    ref = res[(0, 0)]
    assert np.max(np.abs(res[(1, 1)] - ref)) <= 1e-6 * np.max(ref)
    for x in (xr[0], 4095, 4096, xr[1] - 1):
        o = oracle.sum4_xorfwht(psi_np, x, x + 1)
        for v in res.values():
            assert abs(v[x - xr[0]] - o) <= 1e-5 * o


# -------------------------------------------------- full-size (N = 20) checks

def test_n20_full_size_sampled(sre, torch_cuda):
    """N = 20 Haar state, complex64, FP32 path in the benchmark's launch
    configuration: per-shift sums on sampled shifts against the oracle, S
    equals the sum of the per-shift sums, and M2 sits at the Haar value."""
    N = 20
    psi = W.haar_state(N, W.config_seed(2, 0), np.complex64)
    t = dev(torch_cuda, psi)
    with sre.Plan(N, "c64") as p:
        p.autotune(N)  # as bench.py does before timing
        m2 = p.m2(t)
        out, px = p.sum4_range(t, 0, 1 << N, per_x=True)
        torch_cuda.cuda.synchronize()
    px = px.cpu().numpy()
    S = out[0].item()
    assert S == pytest.approx(float(np.sum(px)), rel=1e-12)
    assert m2 == pytest.approx(-(math.log2(S) - N - 4 * math.log2(out[1].item())), abs=1e-12)
    rng = np.random.default_rng(2020)
    sample = sorted(set([0, 1, 4095, 4096, (1 << N) - 1] + list(rng.integers(0, 1 << N, 27))))
    for x in sample:
        ref = oracle.sum4_xorfwht(psi, int(x), int(x) + 1)
        assert abs(px[x] - ref) <= 1e-5 * ref, (x, px[x], ref)
    # Haar states concentrate: 2^-M2 = S/(d n2^4) within a few percent of 4/(d+3)
    assert abs(2.0 ** (-m2) / (4 / ((1 << N) + 3)) - 1) < 0.05


# ------------------------------------------------------------- edge cases

def test_error_statuses(sre, torch_cuda):
    torch = torch_cuda
    with sre.Plan(6, "c64") as p:
        z = torch.zeros(64, dtype=torch.complex64, device="cuda")
        with pytest.raises(sre.SreError) as e:
            p.m2(z)
        assert e.value.status == 3  # SRE_EZERO
        bad = torch.ones(64, dtype=torch.complex64, device="cuda")
        bad[5] = float("nan")
        with pytest.raises(sre.SreError) as e:
            p.m2(bad)
        assert e.value.status == 4  # SRE_ENONFINITE
        inf = torch.ones(64, dtype=torch.complex64, device="cuda")
        inf[63] = complex(float("inf"), 0)
        with pytest.raises(sre.SreError) as e:
            p.m2(inf)
        assert e.value.status == 4
        big = torch.ones(128, dtype=torch.complex64, device="cuda")
        with pytest.raises(sre.SreError) as e:
            p.m2(big)  # N = 7 > plan N = 6
        assert e.value.status == 1
        # a misaligned device pointer is rejected before any launch
        lib = sre.load_library()
        import ctypes
        st = lib.sre_m2(p._h, ctypes.c_void_p(bad.data_ptr() + 4), 6, None, ctypes.byref(ctypes.c_double()))
        assert st == 2  # SRE_EALIGN
        with pytest.raises(sre.SreError):
            p.sum4_range(bad, 10, 10)
        with pytest.raises(sre.SreError):
            p.sum4_range(bad, 0, 65)
        # the plan still works after data errors
        ok = torch.ones(64, dtype=torch.complex64, device="cuda")
        assert abs(p.m2(ok)) < 1e-6  # |+>^6 is a stabilizer state


def test_single_qubit_and_host_entry(sre, torch_cuda):
    s = 1 / math.sqrt(2)
    T = np.array([s, s * np.exp(1j * np.pi / 4)], dtype=np.complex64)
    with sre.Plan(1, "c64") as p:
        assert abs(p.m2(dev(torch_cuda, T)) - math.log2(4 / 3)) <= TOL["fp32"]
        assert abs(p.m2_host(T) - math.log2(4 / 3)) <= TOL["fp32"]
    psi = W.haar_state(14, 9)
    with sre.Plan(14, "c128") as p:
        assert abs(p.m2_host(psi) - oracle.m2(psi)) <= TOL["fp64"]


def test_async_entry(sre, torch_cuda):
    torch = torch_cuda
    psi = W.haar_state(13, 77).astype(np.complex64)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    with sre.Plan(13, "c64") as p:
        p.m2_async(dev(torch, psi), out)
        torch.cuda.synchronize()
    assert abs(out.item() - oracle.m2(psi)) <= TOL["fp32"]


def test_batched_uneven_matches_single(sre, torch_cuda):
    torch = torch_cuda
    spec = [(3, 0), (12, 1), (9, 2), (14, 3), (13, 4), (1, 5), (16, 6)]
    states = [W.brickwork_state(n, 4, 900 + s).astype(np.complex64) for n, s in spec]
    ts = [dev(torch, v) for v in states]
    with sre.Plan(16, "c64") as p:
        out = p.m2_batched(ts)
        torch.cuda.synchronize()
        singles = [p.m2(t) for t in ts]
    got = out.cpu().numpy()
    for v, g, s in zip(states, got, singles):
        assert abs(g - oracle.m2(v)) <= TOL["fp32"]
        assert abs(g - s) <= 1e-12
