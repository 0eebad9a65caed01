"""CPU tests of host-side helpers: the brickwork gate tensor that drives
sre_brickwork_m2_series, and the benchmark's roofline traffic bookkeeping."""
import numpy as np

from paper_2512_24685_gb300 import workloads as W


def test_brickwork_gate_tensor_matches_gate_list():
    """Realization s, step t, bond index b of the tensor is the gate that
    brickwork_gates(N, T, seed_s) applies there (even bonds, then odd)."""
    N, S, T = 7, 3, 4
    g = W.brickwork_gate_tensor(N, S, T)
    assert g.shape == (T, S, N - 1, 4, 4) and g.dtype == np.complex128
    for s in range(S):
        ref = W.brickwork_gates(N, T, W.config_seed(4, s))
        assert len(ref) == T * (N - 1)
        for t in range(T):
            for b in range(N - 1):
                q, U = ref[t * (N - 1) + b]
                expect_q = 2 * b if b < N // 2 else 2 * (b - N // 2) + 1
                assert q == expect_q
                assert np.array_equal(g[t, s, b], U)
    # every gate is unitary
    flat = g.reshape(-1, 4, 4)
    eye = np.eye(4)
    assert max(np.max(np.abs(u.conj().T @ u - eye)) for u in flat) < 1e-12


def test_brickwork_gate_tensor_reproduces_brickwork_state():
    """Applying the tensor's gates in order with apply_2q gives brickwork_state."""
    N, T = 6, 3
    g = W.brickwork_gate_tensor(N, 1, T)
    psi = W.basis_state(N)
    for t in range(T):
        for b in range(N - 1):
            q = 2 * b if b < N // 2 else 2 * (b - N // 2) + 1
            psi = W.apply_2q(psi, N, q, g[t, 0, b])
    assert np.max(np.abs(psi - W.brickwork_state(N, T, W.config_seed(4, 0)))) < 1e-12


def test_bench_traffic_only_for_profiled_configuration():
    """roofline.traffic is reported only for a (mode, tuning) pair that an
    ncu capture measured, scaled from the slice to the halved launch."""
    import bench
    keys = ("x_batch_log", "ring_slots", "lag", "pass2_tiles_log", "pass1_blocks_log")
    for (mode, tup), slice_bytes in bench.TRAFFIC.items():
        tun = dict(zip(keys, tup))
        full = bench.profiled_traffic(20, mode, tun)
        assert full == slice_bytes * ((1 << 20) - 4096) / bench.TRAFFIC_SLICE_SHIFTS
        assert bench.profiled_traffic(19, mode, tun) is None
        assert bench.profiled_traffic(20, "fp64", tun) is None
        tun["ring_slots"] += 1
        assert bench.profiled_traffic(20, mode, tun) is None
