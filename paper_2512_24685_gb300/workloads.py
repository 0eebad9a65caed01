"""Seeded synthetic input states for the M2 path (no M2 arithmetic here).

These generators are the only code shared between the CUDA path's tests and
benchmark and the FP64 oracle: they make state vectors, nothing else.  Every
generator takes an integer seed and draws from numpy's PCG64, so the same
(seed, N) gives the same amplitudes on every machine.

Bit order: qubit j <-> bit j of the basis index t, as in the library.

State families (the paper's workloads):

* ``haar_state``     -- Haar-random pure state: re, im i.i.d. N(0, 1), then
  l2-normalised in FP64 (the benchmark states of the XOR-FWHT section).
* ``product_state``  -- tensor product of single-qubit states
  cos(theta/2)|0> + e^{i phi} sin(theta/2)|1> with Bloch vectors uniform on the
  sphere (cos theta ~ U[-1, 1], phi ~ U[0, 2pi)): the random initial states of
  Example 1 (TFIM quench), Eq. (random_product_state).
* ``stabilizer_state`` -- |0^N> through ``depth`` layers of random single-qubit
  Cliffords (words in H and S) followed by CNOTs on even / odd bonds.
* ``brickwork_state`` -- |0^N> through ``depth`` brickwork steps of Haar-random
  two-qubit gates, even bonds then odd bonds, open boundary: Example 2.
"""
from __future__ import annotations

import numpy as np

_SQ2 = 1.0 / np.sqrt(2.0)
_H = np.array([[_SQ2, _SQ2], [_SQ2, -_SQ2]], dtype=np.complex128)
_S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)
# a few single-qubit Cliffords as words in H and S
_CLIFF1 = [_I2, _H, _S, _H @ _S, _S @ _H, _H @ _S @ _H, _S @ _S, _H @ _S @ _S @ _H]
_CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]],
                 dtype=np.complex128)  # basis index 2*b1 + b0, control b0, target b1


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def config_seed(config_index: int, state_index: int) -> int:
    """Seed convention for workload configurations: 1000*config + state."""
    return 1000 * int(config_index) + int(state_index)


def _cast(psi: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(psi.astype(dtype, copy=False))


def haar_state(N: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Haar-random N-qubit state: complex Gaussian amplitudes, unit l2 in FP64."""
    rng = rng_for(seed)
    d = 1 << N
    re = rng.standard_normal(d)
    im = rng.standard_normal(d)
    psi = re + 1j * im
    psi /= np.sqrt(np.sum(re * re + im * im))
    return _cast(psi, dtype)


def random_bloch(N: int, seed: int) -> np.ndarray:
    """(N, 3) Bloch vectors uniform on the unit sphere."""
    rng = rng_for(seed)
    cos_t = rng.uniform(-1.0, 1.0, N)
    phi = rng.uniform(0.0, 2.0 * np.pi, N)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def qubit_from_bloch(v) -> np.ndarray:
    """cos(theta/2)|0> + e^{i phi} sin(theta/2)|1> for Bloch vector v."""
    x, y, z = (float(c) for c in v)
    theta = np.arccos(np.clip(z, -1.0, 1.0))
    phi = np.arctan2(y, x)
    return np.array([np.cos(theta / 2), np.exp(1j * phi) * np.sin(theta / 2)],
                    dtype=np.complex128)


def product_of(qubits) -> np.ndarray:
    """Tensor product with qubits[j] on bit j of the index."""
    psi = np.ones(1, dtype=np.complex128)
    for q in qubits:
        psi = np.kron(np.asarray(q, dtype=np.complex128), psi)
    return psi


def product_state(N: int, seed: int, dtype=np.complex128):
    """(psi, bloch): random product state and its (N, 3) Bloch vectors."""
    bloch = random_bloch(N, seed)
    psi = product_of([qubit_from_bloch(v) for v in bloch])
    return _cast(psi, dtype), bloch


def apply_1q(psi: np.ndarray, N: int, q: int, U: np.ndarray) -> np.ndarray:
    v = psi.reshape(1 << (N - q - 1), 2, 1 << q)
    return np.einsum("ab,ibj->iaj", U, v).reshape(-1)


def apply_2q(psi: np.ndarray, N: int, q: int, U: np.ndarray) -> np.ndarray:
    """Gate U (4x4, index 2*b_{q+1} + b_q) on neighbouring qubits q, q+1."""
    v = psi.reshape(1 << (N - q - 2), 4, 1 << q)
    return np.einsum("ab,ibj->iaj", U, v).reshape(-1)


def basis_state(N: int, t: int = 0) -> np.ndarray:
    psi = np.zeros(1 << N, dtype=np.complex128)
    psi[t] = 1.0
    return psi


def stabilizer_state(N: int, seed: int, depth: int | None = None,
                     dtype=np.complex128) -> np.ndarray:
    """|0^N> through `depth` (default 2N) layers: a random single-qubit
    Clifford on every qubit, then CNOTs on even bonds (even layers) or odd
    bonds (odd layers)."""
    rng = rng_for(seed)
    depth = 2 * N if depth is None else depth
    psi = basis_state(N)
    for layer in range(depth):
        for q in range(N):
            psi = apply_1q(psi, N, q, _CLIFF1[rng.integers(len(_CLIFF1))])
        for q in range(layer % 2, N - 1, 2):
            psi = apply_2q(psi, N, q, _CNOT)
    return _cast(psi, dtype)


def haar_unitary(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random U(n): QR of a complex Gaussian matrix with the phases of
    R's diagonal moved into Q (Mezzadri's construction)."""
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    diag = np.diagonal(r)
    return q * (diag / np.abs(diag))[None, :]


def brickwork_gates(N: int, depth: int, seed: int) -> list[tuple[int, np.ndarray]]:
    """The (qubit, 4x4 gate) list of a `depth`-step brickwork: per step, Haar
    gates on bonds (0,1),(2,3),... then (1,2),(3,4),... (open chain)."""
    rng = rng_for(seed)
    gates = []
    for _ in range(depth):
        for start in (0, 1):
            for q in range(start, N - 1, 2):
                gates.append((q, haar_unitary(4, rng)))
    return gates


def brickwork_state(N: int, depth: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Example 2's circuit state: |0^N> after `depth` brickwork steps."""
    psi = basis_state(N)
    for q, U in brickwork_gates(N, depth, seed):
        psi = apply_2q(psi, N, q, U)
    return _cast(psi, dtype)


def brickwork_state_torch(N: int, depth: int, seed: int, device, dtype=None):
    """brickwork_state on a torch device (same gates, complex128 arithmetic),
    for large synthetic batches; agrees with the numpy version to rounding."""
    import torch
    psi = torch.zeros(1 << N, dtype=torch.complex128, device=device)
    psi[0] = 1.0
    for q, U in brickwork_gates(N, depth, seed):
        Ut = torch.as_tensor(U, dtype=torch.complex128, device=device)
        v = psi.reshape(1 << (N - q - 2), 4, 1 << q)
        psi = torch.einsum("ab,ibj->iaj", Ut, v).reshape(-1)
    return psi if dtype is None else psi.to(dtype)


def stabilizer_state_torch(N: int, seed: int, device, depth: int | None = None, dtype=None):
    """stabilizer_state on a torch device (same gate sequence, complex128)."""
    import torch
    rng = rng_for(seed)
    depth = 2 * N if depth is None else depth
    psi = torch.zeros(1 << N, dtype=torch.complex128, device=device)
    psi[0] = 1.0
    cl = [torch.as_tensor(g, dtype=torch.complex128, device=device) for g in _CLIFF1]
    cnot = torch.as_tensor(_CNOT, dtype=torch.complex128, device=device)
    for layer in range(depth):
        for q in range(N):
            U = cl[rng.integers(len(_CLIFF1))]
            v = psi.reshape(1 << (N - q - 1), 2, 1 << q)
            psi = torch.einsum("ab,ibj->iaj", U, v).reshape(-1)
        for q in range(layer % 2, N - 1, 2):
            v = psi.reshape(1 << (N - q - 2), 4, 1 << q)
            psi = torch.einsum("ab,ibj->iaj", cnot, v).reshape(-1)
    return psi if dtype is None else psi.to(dtype)


def serving_n_distribution(n_lo: int = 10, n_hi: int = 20):
    """P(N) proportional to 2^{-(N - n_lo)/2} on {n_lo..n_hi} (the serving mix)."""
    ns = np.arange(n_lo, n_hi + 1)
    w = 2.0 ** (-(ns - n_lo) / 2.0)
    return ns, w / w.sum()


def mixed_n16_batch(config_index: int = 1, N: int = 16, per_kind: int = 16,
                    depth: int = 8, dtype=np.complex64):
    """The four-family N=16 batch: `per_kind` each of Haar, product (with
    Bloch vectors), stabilizer and depth-`depth` brickwork states.
    Returns a list of (kind, psi, extra) with extra = Bloch vectors or None."""
    out = []
    j = 0
    for _ in range(per_kind):
        out.append(("haar", haar_state(N, config_seed(config_index, j), dtype), None)); j += 1
    for _ in range(per_kind):
        psi, bloch = product_state(N, config_seed(config_index, j), dtype)
        out.append(("product", psi, bloch)); j += 1
    for _ in range(per_kind):
        out.append(("stabilizer", stabilizer_state(N, config_seed(config_index, j), dtype=dtype), None)); j += 1
    for _ in range(per_kind):
        out.append(("brickwork", brickwork_state(N, depth, config_seed(config_index, j), dtype), None)); j += 1
    return out


def uneven_batch_spec(count: int = 512, n_lo: int = 12, n_hi: int = 18,
                      depth_hi: int = 32, config_index: int = 3, seed: int = 3):
    """(N_i, depth_i, seed_i) for the uneven batched workload: N ~ U{n_lo..n_hi},
    depth ~ U{1..depth_hi}, brickwork Haar circuits on |0^N>."""
    rng = rng_for(config_seed(config_index, 999_000 + seed))
    Ns = rng.integers(n_lo, n_hi + 1, size=count)
    depths = rng.integers(1, depth_hi + 1, size=count)
    return [(int(n), int(t), config_seed(config_index, i)) for i, (n, t) in enumerate(zip(Ns, depths))]


def brickwork_gate_tensor(N: int, S: int, T: int, config_index: int = 4) -> np.ndarray:
    """Gates of S brickwork realizations over T steps, (T, S, N-1, 4, 4)
    complex128, in the order applied (per step: even bonds, then odd bonds);
    realization s draws brickwork_gates(N, T, config_seed(config_index, s)),
    so the same gates drive brickwork_state."""
    out = np.empty((T, S, N - 1, 4, 4), dtype=np.complex128)
    for s in range(S):
        gates = brickwork_gates(N, T, config_seed(config_index, s))
        for t in range(T):
            for b in range(N - 1):
                out[t, s, b] = gates[t * (N - 1) + b][1]
    return out
