"""Pins for the FP64 oracle, against things other than itself.

* explicit Pauli matrices (Kronecker products of I, X, Y, Z) -- the
  definition in Eq. (sre) before the binary encoding;
* scipy's Sylvester Hadamard matrix for the FWHT (supplement, FWHT section);
* closed forms (tests/golden/closed_forms.txt) from single-qubit sums,
  additivity and faithfulness (properties after Eq. (sre));
* invariants: Parseval/purity, bounds, Clifford invariance, the real /
  imaginary pattern of X^x Z^z expectations, the Haar mean of Fig. 1(b).
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg

from paper_2512_24685_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))

PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PI = np.eye(2, dtype=np.complex128)


def kron_list(mats):
    """Kronecker product with mats[j] acting on qubit j (bit j of the index):
    the first factor of np.kron is the most significant bit."""
    out = np.ones((1, 1), dtype=np.complex128)
    for m in mats:
        out = np.kron(m, out)
    return out


def rand_state(N, seed, normalise=True):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << N) + 1j * rng.standard_normal(1 << N)
    return v / np.linalg.norm(v) if normalise else v


def load_golden():
    rows = {}
    with open(os.path.join(HERE, "golden", "closed_forms.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, n, val = line.split("--")[0].split()
            rows[name] = (int(n), float(val))
    return rows


# ---------------------------------------------------------------- definition

@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_table_matches_explicit_pauli_matrices(oracle_mod, N):
    """Every entry <psi|X^x Z^z|psi> of the direct table equals psi^H P psi with
    P = tensor_j X^{x_j} Z^{z_j} built from 2x2 matrices (Eq. (Pauli_expect))."""
    psi = rand_state(N, 11 + N, normalise=False)
    table = oracle_mod.pauli_table(psi)
    d = 1 << N
    for x in range(d):
        for z in range(d):
            mats = []
            for j in range(N):
                m = PI
                if (x >> j) & 1:
                    m = m @ PX
                if (z >> j) & 1:
                    m = m @ PZ
                mats.append(m)
            P = kron_list(mats)
            ref = np.vdot(psi, P @ psi)
            assert abs(table[x, z] - ref) < 1e-13 * max(1.0, abs(ref)), (x, z)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_sum4_matches_hermitian_pauli_group(oracle_mod, N):
    """S over the Hermitian Pauli strings {I,X,Y,Z}^N (Eq. (sre)) equals the
    oracle's S over X^x Z^z (phases dropped), by both O1 and O2."""
    psi = rand_state(N, 100 + N, normalise=False)
    S_ref = 0.0
    for word in itertools.product([PI, PX, PY, PZ], repeat=N):
        e = np.vdot(psi, kron_list(word) @ psi)
        S_ref += abs(e) ** 4
    assert oracle_mod.sum4_direct(psi) == pytest.approx(S_ref, rel=1e-12)
    assert oracle_mod.sum4_xorfwht(psi) == pytest.approx(S_ref, rel=1e-12)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8])
def test_direct_equals_xorfwht(oracle_mod, N):
    """O1 (definition) == O2 (Algorithm 1) on random, unnormalised and
    complex64-rounded states, per shift and in total."""
    for seed, norm, c64 in [(1, True, False), (2, False, False), (3, True, True)]:
        psi = rand_state(N, 1000 * N + seed, normalise=norm)
        if c64:
            psi = psi.astype(np.complex64)
        s1, p1 = oracle_mod.sum4_direct(psi, per_x=True)
        s2, p2 = oracle_mod.sum4_xorfwht(psi, per_x=True)
        assert s2 == pytest.approx(s1, rel=1e-12)
        np.testing.assert_allclose(p2, p1, rtol=1e-11, atol=1e-15 * s1)
        assert oracle_mod.m2(psi, "direct") == pytest.approx(oracle_mod.m2(psi, "xorfwht"), abs=1e-12)


def test_xorfwht_range_partition(oracle_mod):
    """Sum over shift ranges adds up to the full sum (independence over k)."""
    psi = rand_state(7, 5)
    full = oracle_mod.sum4_xorfwht(psi)
    parts = sum(oracle_mod.sum4_xorfwht(psi, a, a + 32) for a in range(0, 128, 32))
    assert parts == pytest.approx(full, rel=1e-14)


# --------------------------------------------------------------------- FWHT

@pytest.mark.parametrize("N", [1, 2, 5, 9])
def test_fwht_is_sylvester_hadamard(oracle_mod, N):
    """FWHT(v) = H v with H = H_2^{tensor N} (scipy's Sylvester matrix)."""
    v = rand_state(N, 7 + N, normalise=False)
    H = scipy.linalg.hadamard(1 << N).astype(np.float64)
    np.testing.assert_allclose(oracle_mod.fwht(v), H @ v, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("N", [3, 10])
def test_fwht_involution_and_parseval(oracle_mod, N):
    """FWHT(FWHT(v)) = d v (involution of the normalised WHT) and
    sum |FWHT v|^2 = d sum |v|^2 (Parseval)."""
    v = rand_state(N, 3, normalise=False)
    d = 1 << N
    w = oracle_mod.fwht(v)
    np.testing.assert_allclose(oracle_mod.fwht(w), d * v, rtol=1e-12, atol=1e-12)
    assert np.sum(np.abs(w) ** 2) == pytest.approx(d * np.sum(np.abs(v) ** 2), rel=1e-12)
    np.testing.assert_allclose(oracle_mod.fwht(np.conj(v)), np.conj(w), rtol=1e-13, atol=1e-13)


def test_shift_transform_is_table_row(oracle_mod):
    """One iteration of Algorithm 1 reproduces row x of the Pauli table."""
    N = 5
    psi = rand_state(N, 9, normalise=False)
    table = oracle_mod.pauli_table(psi)
    for x in (0, 1, 6, 31):
        np.testing.assert_allclose(oracle_mod.shift_transform(psi, x), table[x], rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------- closed forms

def test_golden_closed_forms(oracle_mod):
    g = load_golden()
    s = 1 / math.sqrt(2)
    f = 1 / math.sqrt(3)
    states = {
        "zero": W.basis_state(1),
        "plus": np.array([s, s], dtype=np.complex128),
        "T": W.qubit_from_bloch((s, s, 0)),
        "F": W.qubit_from_bloch((f, f, f)),
    }
    for n in (2, 3, 4, 5, 6, 8, 10):
        states[f"T^{n}"] = W.product_of([states["T"]] * n)
    for n in (2, 4, 7):
        states[f"plus^{n}"] = W.product_of([states["plus"]] * n)
    for n in (2, 3, 5):
        states[f"F^{n}"] = W.product_of([states["F"]] * n)
    for name, psi in states.items():
        n, expect = g[name]
        assert psi.size == 1 << n
        for method in (["direct", "xorfwht"] if n <= 8 else ["xorfwht"]):
            assert oracle_mod.m2(psi, method) == pytest.approx(expect, abs=1e-12), (name, method)


@pytest.mark.parametrize("N", [1, 3, 6, 9])
def test_random_product_states_closed_form(oracle_mod, N):
    """M2 = -sum_q log2((1 + x_q^4 + y_q^4 + z_q^4) / 2) (additivity)."""
    for seed in range(3):
        psi, bloch = W.product_state(N, 500 + seed)
        expect = -np.sum(np.log2((1 + np.sum(bloch ** 4, axis=1)) / 2))
        assert oracle_mod.m2(psi) == pytest.approx(expect, abs=1e-12)


@pytest.mark.parametrize("N", [1, 2, 4, 7, 9])
def test_stabilizer_states_have_zero_magic(oracle_mod, N):
    """Faithfulness: random Clifford-circuit states have M2 = 0; computational
    basis states give S = d exactly."""
    for seed in range(3):
        psi = W.stabilizer_state(N, 40 + seed)
        assert abs(oracle_mod.m2(psi)) < 1e-12
    for t in (0, (1 << N) - 1):
        assert oracle_mod.sum4_xorfwht(W.basis_state(N, t)) == float(1 << N)


# --------------------------------------------------------------- invariants

@pytest.mark.parametrize("N", [2, 5, 6])
def test_purity_parseval(oracle_mod, N):
    """sum_{x,z} |A|^2 = d n2^2, and per x sum_z |A_x(z)|^2 =
    d sum_t |psi_{t^x}|^2 |psi_t|^2 (Parseval applied to the shifted product)."""
    psi = rand_state(N, 77, normalise=False)
    d = 1 << N
    table = oracle_mod.pauli_table(psi)
    p = np.abs(psi) ** 2
    n2 = p.sum()
    assert np.sum(np.abs(table) ** 2) == pytest.approx(d * n2 ** 2, rel=1e-12)
    for x in range(d):
        t = np.arange(d)
        assert np.sum(np.abs(table[x]) ** 2) == pytest.approx(d * np.sum(p[t ^ x] * p), rel=1e-12)


@pytest.mark.parametrize("N", [1, 3, 6, 8])
def test_bounds(oracle_mod, N):
    for seed in range(4):
        m = oracle_mod.m2(rand_state(N, seed))
        assert -1e-12 <= m <= math.log2(((1 << N) + 1) / 2) + 1e-12


def test_real_imaginary_pattern(oracle_mod):
    """<psi|X^x Z^z|psi> is real when popc(x&z) is even and imaginary when odd
    (X^x Z^z is Hermitian up to i^{popc(x&z)})."""
    N = 5
    psi = rand_state(N, 21)
    table = oracle_mod.pauli_table(psi)
    d = 1 << N
    for x in range(d):
        for z in range(d):
            a = table[x, z]
            if bin(x & z).count("1") % 2 == 0:
                assert abs(a.imag) < 1e-14
            else:
                assert abs(a.real) < 1e-14


def _permute_qubits(psi, N, perm):
    t = np.arange(1 << N)
    src = np.zeros_like(t)
    for j in range(N):
        src |= ((t >> perm[j]) & 1) << j
    return psi[src]


@pytest.mark.parametrize("N", [4, 7])
def test_clifford_invariance(oracle_mod, N):
    """M2 is unchanged by qubit permutations, global phase, complex
    conjugation, layers of single-qubit Cliffords and CNOT layers."""
    rng = np.random.default_rng(N)
    psi = rand_state(N, 300 + N)
    m = oracle_mod.m2(psi)
    variants = [
        _permute_qubits(psi, N, rng.permutation(N)),
        psi * np.exp(0.7j),
        np.conj(psi),
    ]
    phi = psi.copy()
    for q in range(N):
        phi = W.apply_1q(phi, N, q, W._CLIFF1[rng.integers(len(W._CLIFF1))])
    variants.append(phi)
    phi = psi.copy()
    for q in range(0, N - 1, 2):
        phi = W.apply_2q(phi, N, q, W._CNOT)
    variants.append(phi)
    for v in variants:
        assert oracle_mod.m2(v) == pytest.approx(m, abs=1e-12)


def test_additivity(oracle_mod):
    a = rand_state(3, 1)
    b = rand_state(4, 2)
    ab = np.kron(b, a)  # a on the low 3 bits, b on the high 4
    assert oracle_mod.m2(ab) == pytest.approx(oracle_mod.m2(a) + oracle_mod.m2(b), abs=1e-12)


def test_non_clifford_gate_changes_magic(oracle_mod):
    """Sensitivity: a T gate on a |+> qubit adds log2(4/3)."""
    s = 1 / math.sqrt(2)
    plus = np.array([s, s], dtype=np.complex128)
    T = np.diag([1, np.exp(1j * np.pi / 4)])
    assert oracle_mod.m2(T @ plus) == pytest.approx(math.log2(4 / 3), abs=1e-14)


@pytest.mark.parametrize("N", [4, 6])
def test_haar_mean(oracle_mod, N):
    """Fig. 1(b): E[S/d] = E[2^{-M2}] = 4/(d+3) for Haar states (the annealed
    mean), checked within 4 standard errors over 96 states."""
    vals = np.array([2.0 ** (-oracle_mod.m2(W.haar_state(N, 7000 + i))) for i in range(96)])
    d = 1 << N
    sem = vals.std(ddof=1) / math.sqrt(vals.size)
    assert abs(vals.mean() - 4 / (d + 3)) < 4 * sem


def _explicit_pauli(N, x, z):
    mats = []
    for j in range(N):
        m = PI
        if (x >> j) & 1:
            m = m @ PX
        if (z >> j) & 1:
            m = m @ PZ
        mats.append(m)
    return kron_list(mats)


def test_planted_mistakes_are_caught(oracle_mod):
    """Sensitivity of the pins: plausible slips in the product of Algorithm 1
    (conjugate dropped; the shift taken as t + x mod d instead of t XOR x;
    Z signs ignored) each move the per-shift sums sum_z |A_x(z)|^4 away from
    the explicit-Pauli-matrix values, shown with a tiny Python restatement of
    the loop.  (Dropping the conjugate leaves the *total* S unchanged -- it
    re-labels the correlation C_x(s) of the supplement's derivation as
    C_s(x XOR s) -- which is why the per-shift sums and the per-entry table
    are pinned, not only S.)"""
    N = 3
    d = 1 << N
    psi = rand_state(N, 4242)
    expect = np.array([sum(abs(np.vdot(psi, _explicit_pauli(N, x, z) @ psi)) ** 4
                           for z in range(d)) for x in range(d)])
    H = scipy.linalg.hadamard(d)
    t = np.arange(d)

    def per_x(prod, signs=True):
        out = []
        for x in range(d):
            g = prod(x)
            A = H @ g if signs else np.full(d, g.sum())
            out.append(np.sum(np.abs(A) ** 4))
        return np.array(out)

    np.testing.assert_allclose(per_x(lambda x: np.conj(psi[t ^ x]) * psi[t]), expect, rtol=1e-12)
    np.testing.assert_allclose(oracle_mod.sum4_xorfwht(psi, per_x=True)[1], expect, rtol=1e-12)
    for slip in (per_x(lambda x: psi[t ^ x] * psi[t]),
                 per_x(lambda x: np.conj(psi[(t + x) % d]) * psi[t]),
                 per_x(lambda x: np.conj(psi[t ^ x]) * psi[t], signs=False)):
        assert np.max(np.abs(slip - expect)) > 1e-3 * expect.max()


# ------------------------------------- general integer Renyi order (Eq. (sre))

ALPHAS = (2, 3, 4, 6)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_sum_pow_matches_hermitian_pauli_group(oracle_mod, N):
    """S_alpha = sum over the Hermitian Pauli strings {I,X,Y,Z}^N of
    |psi^H P psi|^(2 alpha), P from explicit 2x2 matrices (Eq. (sre)), equals
    the oracle's S_alpha by O1 and O2 for every order tested."""
    psi = rand_state(N, 700 + N, normalise=False)
    vals = [abs(np.vdot(psi, kron_list(w) @ psi)) for w in itertools.product([PI, PX, PY, PZ], repeat=N)]
    for a in ALPHAS:
        ref = sum(v ** (2 * a) for v in vals)
        assert oracle_mod.sum_pow_direct(psi, a) == pytest.approx(ref, rel=1e-12), a
        assert oracle_mod.sum_pow_xorfwht(psi, a) == pytest.approx(ref, rel=1e-12), a


@pytest.mark.parametrize("N", [3, 6, 8])
def test_sum_pow_direct_equals_xorfwht(oracle_mod, N):
    """O1 == O2 per shift for orders 3, 4, 6; at order 2 both equal the
    M2 routines exactly (same arithmetic)."""
    psi = rand_state(N, 800 + N, normalise=False)
    for a in (3, 4, 6):
        s1, p1 = oracle_mod.sum_pow_direct(psi, a, per_x=True)
        s2, p2 = oracle_mod.sum_pow_xorfwht(psi, a, per_x=True)
        assert np.allclose(p1, p2, rtol=1e-11, atol=0), a
        assert s1 == pytest.approx(s2, rel=1e-12)
    assert oracle_mod.sum_pow_direct(psi, 2) == oracle_mod.sum4_direct(psi)
    assert oracle_mod.sum_pow_xorfwht(psi, 2) == oracle_mod.sum4_xorfwht(psi)
    assert oracle_mod.malpha(psi, 2) == pytest.approx(oracle_mod.m2(psi), abs=1e-13)


@pytest.mark.parametrize("N", [1, 3, 6, 9])
def test_malpha_product_states_closed_form(oracle_mod, N):
    """Random product states: M_alpha = sum_q log2((1 + x_q^(2a) + y_q^(2a) +
    z_q^(2a)) / 2) / (1 - a) (single-qubit Paulis I, X, Y, Z have
    expectations 1, x, y, z; additivity)."""
    for seed in range(2):
        psi, bloch = W.product_state(N, 900 + seed)
        for a in ALPHAS:
            expect = np.sum(np.log2((1 + np.sum(bloch ** (2 * a), axis=1)) / 2)) / (1 - a)
            assert oracle_mod.malpha(psi, a) == pytest.approx(expect, abs=1e-12), a


def test_malpha_t_state(oracle_mod):
    """T|+> has Bloch vector (1/sqrt 2, 1/sqrt 2, 0): M_alpha =
    log2((1 + 2^(1-a)) / 2) / (1 - a); 3 copies give three times that."""
    s = 1 / math.sqrt(2)
    t1 = np.diag([1, np.exp(1j * np.pi / 4)]) @ np.array([s, s], dtype=np.complex128)
    t3 = np.kron(t1, np.kron(t1, t1))
    for a in ALPHAS:
        one = math.log2((1 + 2.0 ** (1 - a)) / 2) / (1 - a)
        assert oracle_mod.malpha(t1, a) == pytest.approx(one, abs=1e-14), a
        assert oracle_mod.malpha(t3, a) == pytest.approx(3 * one, abs=1e-12), a


@pytest.mark.parametrize("N", [2, 5, 8])
def test_malpha_stabilizer_zero_and_order_monotone(oracle_mod, N):
    """Faithfulness at every order (stabilizer states: d Pauli expectations
    of modulus 1, the rest 0, so S_alpha = d); for a generic state M_alpha
    does not increase with alpha (a Renyi entropy of the distribution
    <P>^2 / d, shifted by log2 d)."""
    for seed in range(2):
        stab = W.stabilizer_state(N, 60 + seed)
        for a in ALPHAS:
            assert abs(oracle_mod.malpha(stab, a)) < 1e-12
    psi = rand_state(N, 950 + N)
    m = [oracle_mod.malpha(psi, a) for a in (2, 3, 4, 5, 6)]
    assert all(m[i] >= m[i + 1] - 1e-12 for i in range(len(m) - 1)), m


def test_malpha_invariances(oracle_mod):
    """Clifford invariance, unnormalised input and additivity at order 3."""
    rng = np.random.default_rng(5)
    psi = rand_state(5, 17)
    m = oracle_mod.malpha(psi, 3)
    phi = psi.copy()
    for q in range(5):
        phi = W.apply_1q(phi, 5, q, W._CLIFF1[rng.integers(len(W._CLIFF1))])
    for q in range(0, 4, 2):
        phi = W.apply_2q(phi, 5, q, W._CNOT)
    assert oracle_mod.malpha(phi, 3) == pytest.approx(m, abs=1e-12)
    assert oracle_mod.malpha(3.7 * psi, 3) == pytest.approx(m, abs=1e-12)
    a, b = rand_state(2, 21), rand_state(3, 22)
    assert oracle_mod.malpha(np.kron(b, a), 3) == pytest.approx(
        oracle_mod.malpha(a, 3) + oracle_mod.malpha(b, 3), abs=1e-12)


def test_malpha_planted_exponent_slip_is_caught(oracle_mod):
    """A plausible slip -- using |A|^alpha instead of |A|^(2 alpha) -- is
    caught by the product-state closed form at order 3."""
    psi, bloch = W.product_state(4, 77)
    expect = np.sum(np.log2((1 + np.sum(bloch ** 6, axis=1)) / 2)) / (1 - 3)
    n2 = oracle_mod.norm2(psi)
    table = oracle_mod.pauli_table(psi)
    wrong = np.sum(np.abs(table) ** 3)
    wrong_m = oracle_mod.malpha_from_sum(wrong, n2, 4, 3)
    assert abs(wrong_m - expect) > 1e-3
    right = np.sum(np.abs(table) ** 6)
    assert oracle_mod.malpha_from_sum(right, n2, 4, 3) == pytest.approx(expect, abs=1e-12)


# ------------------------------------- TFIM quench reference (Example 1)

def test_tfim_hamiltonian_matches_kronecker_terms(oracle_mod):
    """H of Eq. (TFIM_LF_OBC) built term by term from 2x2 matrices (open
    chain: bonds (i, i+1), i = 0..N-2) equals the oracle's sparse H."""
    N, J, hx, hz = 4, 1.0, 1.5, 1.5
    H = np.zeros((1 << N, 1 << N), dtype=np.complex128)
    for i in range(N - 1):
        H -= J * kron_list([PZ if j in (i, i + 1) else PI for j in range(N)])
    for i in range(N):
        H -= hx * kron_list([PX if j == i else PI for j in range(N)])
        H -= hz * kron_list([PZ if j == i else PI for j in range(N)])
    assert np.allclose(oracle_mod.tfim_hamiltonian(N, J, hx, hz).toarray(), H, atol=1e-14)


def test_tfim_single_qubit_closed_form(oracle_mod):
    """N = 1: H = -hx X - hz Z, so exp(-iHt) = cos(wt) I - i sin(wt) H / w with
    w = sqrt(hx^2 + hz^2)."""
    hx, hz, dt = 1.5, 1.5, 0.2
    psi = np.array([0.6, 0.8j])
    w = math.hypot(hx, hz)
    H = -hx * PX - hz * PZ
    states = oracle_mod.tfim_evolve(psi, dt, 3, 1.0, hx, hz)
    for k, st in enumerate(states, start=1):
        U = math.cos(w * k * dt) * PI - 1j * math.sin(w * k * dt) * H / w
        assert np.allclose(st, U @ psi, atol=1e-13)


def test_tfim_evolution_dense_and_conservation(oracle_mod):
    """N = 5: equals the dense matrix exponential; norm and energy conserved."""
    psi, _ = W.product_state(5, 12)
    H = oracle_mod.tfim_hamiltonian(5)
    states = oracle_mod.tfim_evolve(psi, 0.2, 4)
    U = scipy.linalg.expm(-1j * 0.2 * H.toarray())
    ref = psi.copy()
    e0 = np.vdot(psi, H @ psi).real
    for st in states:
        ref = U @ ref
        assert np.allclose(st, ref, atol=1e-12)
        assert abs(np.linalg.norm(st) - 1) < 1e-12
        assert abs(np.vdot(st, H @ st).real - e0) < 1e-10
