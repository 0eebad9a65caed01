"""Writes tests/golden/closed_forms.txt: M2 values fixed by closed forms.

Nothing here runs the oracle or the CUDA path; every value follows from the
paper's properties of M2 and the single-qubit Pauli sum:

* single qubit with Bloch vector (a, b, c): the Pauli expectations are
  1, a, b, c, so S = 1 + a^4 + b^4 + c^4 and M2 = -log2(S / 2)
  (Eq. (sre) at alpha = 2 with d = 2);
* additivity under tensor products (property (iii) after Eq. (sre)) gives
  M2 of a product state as the sum over its qubits;
* faithfulness (property (i)): stabilizer states have M2 = 0;
* Haar-random states: annealed mean log2(2^N + 3) - 2 (Fig. 1(b) caption),
  i.e. E[2^{-M2}] = 4 / (2^N + 3).

Run:  python tests/golden/make_closed_forms.py
"""
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def single(a, b, c):
    return -math.log2((1 + a ** 4 + b ** 4 + c ** 4) / 2)


rows = []
s = 1 / math.sqrt(2)
f = 1 / math.sqrt(3)
rows.append(("zero", 1, single(0, 0, 1), "faithfulness: |0> is a stabilizer state"))
rows.append(("plus", 1, single(1, 0, 0), "faithfulness: |+> is a stabilizer state"))
rows.append(("T", 1, single(s, s, 0), "|T> = (|0> + e^{i pi/4}|1>)/sqrt2, Bloch (1/sqrt2, 1/sqrt2, 0)"))
rows.append(("F", 1, single(f, f, f), "facet state, Bloch (1,1,1)/sqrt3"))
for n in (2, 3, 4, 5, 6, 8, 10):
    rows.append((f"T^{n}", n, n * single(s, s, 0), "additivity: N log2(4/3)"))
for n in (2, 4, 7):
    rows.append((f"plus^{n}", n, 0.0, "additivity + faithfulness"))
for n in (2, 3, 5):
    rows.append((f"F^{n}", n, n * single(f, f, f), "additivity: N log2(3/2)"))
for n in range(1, 21):
    rows.append((f"haar_mean_{n}", n, math.log2(2 ** n + 3) - 2,
                 "annealed Haar mean, Fig. 1(b) caption"))

with open(os.path.join(HERE, "closed_forms.txt"), "w") as fh:
    fh.write("# name  N  M2  -- source (see make_closed_forms.py)\n")
    for name, n, val, why in rows:
        fh.write(f"{name} {n} {val!r} -- {why}\n")
print(f"wrote {len(rows)} rows")
