"""Seeded test inputs shared by the test modules."""
import numpy as np

from paper_2605_15098_gb300 import circuits as C


def mixed_circuit(n, m, seed, kinds=tuple(range(11))):
    """Random circuit over every gate kind (test input)."""
    rng = np.random.default_rng(seed)
    recs = []
    for _ in range(m):
        kind = int(kinds[int(rng.integers(0, len(kinds)))])
        t = int(rng.integers(0, n))
        o = int(rng.integers(0, n - 1)) if n > 1 else 0
        o = o + 1 if o >= t else o
        if n == 1 and kind in (C.CP, C.CZ, C.SWAP, C.CU, C.CPK):
            kind = C.U3
        if kind == C.X:
            recs.append(C.x(t))
        elif kind == C.H:
            recs.append(C.h(t))
        elif kind == C.P:
            recs.append(C.p(t, float(rng.uniform(-7, 7))))
        elif kind == C.CP:
            recs.append(C.cp(o, t, float(rng.uniform(-7, 7))))
        elif kind == C.CZ:
            recs.append(C.cz(o, t))
        elif kind == C.SWAP:
            recs.append(C.swap(t, o))
        elif kind == C.U3:
            recs.append(C.u3(t, *(float(v) for v in rng.uniform(0, 2 * np.pi, 3))))
        elif kind == C.U:
            recs.append(C.u(t, C.random_unitary(rng)))
        elif kind == C.CU:
            recs.append(C.cu(o, t, C.random_unitary(rng)))
        elif kind == C.PK:
            j = int(rng.integers(0, 40))
            recs.append(C.pk(t, int(rng.integers(-(1 << 40), 1 << 40)), j))
        else:
            j = int(rng.integers(0, 40))
            recs.append(C.cpk(o, t, int(rng.integers(-(1 << 40), 1 << 40)), j))
    return C.gates(recs)


def fold_leading(g):
    """The library's fold of a recorded basis state: while a qubit is
    untouched, X flips its bit of the basis index (when it carries no
    Hadamard) and H toggles it in the Hadamard mask; every other gate, and an
    X on a Hadamard qubit, touches its qubits.  Identity qubit map.  Returns
    (basis index, Hadamard mask, the rest of the list)."""
    basis, hq, touched, rest = 0, 0, set(), []
    for r in g:
        kind, t, c = int(r["kind"]), int(r["target"]), int(r["control"])
        if t not in touched and kind == C.X and not (hq >> t) & 1:
            basis ^= 1 << t
            continue
        if t not in touched and kind == C.H:
            hq ^= 1 << t
            continue
        touched.add(t)
        if c >= 0:
            touched.add(c)
        rest.append(r)
    return basis, hq, (C.gates(rest) if rest else C.gates([]))


def without_leading_x(g):
    """The gate list the library plans when the state is a recorded basis
    state: the leading X and H gates that only change the recorded state are
    dropped (fold_leading)."""
    return fold_leading(g)[2]


def general_circuit(n, m, seed, orc=None):
    """Seeded circuit mixing the paper's gates with the general set:
    multi-controlled U (1..3 controls), two-qubit unitaries (four records)
    and measurements.  Each measurement's u is chosen from the oracle's own
    probability p0 at that point, half-way inside the outcome it selects, so
    that no outcome sits on a CDF boundary (input construction only)."""
    import numpy as np

    rng = np.random.default_rng(seed)
    recs = []
    for r in mixed_circuit(n, m, seed + 1):
        recs.append(r)
        draw = rng.integers(0, 10)
        if draw < 2:
            t = int(rng.integers(0, n))
            others = [q for q in range(n) if q != t]
            k = int(rng.integers(1, min(3, n - 1) + 1))
            ctr = [int(c) for c in rng.choice(others, size=k, replace=False)]
            recs.append(C.mcu(ctr, t, C.random_unitary(rng)))
        elif draw < 4 and n >= 2:
            a, b = (int(q) for q in rng.choice(n, size=2, replace=False))
            z = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
            q4, r4 = np.linalg.qr(z)
            recs += C.u2q(a, b, q4 * (np.diag(r4) / np.abs(np.diag(r4))))
        elif draw < 5 and orc is not None:
            t = int(rng.integers(0, n))
            psi = orc.run(n, C.gates(recs))
            x = np.arange(1 << n)
            p0 = float(np.sum(np.abs(psi[((x >> t) & 1) == 0]) ** 2))
            u = 0.5 * p0 if (rng.random() < 0.5 and p0 > 1e-6) or p0 > 1 - 1e-6 else 0.5 * (1 + p0)
            recs.append(C.measure(t, u))
    return C.gates(recs)
