"""Checks that pin the FP64 oracle to facts fixed outside it.

Each ``pin_*`` takes ``run(n, gates) -> complex128 state`` and returns a list
of failure strings (empty = pass), so that the same checks can be run against
the oracle and against deliberately broken builds of it.

What fixes each expected value:
  * Kronecker brute force: Eq. 1 written as explicit 2^n x 2^n operators with
    qubit q as Kronecker factor n-1-q (the ordering under which Eq. 1 and the
    stride 2^t of Algorithm 1 agree), for explicit random 2x2 matrices.
  * QPE (Eq. 2-3): an eigenphase of exactly y/2^t is read out as y with
    probability 1.
  * QFT on a basis state |y>: amplitudes exp(2*pi*i*x*y/2^t) / 2^(t/2).
  * H^n |0> is the uniform state 2^(-n/2).
  * Textbook identities: HH = I, XX = I, H.CZ.H = CNOT, HP(pi)H = X, CP(f)CP(-f) = I,
    SWAP = CNOT.CNOT.CNOT, U3(pi/2,0,pi) = H, U3(pi,0,pi) = X, U3(0,0,l) = P(l),
    U3(t,p,l)^-1 = U3(-t,-l,-p).
  * The general gate set: a multi-controlled U as I - P + P (x) U with P the
    product of the controls' |1><1| projectors (Eq. 1's operators); a
    two-qubit unitary expanded in the Pauli basis, sum of c_PQ P_b (x) Q_a,
    each term an Eq. 1 Kronecker product; Toffoli's truth table, U2Q of the
    SWAP / CNOT / product matrices against SWAP, CU and two U gates; the
    Born rule for a measurement (outcome of a basis state, of |+>, and the
    projected, renormalised state of a brute-force random state).
"""
from __future__ import annotations

import numpy as np

from paper_2605_15098_gb300 import circuits as C


# ---------------------------------------------------------------- brute force
def _embed_1q(n: int, q: int, m: np.ndarray) -> np.ndarray:
    """I^(n-1-q) (x) m (x) I^q."""
    return np.kron(np.kron(np.eye(1 << (n - 1 - q)), m), np.eye(1 << q))


def _proj(n: int, q: int, bit: int) -> np.ndarray:
    pb = np.zeros((2, 2))
    pb[bit, bit] = 1.0
    return _embed_1q(n, q, pb)


def kron_operator(n: int, rec) -> np.ndarray:
    """Full operator of one U / CU / SWAP record (explicit matrix inputs only)."""
    kind = int(rec["kind"])
    t = int(rec["target"])
    if kind in (C.U, C.CU):
        pr = np.asarray(rec["p"], dtype=np.float64)
        m = (pr[0::2] + 1j * pr[1::2]).reshape(2, 2)
        if kind == C.U:
            return _embed_1q(n, t, m)
        c = int(rec["control"])
        return _proj(n, c, 0) + _proj(n, c, 1) @ _embed_1q(n, t, m)
    if kind == C.SWAP:
        a, b = t, int(rec["control"])
        dim = 1 << n
        op = np.zeros((dim, dim))
        for xi in range(dim):
            ba, bb = (xi >> a) & 1, (xi >> b) & 1
            yi = xi
            if ba != bb:
                yi = xi ^ (1 << a) ^ (1 << b)
            op[yi, xi] = 1.0
        return op
    raise ValueError("brute force covers explicit-matrix gates and SWAP only")


_PAULI = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.diag([1.0, -1.0])]


def mcu_operator(n: int, controls, t: int, m: np.ndarray) -> np.ndarray:
    """I - P + P (x) U, P = product of |1><1| on every control."""
    dim = 1 << n
    proj = np.eye(dim)
    for c in controls:
        proj = proj @ _proj(n, c, 1)
    return np.eye(dim) - proj + proj @ _embed_1q(n, t, m)


def u2q_operator(n: int, a: int, b: int, m4: np.ndarray) -> np.ndarray:
    """m4 acts on k = bit_a + 2 bit_b, i.e. it is sum over Paulis P, Q of
    c_PQ P (x) Q with P on qubit b and Q on qubit a, c_PQ = tr((P (x) Q)^+ m4) / 4."""
    op = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for pb in _PAULI:
        for qa in _PAULI:
            c = np.trace(np.kron(pb, qa).conj().T @ m4) / 4.0
            if abs(c) > 0:
                op += c * (_embed_1q(n, b, pb) @ _embed_1q(n, a, qa))
    return op


def random_u4(rng) -> np.ndarray:
    z = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def brute_force(n: int, gates: np.ndarray) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    for rec in gates:
        psi = kron_operator(n, rec) @ psi
    return psi


def random_explicit_circuit(n: int, m: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    recs = []
    for _ in range(m):
        r = rng.integers(0, 3)
        t = int(rng.integers(0, n))
        if r == 0:
            recs.append(C.u(t, C.random_unitary(rng)))
        elif r == 1:
            c = int(rng.integers(0, n - 1))
            c = c + 1 if c >= t else c
            recs.append(C.cu(c, t, C.random_unitary(rng)))
        else:
            b = int(rng.integers(0, n - 1))
            b = b + 1 if b >= t else b
            recs.append(C.swap(t, b))
    return C.gates(recs)


# ---------------------------------------------------------------- pins
def pin_kronecker(run, sizes=(1, 2, 3, 5, 7), gates_per=24, seeds=(1, 2)) -> list[str]:
    bad = []
    for n in sizes:
        for s in seeds:
            g = random_explicit_circuit(max(n, 2), gates_per, 1000 * n + s)
            nn = max(n, 2)
            ref = brute_force(nn, g)
            got = run(nn, g)
            err = float(np.max(np.abs(ref - got)))
            if not err < 1e-13:
                bad.append(f"kronecker n={nn} seed={s}: max err {err:.3e}")
    return bad


def pin_qpe(run, sizes=(5, 6, 8, 10, 12), seeds=(C.DEFAULT_SEED, 7, 99)) -> list[str]:
    bad = []
    for n in sizes:
        for s in seeds:
            g, expected, _ = C.qpe(n, s)
            psi = run(n, g)
            p = np.abs(psi) ** 2
            if not abs(p[expected] - 1.0) < 1e-12:
                bad.append(f"qpe n={n} seed={s}: P(expected)={p[expected]!r}")
    return bad


def pin_paper_qpe(run, fixture) -> list[str]:
    """The paper's own QPE instances (tests/golden/paper_qpe.txt)."""
    bad = []
    for nc, bitstring, prob in fixture:
        g, mask, _ = C.paper_qpe(nc)
        psi = run(nc + 1, g)
        p = np.abs(psi) ** 2
        # counting outcome from the bitstring q0..q(nc-1)
        idx = sum(1 << q for q, ch in enumerate(bitstring) if ch == "1")
        full = idx | (1 << nc)  # eigenstate qubit stays |1>
        if not abs(p[full] - prob) < 1e-12:
            bad.append(f"paper qpe nc={nc}: P({bitstring})={p[full]!r}")
    return bad


def pin_qft_closed_form(run, sizes=(1, 2, 3, 4, 6, 8)) -> list[str]:
    bad = []
    for t in sizes:
        for y in sorted({0, 1, (1 << t) - 1, (5 * t) % (1 << t)}):
            recs = [C.x(q) for q in range(t) if (y >> q) & 1] + C.qft(t)
            psi = run(t, C.gates(recs))
            xs = np.arange(1 << t)
            ref = np.exp(2j * np.pi * xs * y / (1 << t)) / np.sqrt(1 << t)
            err = float(np.max(np.abs(psi - ref)))
            if not err < 1e-13:
                bad.append(f"qft t={t} y={y}: max err {err:.3e}")
    return bad


def pin_uniform(run, sizes=(1, 3, 9)) -> list[str]:
    bad = []
    for n in sizes:
        psi = run(n, C.gates([C.h(q) for q in range(n)]))
        err = float(np.max(np.abs(psi - 2.0 ** (-n / 2))))
        if not err < 1e-15:
            bad.append(f"uniform n={n}: max err {err:.3e}")
    return bad


def _eq_states(run, n, g1, g2, tol=1e-13):
    """Compare two circuits on a fixed random-ish input prepared by U gates."""
    rng = np.random.default_rng(n * 31 + len(g1))
    prep = [C.u(q, C.random_unitary(rng)) for q in range(n)]
    a = run(n, C.gates(prep + list(g1)))
    b = run(n, C.gates(prep + list(g2)))
    return float(np.max(np.abs(a - b))) < tol


def pin_identities(run) -> list[str]:
    bad = []
    n = 3
    checks = {
        "HH=I": ([C.h(1), C.h(1)], []),
        "XX=I": ([C.x(2), C.x(2)], []),
        "H.CZ.H=CNOT": ([C.h(0), C.cz(1, 0), C.h(0)], [C.cu(1, 0, [[0, 1], [1, 0]])]),
        "HPH=X": ([C.h(0), C.p(0, np.pi), C.h(0)], [C.x(0)]),
        "CP(f)CP(-f)=I": ([C.cp(0, 2, 0.7), C.cp(0, 2, -0.7)], []),
        "CPK(k)CPK(-k)=I": ([C.cpk(2, 1, 3, 5), C.cpk(2, 1, -3, 5)], []),
        "CPK(2^j)=CZ": ([C.cpk(1, 2, 8, 4)], [C.cz(1, 2)]),
        "PK(1,2)^2=PK(1,1)": ([C.pk(0, 1, 2), C.pk(0, 1, 2)], [C.pk(0, 1, 1)]),
        "SWAP=3CNOT": ([C.swap(0, 2)],
                       [C.cu(0, 2, [[0, 1], [1, 0]]), C.cu(2, 0, [[0, 1], [1, 0]]),
                        C.cu(0, 2, [[0, 1], [1, 0]])]),
        "U3(pi/2,0,pi)=H": ([C.u3(1, np.pi / 2, 0.0, np.pi)], [C.h(1)]),
        "U3(pi,0,pi)=X": ([C.u3(2, np.pi, 0.0, np.pi)], [C.x(2)]),
        "U3(0,0,l)=P(l)": ([C.u3(0, 0.0, 0.0, 1.3)], [C.p(0, 1.3)]),
        "U3(t,p,l)U3(t,p,l)^-1=I": ([C.u3(1, 0.4, 1.1, -2.3), C.u3(1, -0.4, 2.3, -1.1)], []),
    }
    for name, (g1, g2) in checks.items():
        if not _eq_states(run, n, g1, g2):
            bad.append(f"identity {name} fails")
    # X|0> = |1>, H|0> = (|0>+|1>)/sqrt2, P(phi)|1> = e^{i phi}|1>
    psi = run(1, C.gates([C.x(0)]))
    if not (abs(psi[1] - 1) < 1e-15 and abs(psi[0]) < 1e-15):
        bad.append("X|0> != |1>")
    psi = run(1, C.gates([C.x(0), C.p(0, 0.3)]))
    if not abs(psi[1] - np.exp(0.3j)) < 1e-15:
        bad.append("P(phi)|1> != e^{i phi}|1>")
    psi = run(1, C.gates([C.x(0), C.pk(0, 1, 3)]))
    if not abs(psi[1] - np.exp(2j * np.pi / 8)) < 1e-15:
        bad.append("PK(1,3)|1> != e^{i pi/4}|1>")
    return bad


def pin_norm(run, n=10, depth=6, seed=5) -> list[str]:
    g = C.random_circuit(n, depth, seed)
    psi = run(n, g)
    err = abs(float(np.vdot(psi, psi).real) - 1.0)
    return [] if err < 1e-13 * len(g) else [f"norm drift {err:.3e}"]


def _state_prep(rng, n):
    return [C.u(q, C.random_unitary(rng)) for q in range(n)]


def pin_mcu_kronecker(run, sizes=(3, 4, 6), seeds=(1, 2, 3)) -> list[str]:
    """Random multi-controlled U gates (1 to 3 controls) after random local
    unitaries, against I - P + P (x) U."""
    bad = []
    for n in sizes:
        for s in seeds:
            rng = np.random.default_rng(500 * n + s)
            recs = _state_prep(rng, n)
            ref = brute_force(n, C.gates(recs))
            for _ in range(6):
                t = int(rng.integers(0, n))
                others = [q for q in range(n) if q != t]
                k = int(rng.integers(1, min(3, n - 1) + 1))
                ctr = [int(c) for c in rng.choice(others, size=k, replace=False)]
                m = C.random_unitary(rng)
                recs.append(C.mcu(ctr, t, m))
                ref = mcu_operator(n, ctr, t, m) @ ref
            got = run(n, C.gates(recs))
            err = float(np.max(np.abs(got - ref)))
            if not err < 1e-13:
                bad.append(f"mcu n={n} seed={s}: max err {err:.3e}")
    return bad


def pin_u2q_pauli(run, sizes=(2, 3, 5), seeds=(1, 2)) -> list[str]:
    """Random two-qubit unitaries on random ordered pairs, against their
    Pauli expansion."""
    bad = []
    for n in sizes:
        for s in seeds:
            rng = np.random.default_rng(700 * n + s)
            recs = _state_prep(rng, n)
            ref = brute_force(n, C.gates(recs))
            for _ in range(5):
                a, b = (int(q) for q in rng.choice(n, size=2, replace=False))
                m4 = random_u4(rng)
                recs += C.u2q(a, b, m4)
                ref = u2q_operator(n, a, b, m4) @ ref
            got = run(n, C.gates(recs))
            err = float(np.max(np.abs(got - ref)))
            if not err < 1e-13:
                bad.append(f"u2q n={n} seed={s}: max err {err:.3e}")
    return bad


def pin_general_identities(run) -> list[str]:
    bad = []
    n = 3
    rng = np.random.default_rng(11)
    A, B = C.random_unitary(rng), C.random_unitary(rng)
    X = [[0, 1], [1, 0]]
    swap4 = np.eye(4)[[0, 2, 1, 3]]
    cnot_b_to_a = np.eye(4)[[0, 1, 3, 2]]  # flips bit a (k bit 0) when bit b (k bit 1) is 1
    checks = {
        "MCU(1 control)=CU": ([C.mcu([2], 0, A)], [C.cu(2, 0, A)]),
        "U2Q(SWAP)=SWAP": (C.u2q(0, 2, swap4), [C.swap(0, 2)]),
        "U2Q(A(x)B)=B on a, A on b": (C.u2q(1, 2, np.kron(A, B)), [C.u(1, B), C.u(2, A)]),
        "U2Q(CNOT)=CU(X)": (C.u2q(0, 1, cnot_b_to_a), [C.cu(1, 0, X)]),
    }
    for name, (g1, g2) in checks.items():
        if not _eq_states(run, n, g1, g2):
            bad.append(f"identity {name} fails")
    for x in range(8):  # Toffoli: flip qubit 2 iff qubits 0 and 1 are 1
        prep = [C.x(q) for q in range(3) if (x >> q) & 1]
        psi = run(3, C.gates(prep + [C.mcu([0, 1], 2, X)]))
        y = x ^ 4 if (x & 3) == 3 else x
        if not abs(psi[y] - 1.0) < 1e-15:
            bad.append(f"toffoli |{x}> -> |{y}> fails")
    return bad


def pin_measure(run) -> list[str]:
    bad = []
    # a basis state is left as it is, whatever u
    for x, q, u in ((5, 0, 0.3), (5, 1, 0.99), (6, 2, 0.0)):
        prep = [C.x(b) for b in range(3) if (x >> b) & 1]
        psi = run(3, C.gates(prep + [C.measure(q, u)]))
        if not abs(psi[x] - 1.0) < 1e-15:
            bad.append(f"measure basis |{x}> qubit {q} changed the state")
    # |+>: outcome 0 iff u < 1/2, then |0> or |1> exactly
    for u in (0.1, 0.49, 0.51, 0.9):
        psi = run(1, C.gates([C.h(0), C.measure(0, u)]))
        want = 0 if u < 0.5 else 1
        if not (abs(psi[want] - 1.0) < 1e-15 and abs(psi[1 - want]) < 1e-15):
            bad.append(f"measure |+> with u={u}: {psi}")
    # Born rule on a brute-force random state: outcome by the CDF rule, then
    # the projection renormalised
    rng = np.random.default_rng(21)
    n = 4
    prep = _state_prep(rng, n) + [C.cu(0, 3, C.random_unitary(rng)), C.cu(2, 1, C.random_unitary(rng))]
    pre = brute_force(n, C.gates(prep))
    for q in range(n):
        xs = np.arange(1 << n)
        p0 = float(np.sum(np.abs(pre[((xs >> q) & 1) == 0]) ** 2))
        for u in (0.5 * p0, 0.5 * (1 + p0)):
            out = 0 if p0 > u else 1
            keep = ((xs >> q) & 1) == out
            post = np.where(keep, pre, 0) / np.sqrt(np.sum(np.abs(pre[keep]) ** 2))
            psi = run(n, C.gates(prep + [C.measure(q, u)]))
            err = float(np.max(np.abs(psi - post)))
            if not err < 1e-13:
                bad.append(f"measure qubit {q} u={u:.3f}: max err {err:.3e}")
            # measuring again repeats the outcome and leaves the state
            psi2 = run(n, C.gates(prep + [C.measure(q, u), C.measure(q, 1.0 - 1e-9 if out else 0.0)]))
            if not float(np.max(np.abs(psi2 - post))) < 1e-13:
                bad.append(f"repeated measure qubit {q} changed the state")
    return bad


ALL_PINS = ("pin_kronecker", "pin_qpe", "pin_qft_closed_form", "pin_uniform",
            "pin_identities", "pin_norm", "pin_mcu_kronecker", "pin_u2q_pauli",
            "pin_general_identities", "pin_measure")
