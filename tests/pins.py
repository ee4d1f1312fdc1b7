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


ALL_PINS = ("pin_kronecker", "pin_qpe", "pin_qft_closed_form", "pin_uniform",
            "pin_identities", "pin_norm")
