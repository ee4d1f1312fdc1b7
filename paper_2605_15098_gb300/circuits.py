"""Seeded circuit generators: the synthetic workloads of the QPE benchmark.

This module builds gate lists only.  It applies no gate, builds no matrix and
evaluates no phase: the amplitude arithmetic lives in the CUDA library (and,
independently, in the test oracle).  Both sides receive the same records.

Random numbers come from SplitMix64 (S. Vigna's public 64-bit generator:
add the golden-ratio increment 0x9E3779B97F4A7C15, then two xor-shift /
multiply rounds and a final xor-shift), written here from that description.

Workloads:

* ``qpe(n, seed)`` - the phase-estimation benchmark of Sec. IV-A generalised
  to four eigenstate qubits: t = n - 4 counting qubits q0..q(t-1), targets
  q(t)..q(t+3) put in |1> by X, U_i = P(2*pi*a_i / 2^t) on target i with
  a_i in [0, 63] drawn from the seed, controlled-U^(2^j) from counting qubit j
  written as CP(2*pi*a_i*2^j / 2^t) (Eq. 3: U^a = P(2*pi*2^-t*a)), then the
  inverse QFT of the counting register made of SWAPs, CP(-pi/2^(m-k)) and H.
  The counting register then holds y = sum(a_i) mod 2^t with probability 1.
* ``paper_qpe(n)`` - the paper's own instance (Fig. 3 circuit, Eq. 2): n
  counting qubits, one eigenstate qubit, U = P(2*pi*2^-n), qubit 0 controls
  U^(2^(n-1)); the measured counting bitstring q0..q(n-1) is 00...01.
* ``random_circuit(n, depth, seed)`` - layers of U3 on every qubit with angles
  uniform in [0, 2*pi), then CZ on a random perfect matching.
* ``batch_specs(count, seed)`` - per-instance qubit counts and seeds for the
  batched QPE workload.
"""
from __future__ import annotations

import numpy as np

# Public gate record (96 bytes); identical to ``sv_gate`` in include/sv.h.
GATE_DTYPE = np.dtype(
    [
        ("kind", "<i4"),
        ("target", "<i4"),
        ("control", "<i4"),
        ("log2den", "<i4"),
        ("num", "<i8"),
        ("reserved", "<i8"),
        ("p", "<f8", (8,)),
    ]
)
assert GATE_DTYPE.itemsize == 96

X, H, P, CP, CZ, SWAP, U3, U, CU, PK, CPK, MCU, U2Q, MAT, MEASURE = range(15)
KIND_NAMES = ["X", "H", "P", "CP", "CZ", "SWAP", "U3", "U", "CU", "PK", "CPK", "MCU", "U2Q", "MAT",
              "MEASURE"]
DIAGONAL_KINDS = (P, CP, CZ, PK, CPK)

DEFAULT_SEED = 2605150980
_MASK64 = (1 << 64) - 1


class SplitMix64:
    """64-bit SplitMix generator (public algorithm)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))


def _rec(kind, target, control=-1, p=(), num=0, log2den=0):
    return (kind, target, control, log2den, num, 0, tuple(p) + (0.0,) * (8 - len(p)))


def gates(records) -> np.ndarray:
    return np.array(list(records), dtype=GATE_DTYPE)


# ---- single records -------------------------------------------------------
def x(q):
    return _rec(X, q)


def h(q):
    return _rec(H, q)


def p(q, phi):
    return _rec(P, q, p=(phi,))


def cp(c, t, phi):
    return _rec(CP, t, c, p=(phi,))


def cz(a, b):
    return _rec(CZ, b, a)


def swap(a, b):
    return _rec(SWAP, a, b)


def u3(q, theta, phi, lam):
    return _rec(U3, q, p=(theta, phi, lam))


def u(q, m):
    m = np.asarray(m, dtype=np.complex128).reshape(2, 2)
    flat = []
    for e in m.reshape(-1):
        flat += [float(e.real), float(e.imag)]
    return _rec(U, q, p=flat)


def cu(c, t, m):
    r = list(u(t, m))
    r[0], r[2] = CU, c
    return tuple(r)


def pk(q, k, j):
    """P(2*pi*k/2^j)."""
    return _rec(PK, q, num=int(k), log2den=int(j))


def cpk(c, t, k, j):
    """CP(2*pi*k/2^j) with control c, target t."""
    return _rec(CPK, t, c, num=int(k), log2den=int(j))


def mcu(controls, t, m):
    """U (2x2) on t where every qubit in `controls` is 1: the control mask in num."""
    r = list(u(t, m))
    r[0], r[2], r[4] = MCU, -1, int(sum(1 << int(c) for c in controls))
    return tuple(r)


def u2q(a, b, m4):
    """Four records: a 4x4 unitary on the pair (a, b), basis index k = bit_a +
    2 bit_b; rows 0..3 of the matrix in the p of this record (kind U2Q) and
    of three continuation records (kind MAT)."""
    m4 = np.asarray(m4, dtype=np.complex128).reshape(4, 4)
    out = []
    for r in range(4):
        flat = []
        for e in m4[r]:
            flat += [float(e.real), float(e.imag)]
        out.append(_rec(U2Q if r == 0 else MAT, a, b, p=flat))
    return out


def measure(q, uval):
    """Projective measurement of q with the caller's uniform uval in [0, 1)."""
    return _rec(MEASURE, q, p=(float(uval),))


# ---- workloads ------------------------------------------------------------
def qpe_phases(seed: int, count: int = 4) -> list[int]:
    g = SplitMix64(seed)
    return [g.next() >> 58 for _ in range(count)]


def inverse_qft(t: int, first: int = 0) -> list:
    """Inverse QFT on qubits first..first+t-1, qubit first = least significant."""
    recs = [swap(first + m, first + t - 1 - m) for m in range(t // 2)]
    for m in range(t):
        for k in range(m):
            # CP(-pi / 2^(m-k)) = CP(2*pi * (-1) / 2^(m-k+1))
            recs.append(cpk(first + k, first + m, -1, m - k + 1))
        recs.append(h(first + m))
    return recs


def qft(t: int, first: int = 0) -> list:
    """Forward QFT (the inverse's gates reversed, angles negated)."""
    recs = []
    for m in reversed(range(t)):
        recs.append(h(first + m))
        for k in reversed(range(m)):
            recs.append(cpk(first + k, first + m, 1, m - k + 1))
    recs += [swap(first + m, first + t - 1 - m) for m in range(t // 2)]
    return recs


def qpe(n: int, seed: int = DEFAULT_SEED, targets: int = 4):
    """QPE benchmark circuit on n qubits (t = n - targets counting qubits).

    Returns (gate array, expected basis index, info dict)."""
    t = n - targets
    if t < 1:
        raise ValueError("qpe needs more qubits than targets")
    a = qpe_phases(seed, targets)
    recs = [x(t + i) for i in range(targets)]
    recs += [h(j) for j in range(t)]
    for j in range(t):
        for i in range(targets):
            recs.append(cpk(j, t + i, a[i] << j, t))
    recs += inverse_qft(t)
    y = sum(a) % (1 << t)
    expected = y | (((1 << targets) - 1) << t)
    return gates(recs), expected, {"t": t, "a": a, "y": y, "mask": (1 << t) - 1}


def qpe_gate_count(n: int, targets: int = 4) -> int:
    t = n - targets
    return targets + t + targets * t + t // 2 + t + t * (t - 1) // 2


def paper_qpe(nc: int):
    """The paper's QPE instance: nc counting qubits + 1 eigenstate qubit.

    Counting qubit q controls U^(2^(nc-1-q)) with U = P(2*pi*2^-nc) (Eq. 2-3,
    Fig. 3); qubit 0 is the most significant bit of the estimate.  Returns
    (gates, counting mask, expected counting outcome index)."""
    tq = nc
    recs = [x(tq)] + [h(q) for q in range(nc)]
    for q in range(nc):
        recs.append(cpk(q, tq, 1 << (nc - 1 - q), nc))
    # inverse QFT with qubit 0 most significant
    recs += [swap(q, nc - 1 - q) for q in range(nc // 2)]
    for q in reversed(range(nc)):
        for r in reversed(range(q + 1, nc)):
            recs.append(cpk(r, q, -1, r - q + 1))
        recs.append(h(q))
    # bitstring q0..q(nc-1) = 0...01  ->  only qubit nc-1 is 1
    return gates(recs), (1 << nc) - 1, 1 << (nc - 1)


def random_circuit(n: int, depth: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Layers of U3 (angles uniform in [0, 2*pi)) then CZ on a random matching."""
    g = SplitMix64(seed)
    two_pi = 2.0 * np.pi
    recs = []
    for _ in range(depth):
        for q in range(n):
            th, ph, la = (two_pi * g.uniform() for _ in range(3))
            recs.append(u3(q, th, ph, la))
        perm = list(range(n))
        for i in range(n - 1, 0, -1):  # Fisher-Yates
            j = g.next() % (i + 1)
            perm[i], perm[j] = perm[j], perm[i]
        for m in range(n // 2):
            recs.append(cz(perm[2 * m], perm[2 * m + 1]))
    return gates(recs)


def batch_specs(count: int, seed: int = DEFAULT_SEED, n_lo: int = 10, n_hi: int = 20):
    """(n_i, seed_i) for the batched QPE workload; n_i uniform in [n_lo, n_hi]."""
    g = SplitMix64(seed)
    span = n_hi - n_lo + 1
    return [(n_lo + g.next() % span, seed + 1 + i) for i in range(count)]


def qpe_batch(count: int, seed: int = DEFAULT_SEED, n_lo: int = 10, n_hi: int = 20):
    """The batched QPE workload: (n_i, gates_i, counting mask_i, expected y_i) per instance."""
    out = []
    for n, s in batch_specs(count, seed, n_lo, n_hi):
        g, _, info = qpe(n, s)
        out.append((n, g, info["mask"], info["y"]))
    return out


def random_unitary(rng: np.random.Generator) -> np.ndarray:
    """Haar-ish random 2x2 unitary from a QR decomposition (test input)."""
    z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))
