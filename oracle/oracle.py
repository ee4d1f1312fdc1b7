"""Python front end of the FP64 CPU oracle (``sv_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg may import this module; the library does not.  It loads its
own shared object, built from ``sv_oracle.c`` with gcc, and never touches the
CUDA library.

Functions follow the paper's definitions (arxiv 2605.15098):
``apply`` runs Algorithm 1 gate by gate with the control rule of Sec. III-A
(taken to a set of controls for MCU), a general two-qubit unitary U2Q and a
collapsing MEASURE (``apply_measured`` also returns the outcomes),
``marginal`` / ``argmax`` / ``sample`` read out the measured outcome of
Sec. IV-A.  Gate records are NumPy structured arrays with the byte layout of
the library's gate record (96 bytes, see ``GATE_DTYPE``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sv_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")

# Same layout as the library's gate record; declared here on its own.
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

_lock = threading.Lock()
_libs: dict[int, ctypes.CDLL] = {}


def lib_path(mutation: int = 0) -> str:
    name = "liboracle.so" if mutation == 0 else f"liboracle_mut{mutation}.so"
    return os.path.join(BUILD_DIR, name)


def build(mutation: int = 0, force: bool = False) -> str:
    """Compile the oracle (optionally with a planted mistake for pin tests)."""
    out = lib_path(mutation)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(SRC)):
        return out
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-std=c11", "-shared", "-fPIC", f"-DOR_MUTATION={mutation}",
           SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load(mutation: int = 0) -> ctypes.CDLL:
    with _lock:
        if mutation in _libs:
            return _libs[mutation]
        lib = ctypes.CDLL(build(mutation))
        u64, i32, dp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        lib.or_init.argtypes = [i32, dp]
        lib.or_apply.argtypes = [i32, dp, dp, u64]
        lib.or_apply_measured.argtypes = [i32, dp, dp, u64, dp]
        lib.or_marginal.argtypes = [i32, dp, u64, dp]
        lib.or_argmax.argtypes = [dp, u64, dp, dp]
        lib.or_cdf.argtypes = [dp, u64, dp]
        lib.or_sample.argtypes = [dp, u64, dp, u64, dp, dp]
        lib.or_num_threads.restype = i32
        lib.or_set_threads.argtypes = [i32]
        for f in (lib.or_init, lib.or_apply, lib.or_apply_measured, lib.or_marginal, lib.or_argmax,
                  lib.or_cdf, lib.or_sample):
            f.restype = i32
        _libs[mutation] = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def num_threads() -> int:
    return load().or_num_threads()


def set_threads(t: int) -> None:
    load().or_set_threads(int(t))


def init(n: int) -> np.ndarray:
    """|0...0> as complex128 (Sec. III-A state of 2^n amplitudes)."""
    psi = np.empty(1 << n, dtype=np.complex128)
    rc = load().or_init(n, _ptr(psi))
    if rc:
        raise ValueError(f"oracle init failed for n={n}")
    return psi


def apply(n: int, psi: np.ndarray, gates: np.ndarray, mutation: int = 0) -> np.ndarray:
    """Apply the gate list in order, in place, by Algorithm 1."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == 1 << n
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    rc = load(mutation).or_apply(n, _ptr(psi), _ptr(g) if g.size else None, g.size)
    if rc:
        raise ValueError(f"oracle rejected gate list (code {rc})")
    return psi


def apply_measured(n: int, psi: np.ndarray, gates: np.ndarray, mutation: int = 0) -> np.ndarray:
    """Apply the list in place; returns the outcomes of its MEASURE gates, in order."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == 1 << n
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    out = np.zeros(max(1, g.size), dtype=np.uint8)
    rc = load(mutation).or_apply_measured(n, _ptr(psi), _ptr(g) if g.size else None, g.size, _ptr(out))
    if rc:
        raise ValueError(f"oracle rejected gate list (code {rc})")
    nm = int(np.sum(g["kind"] == 14)) if g.size else 0
    return out[:nm].copy()


def run(n: int, gates: np.ndarray, mutation: int = 0) -> np.ndarray:
    psi = init(n)
    return apply(n, psi, gates, mutation)


def marginal(n: int, psi: np.ndarray, mask: int) -> np.ndarray:
    """Renormalised marginal probabilities over the qubits of ``mask``."""
    k = bin(mask).count("1")
    out = np.empty(1 << k, dtype=np.float64)
    rc = load().or_marginal(n, _ptr(psi), mask, _ptr(out))
    if rc:
        raise ValueError(f"oracle marginal failed ({rc})")
    return out


def argmax(p: np.ndarray) -> tuple[int, float]:
    idx = np.zeros(1, dtype=np.uint64)
    pm = np.zeros(1, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    load().or_argmax(_ptr(p), p.size, _ptr(idx), _ptr(pm))
    return int(idx[0]), float(pm[0])


def cdf(p: np.ndarray) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.empty_like(p)
    load().or_cdf(_ptr(p), p.size, _ptr(out))
    return out


def sample(p: np.ndarray, u: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Inverse-CDF outcomes for the uniforms ``u`` and each shot's boundary margin."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(u.size, dtype=np.uint64)
    margin = np.empty(u.size, dtype=np.float64)
    rc = load().or_sample(_ptr(p), p.size, _ptr(u), u.size, _ptr(out), _ptr(margin))
    if rc:
        raise ValueError(f"oracle sample failed ({rc})")
    return out, margin
