"""The paper's partitioned simulation on the host CPU (Sec. III-B), a second
CPU baseline beside the oracle's plain Algorithm 1 (see ``cpupart.c``).

Not part of the GPU path: the benchmark times it on the host cores to check
the paper's finding that partitioning does not pay on a CPU.  The shared
object is built in-tree with gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpupart.c")
OUT = os.path.join(HERE, "_build", "libcpupart.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    tmp = OUT + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O3", "-fopenmp", "-std=c11", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, OUT)
    return OUT


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            lb = ctypes.CDLL(build())
            lb.cp_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                  ctypes.c_void_p]
            lb.cp_run.restype = ctypes.c_int
            lb.cp_num_threads.restype = ctypes.c_int
            _lib = lb
        return _lib


def num_threads() -> int:
    return lib().cp_num_threads()


def run(n: int, gates: np.ndarray, l: int) -> tuple[np.ndarray, dict]:
    """|0...0> then the gate list with blocks of 2^l amplitudes; the state in
    logical order and the counts of flushes and global-local swaps."""
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    g = np.ascontiguousarray(gates)
    assert g.dtype.itemsize == 96
    stats = np.zeros(2, dtype=np.int64)
    rc = lib().cp_run(n, l, psi.ctypes.data, g.ctypes.data if g.size else None, g.size, stats.ctypes.data)
    if rc:
        raise ValueError(f"cp_run failed ({rc})")
    return psi, {"passes": int(stats[0]), "swaps": int(stats[1])}
