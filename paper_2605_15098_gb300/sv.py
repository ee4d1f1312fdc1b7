"""Thin ctypes binding of libsv (include/sv.h): same names, argument marshalling only.

Every step of the simulation runs in the CUDA library; this module converts
Python / NumPy / PyTorch arguments into pointers and sizes and turns error
codes into exceptions.  It fails loudly (``LibraryMissing``) when libsv.so has
not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .circuits import GATE_DTYPE

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsv.so")

SV_C64, SV_C128 = 0, 1
SV_OK, SV_ERR_ARG, SV_ERR_OOM, SV_ERR_CUDA, SV_ERR_TIMEOUT, SV_ERR_STATE, SV_ERR_UNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6)
SV_MODE_AUTO, SV_MODE_PERGATE, SV_MODE_PARTITIONED, SV_MODE_FUSED = 0, 1, 2, 3
SV_FLAG_NO_DIAG_MERGE, SV_FLAG_PAPER_SWAP, SV_FLAG_NO_RELABEL, SV_FLAG_GENERIC_TILE = 1, 2, 4, 8
SV_FLAG_NO_PLAN_CACHE = 16
SV_FLAG_EARLY_DIAG = 32
SV_FLAG_GREEDY_ONLY = 64
SV_FLAG_L2_BLOCKS = 128
SV_FLAG_NARROW_FIRST = 256
SV_PLANNER_GREEDY, SV_PLANNER_LEARNED = 0, 1

EXPORTS = (
    "sv_create", "sv_create_on", "sv_destroy", "sv_reset", "sv_info", "sv_qubit_map",
    "sv_apply_circuit", "sv_last_stats", "sv_last_measurements", "sv_probabilities",
    "sv_probabilities_device",
    "sv_argmax", "sv_sample", "sv_copy_out", "sv_copy_in", "sv_last_error", "sv_version",
    "sv_profile", "sv_profile_read", "sv_launch_count", "sv_marginal_noalloc", "sv_plan_export",
    "sv_batch_create", "sv_batch_run", "sv_batch_info", "sv_batch_destroy", "sv_apply_circuit_batch",
    "sv_autotune", "sv_batch_autotune",
    "sv_cost_features", "sv_cost_model_create", "sv_cost_model_destroy", "sv_cost_model_get_params",
    "sv_cost_model_set_params", "sv_cost_model_predict", "sv_cost_model_gradient",
    "sv_cost_model_train", "sv_cost_model_save", "sv_cost_model_load", "sv_set_cost_model",
    "sv_learned_plan", "sv_planner_judge", "sv_fault_inject", "sv_fault_raise_device_flag",
)
SV_FAULT_ALLOC, SV_FAULT_UPLOAD, SV_FAULT_LAUNCH = 0, 1, 2
SV_COST_FEATURES, SV_COST_HIDDEN, SV_COST_PARAMS = 52, 64, 7617
SV_KERNEL_PERGATE, SV_KERNEL_TILE, SV_KERNEL_REMAP, SV_KERNEL_FUSED, SV_KERNEL_L2BLOCK = 0, 1, 2, 3, 4


class LibraryMissing(RuntimeError):
    pass


class SvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libsv error {code}: {msg}")
        self.code = code


class sv_config(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tile_qubits", ctypes.c_int32),
                ("chunk_qubits", ctypes.c_int32), ("fuse_qubits", ctypes.c_int32),
                ("planner", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("l2_qubits", ctypes.c_int32), ("l2_chunk", ctypes.c_int32),
                ("batch_split", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7)]


class sv_stats(ctypes.Structure):
    _fields_ = [("gates", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("remaps", ctypes.c_int32), ("kernels", ctypes.c_int32),
                ("relabels", ctypes.c_int32), ("fused_blocks", ctypes.c_int32),
                ("sweep_bytes", ctypes.c_double), ("touched_bytes", ctypes.c_double),
                ("h2d_bytes", ctypes.c_double), ("planner", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("predicted_ms", ctypes.c_double),
                ("ctas_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class sv_launch_record(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pass_", ctypes.c_int32), ("n", ctypes.c_int32),
                ("k", ctypes.c_int32), ("nops", ctypes.c_int32), ("ngates", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("gate_kind", ctypes.c_int32),
                ("bytes", ctypes.c_double), ("ms", ctypes.c_double), ("feat", ctypes.c_uint64),
                ("c", ctypes.c_int32), ("stages", ctypes.c_int32), ("blocks", ctypes.c_int32),
                ("nins", ctypes.c_int32), ("nfactors", ctypes.c_int32),
                ("generated", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class sv_train_config(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("reserved", ctypes.c_int32 * 6)]


class sv_plan_choice(ctypes.Structure):
    _fields_ = [("chunk_qubits", ctypes.c_int32), ("paper_swap", ctypes.c_int32),
                ("passes", ctypes.c_int32), ("remaps", ctypes.c_int32),
                ("fused_passes", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("predicted_ms", ctypes.c_double), ("greedy_predicted_ms", ctypes.c_double),
                ("learned_ms", ctypes.c_double), ("greedy_ms", ctypes.c_double),
                ("verdict", ctypes.c_int32), ("early_diag", ctypes.c_int32),
                ("rule_kernels", ctypes.c_int32), ("narrow_first", ctypes.c_int32),
                ("rule_ms", ctypes.c_double), ("reserved", ctypes.c_int32 * 2)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class sv_batch_item(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("reserved", ctypes.c_int32), ("gates", ctypes.c_void_p),
                ("m", ctypes.c_size_t), ("qubit_mask", ctypes.c_uint64)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise LibraryMissing(f"{LIB_PATH} not built; run paper_2605_15098_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, u64, i32, sz, dp = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t,
                            ctypes.POINTER(ctypes.c_double))
    sig = {
        "sv_create": [i32, i32, ctypes.POINTER(vp)],
        "sv_create_on": [i32, i32, vp, sz, vp, ctypes.POINTER(vp)],
        "sv_destroy": [vp],
        "sv_reset": [vp],
        "sv_info": [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(vp)],
        "sv_qubit_map": [vp, vp],
        "sv_apply_circuit": [vp, vp, sz, ctypes.POINTER(sv_config)],
        "sv_last_stats": [vp, ctypes.POINTER(sv_stats)],
        "sv_last_measurements": [vp, vp, sz, ctypes.POINTER(sz)],
        "sv_fault_inject": [i32, i32],
        "sv_fault_raise_device_flag": [vp],
        "sv_probabilities": [vp, u64, vp],
        "sv_probabilities_device": [vp, u64, vp],
        "sv_argmax": [vp, u64, ctypes.POINTER(u64), dp],
        "sv_sample": [vp, u64, vp, sz, vp],
        "sv_copy_out": [vp, vp],
        "sv_copy_in": [vp, vp],
        "sv_profile": [vp, i32],
        "sv_marginal_noalloc": [vp, i32, i32, vp, u64, vp, vp],
        "sv_plan_export": [i32, i32, vp, vp, sz, ctypes.POINTER(sv_config), vp, sz,
                           ctypes.POINTER(sz)],
        "sv_batch_create": [vp, sz, ctypes.POINTER(sv_config), ctypes.POINTER(vp)],
        "sv_batch_run": [vp, vp, vp, dp],
        "sv_batch_info": [vp, ctypes.POINTER(sz), ctypes.POINTER(i32), dp],
        "sv_batch_destroy": [vp],
        "sv_apply_circuit_batch": [vp, sz, ctypes.POINTER(sv_config), vp, vp],
        "sv_autotune": [vp, vp, sz, ctypes.c_char_p, ctypes.POINTER(sv_config), dp],
        "sv_batch_autotune": [vp, sz, ctypes.POINTER(sv_config), dp],
        "sv_profile_read": [vp, vp, sz, ctypes.POINTER(sz)],
        "sv_cost_features": [ctypes.POINTER(sv_launch_record), vp],
        "sv_cost_model_create": [u64, ctypes.POINTER(vp)],
        "sv_cost_model_destroy": [vp],
        "sv_cost_model_get_params": [vp, vp],
        "sv_cost_model_set_params": [vp, vp],
        "sv_cost_model_predict": [vp, vp, sz, vp],
        "sv_cost_model_gradient": [vp, vp, vp, sz, vp, dp],
        "sv_cost_model_train": [vp, vp, vp, sz, ctypes.POINTER(sv_train_config), vp],
        "sv_cost_model_save": [vp, ctypes.c_char_p],
        "sv_cost_model_load": [ctypes.c_char_p, ctypes.POINTER(vp)],
        "sv_set_cost_model": [vp, vp],
        "sv_learned_plan": [vp, vp, sz, ctypes.POINTER(sv_config), ctypes.POINTER(sv_plan_choice)],
        "sv_planner_judge": [vp, vp, sz, ctypes.POINTER(sv_config),
                             ctypes.POINTER(sv_plan_choice)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = i32
    L.sv_last_error.restype = ctypes.c_char_p
    L.sv_version.restype = ctypes.c_char_p
    L.sv_launch_count.restype = ctypes.c_uint64
    L.sv_launch_count.argtypes = []
    _lib = L
    return L


def _check(code: int) -> None:
    if code != SV_OK:
        raise SvError(code, lib().sv_last_error().decode())


def sv_version() -> str:
    return lib().sv_version().decode()


def sv_last_error() -> str:
    return lib().sv_last_error().decode()


def make_config(mode=SV_MODE_AUTO, tile_qubits=0, chunk_qubits=0, fuse_qubits=0,
                planner=SV_PLANNER_GREEDY, flags=0, l2_qubits=0, l2_chunk=0, batch_split=0) -> sv_config:
    return sv_config(mode, tile_qubits, chunk_qubits, fuse_qubits, planner, flags, l2_qubits, l2_chunk,
                     batch_split)


# ---- handle-level functions (same names as the C ABI) ------------------------
def sv_create(n: int, dtype: int = SV_C64) -> int:
    h = ctypes.c_void_p()
    _check(lib().sv_create(n, dtype, ctypes.byref(h)))
    return h.value


def sv_create_on(n: int, dtype: int, dev_ptr: int, nbytes: int, stream: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().sv_create_on(n, dtype, ctypes.c_void_p(dev_ptr), nbytes,
                              ctypes.c_void_p(stream), ctypes.byref(h)))
    return h.value


def sv_destroy(h: int) -> None:
    _check(lib().sv_destroy(ctypes.c_void_p(h)))


def sv_reset(h: int) -> None:
    _check(lib().sv_reset(ctypes.c_void_p(h)))


def sv_info(h: int) -> tuple[int, int, int]:
    n, dt, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_void_p()
    _check(lib().sv_info(ctypes.c_void_p(h), ctypes.byref(n), ctypes.byref(dt), ctypes.byref(p)))
    return n.value, dt.value, p.value


def sv_qubit_map(h: int) -> list[int]:
    n = sv_info(h)[0]
    out = np.zeros(n, dtype=np.int32)
    _check(lib().sv_qubit_map(ctypes.c_void_p(h), out.ctypes.data))
    return out.tolist()


def sv_apply_circuit(h: int, gates: np.ndarray, cfg: sv_config | None = None) -> None:
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    _check(lib().sv_apply_circuit(ctypes.c_void_p(h), g.ctypes.data if g.size else None, g.size,
                                  ctypes.byref(cfg) if cfg is not None else None))


def sv_last_stats(h: int) -> dict:
    st = sv_stats()
    _check(lib().sv_last_stats(ctypes.c_void_p(h), ctypes.byref(st)))
    return st.as_dict()


def sv_last_measurements(h: int) -> np.ndarray:
    """Outcomes (uint8, list order) of the measurements of the last sv_apply_circuit."""
    cnt = ctypes.c_size_t()
    _check(lib().sv_last_measurements(ctypes.c_void_p(h), None, 0, ctypes.byref(cnt)))
    out = np.zeros(max(1, cnt.value), dtype=np.uint8)
    _check(lib().sv_last_measurements(ctypes.c_void_p(h), out.ctypes.data, cnt.value, ctypes.byref(cnt)))
    return out[:cnt.value].copy()


def sv_fault_inject(site: int, after: int = 0) -> None:
    _check(lib().sv_fault_inject(site, after))


def sv_fault_raise_device_flag(h: int) -> None:
    _check(lib().sv_fault_raise_device_flag(ctypes.c_void_p(h)))


def sv_probabilities(h: int, qubit_mask: int) -> np.ndarray:
    out = np.empty(1 << bin(qubit_mask).count("1"), dtype=np.float64)
    _check(lib().sv_probabilities(ctypes.c_void_p(h), qubit_mask, out.ctypes.data))
    return out


def sv_probabilities_device(h: int, qubit_mask: int, dev_ptr: int) -> None:
    _check(lib().sv_probabilities_device(ctypes.c_void_p(h), qubit_mask, ctypes.c_void_p(dev_ptr)))


def sv_marginal_noalloc(dev_amps: int, n: int, dtype: int, phys: list[int] | None,
                        qubit_mask: int, dev_out: int, stream: int = 0) -> None:
    """Allocation-free marginal of a caller-owned state buffer (see include/sv.h)."""
    pm = None
    if phys is not None:
        arr = np.ascontiguousarray(phys, dtype=np.int32)
        pm = arr.ctypes.data
    _check(lib().sv_marginal_noalloc(ctypes.c_void_p(dev_amps), n, dtype, pm, qubit_mask,
                                     ctypes.c_void_p(dev_out), ctypes.c_void_p(stream)))


def sv_argmax(h: int, qubit_mask: int) -> tuple[int, float]:
    idx, p = ctypes.c_uint64(), ctypes.c_double()
    _check(lib().sv_argmax(ctypes.c_void_p(h), qubit_mask, ctypes.byref(idx), ctypes.byref(p)))
    return idx.value, p.value


def sv_sample(h: int, qubit_mask: int, u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(u.size, dtype=np.uint64)
    _check(lib().sv_sample(ctypes.c_void_p(h), qubit_mask, u.ctypes.data if u.size else None,
                           u.size, out.ctypes.data if u.size else None))
    return out


def sv_copy_out(h: int) -> np.ndarray:
    n, dt, _ = sv_info(h)
    out = np.empty(1 << n, dtype=np.complex128 if dt == SV_C128 else np.complex64)
    _check(lib().sv_copy_out(ctypes.c_void_p(h), out.ctypes.data))
    return out


def sv_copy_in(h: int, amps: np.ndarray) -> None:
    n, dt, _ = sv_info(h)
    a = np.ascontiguousarray(amps, dtype=np.complex128 if dt == SV_C128 else np.complex64)
    assert a.size == 1 << n
    _check(lib().sv_copy_in(ctypes.c_void_p(h), a.ctypes.data))


def sv_profile(h: int, enable: bool) -> None:
    _check(lib().sv_profile(ctypes.c_void_p(h), 1 if enable else 0))


def sv_profile_read(h: int, cap: int = 1 << 16) -> list[dict]:
    buf = (sv_launch_record * cap)()
    cnt = ctypes.c_size_t()
    _check(lib().sv_profile_read(ctypes.c_void_p(h), buf, cap, ctypes.byref(cnt)))
    return [buf[i].as_dict() for i in range(min(cap, cnt.value))]


def sv_plan_export(n: int, dtype: int, gates: np.ndarray, cfg: sv_config | None = None,
                   phys: list[int] | None = None) -> dict:
    """The partitioned programme for a gate list, parsed from the library's JSON."""
    import json

    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    pm = np.ascontiguousarray(phys, dtype=np.int32) if phys is not None else None
    ln = ctypes.c_size_t()
    args = (n, dtype, pm.ctypes.data if pm is not None else None,
            g.ctypes.data if g.size else None, g.size,
            ctypes.byref(cfg) if cfg is not None else None)
    _check(lib().sv_plan_export(*args, None, 0, ctypes.byref(ln)))
    buf = ctypes.create_string_buffer(ln.value + 1)
    _check(lib().sv_plan_export(*args, buf, ln.value + 1, ctypes.byref(ln)))
    return json.loads(buf.value.decode())


def _batch_items(circuits):
    """circuits: list of (n, gate array, qubit_mask); returns (ctypes array, keep-alive list)."""
    keep = []
    arr = (sv_batch_item * len(circuits))()
    for i, (n, g, mask) in enumerate(circuits):
        g = np.ascontiguousarray(g, dtype=GATE_DTYPE)
        keep.append(g)
        arr[i] = sv_batch_item(n, 0, g.ctypes.data if g.size else None, g.size, mask)
    return arr, keep


def sv_batch_create(circuits, cfg: sv_config | None = None) -> int:
    arr, keep = _batch_items(circuits)
    b = ctypes.c_void_p()
    _check(lib().sv_batch_create(arr, len(circuits), ctypes.byref(cfg) if cfg is not None else None,
                                 ctypes.byref(b)))
    del keep
    return b.value


def sv_batch_run(b: int, count: int):
    idx = np.empty(count, dtype=np.uint64)
    p = np.empty(count, dtype=np.float64)
    ms = ctypes.c_double()
    _check(lib().sv_batch_run(ctypes.c_void_p(b), idx.ctypes.data, p.ctypes.data, ctypes.byref(ms)))
    return idx, p, ms.value


def sv_batch_info(b: int) -> dict:
    cnt, passes, sb = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_double()
    _check(lib().sv_batch_info(ctypes.c_void_p(b), ctypes.byref(cnt), ctypes.byref(passes),
                               ctypes.byref(sb)))
    return {"count": cnt.value, "passes": passes.value, "sweep_bytes": sb.value}


def sv_batch_destroy(b: int) -> None:
    _check(lib().sv_batch_destroy(ctypes.c_void_p(b)))


def sv_apply_circuit_batch(circuits, cfg: sv_config | None = None):
    arr, keep = _batch_items(circuits)
    idx = np.empty(len(circuits), dtype=np.uint64)
    p = np.empty(len(circuits), dtype=np.float64)
    _check(lib().sv_apply_circuit_batch(arr, len(circuits),
                                        ctypes.byref(cfg) if cfg is not None else None,
                                        idx.ctypes.data, p.ctypes.data))
    del keep
    return idx, p


def sv_autotune(h: int, gates: np.ndarray, cache_path: str | None = None):
    """Fastest measured configuration for this circuit: (sv_config, median ms)."""
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    best = sv_config()
    ms = ctypes.c_double()
    _check(lib().sv_autotune(ctypes.c_void_p(h), g.ctypes.data if g.size else None, g.size,
                             cache_path.encode() if cache_path else None, ctypes.byref(best),
                             ctypes.byref(ms)))
    return best, ms.value


def sv_batch_autotune(circuits):
    arr, keep = _batch_items(circuits)
    best = sv_config()
    ms = ctypes.c_double()
    _check(lib().sv_batch_autotune(arr, len(circuits), ctypes.byref(best), ctypes.byref(ms)))
    del keep
    return best, ms.value


def _f32(a, cols=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if cols is not None:
        assert a.ndim == 2 and a.shape[1] == cols, a.shape
    return a


def sv_cost_features(rec: dict) -> np.ndarray:
    """Feature vector of one launch record (dict as returned by sv_profile_read)."""
    r = sv_launch_record(**{f: rec.get(f, 0) for f, _ in sv_launch_record._fields_})
    out = np.zeros(SV_COST_FEATURES, dtype=np.float32)
    _check(lib().sv_cost_features(ctypes.byref(r), out.ctypes.data))
    return out


def cost_target(rec: dict) -> float:
    """What the cost model predicts for a record: ln(ms per algorithmic GB)."""
    return float(np.log(rec["ms"]) - np.log(rec["bytes"] * 1e-9))


def sv_cost_model_create(seed: int = 0) -> int:
    m = ctypes.c_void_p()
    _check(lib().sv_cost_model_create(seed, ctypes.byref(m)))
    return m.value


def sv_cost_model_destroy(m: int) -> None:
    _check(lib().sv_cost_model_destroy(ctypes.c_void_p(m)))


def sv_cost_model_get_params(m: int) -> np.ndarray:
    p = np.empty(SV_COST_PARAMS, dtype=np.float32)
    _check(lib().sv_cost_model_get_params(ctypes.c_void_p(m), p.ctypes.data))
    return p


def sv_cost_model_set_params(m: int, p) -> None:
    p = _f32(p)
    assert p.size == SV_COST_PARAMS
    _check(lib().sv_cost_model_set_params(ctypes.c_void_p(m), p.ctypes.data))


def sv_cost_model_predict(m: int, X) -> np.ndarray:
    X = _f32(X, SV_COST_FEATURES)
    y = np.empty(X.shape[0], dtype=np.float32)
    _check(lib().sv_cost_model_predict(ctypes.c_void_p(m), X.ctypes.data if X.size else None,
                                       X.shape[0], y.ctypes.data if y.size else None))
    return y


def sv_cost_model_gradient(m: int, X, T):
    X, T = _f32(X, SV_COST_FEATURES), _f32(T)
    g = np.empty(SV_COST_PARAMS, dtype=np.float32)
    loss = ctypes.c_double()
    _check(lib().sv_cost_model_gradient(ctypes.c_void_p(m), X.ctypes.data, T.ctypes.data,
                                        X.shape[0], g.ctypes.data, ctypes.byref(loss)))
    return g, loss.value


def sv_cost_model_train(m: int, X, T, epochs=100, batch=4096, lr=1e-3, seed=0,
                        beta1=0.9, beta2=0.999, eps=1e-8) -> np.ndarray:
    X, T = _f32(X, SV_COST_FEATURES), _f32(T)
    cfg = sv_train_config(epochs, batch, lr, beta1, beta2, eps, seed)
    losses = np.empty(epochs, dtype=np.float32)
    _check(lib().sv_cost_model_train(ctypes.c_void_p(m), X.ctypes.data, T.ctypes.data,
                                     X.shape[0], ctypes.byref(cfg), losses.ctypes.data))
    return losses


def sv_cost_model_save(m: int, path: str) -> None:
    _check(lib().sv_cost_model_save(ctypes.c_void_p(m), path.encode()))


def sv_cost_model_load(path: str) -> int:
    m = ctypes.c_void_p()
    _check(lib().sv_cost_model_load(path.encode(), ctypes.byref(m)))
    return m.value


def sv_set_cost_model(h: int, m: int | None) -> None:
    _check(lib().sv_set_cost_model(ctypes.c_void_p(h), ctypes.c_void_p(m) if m else None))


def sv_learned_plan(h: int, gates, cfg: sv_config | None = None) -> dict:
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    out = sv_plan_choice()
    _check(lib().sv_learned_plan(ctypes.c_void_p(h), g.ctypes.data if g.size else None, g.size,
                                 ctypes.byref(cfg) if cfg is not None else None,
                                 ctypes.byref(out)))
    return out.as_dict()


def sv_planner_judge(h: int, gates, cfg: sv_config | None = None) -> dict:
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    out = sv_plan_choice()
    _check(lib().sv_planner_judge(ctypes.c_void_p(h), g.ctypes.data if g.size else None, g.size,
                                  ctypes.byref(cfg) if cfg is not None else None,
                                  ctypes.byref(out)))
    return out.as_dict()


def config_dict(c: sv_config) -> dict:
    names = {SV_MODE_AUTO: "auto", SV_MODE_PERGATE: "per-gate", SV_MODE_PARTITIONED: "partitioned",
             SV_MODE_FUSED: "fused"}
    return {"mode": names.get(c.mode, c.mode), "tile_qubits": c.tile_qubits,
            "chunk_qubits": c.chunk_qubits, "planner": c.planner, "flags": c.flags,
            "l2_qubits": c.l2_qubits, "l2_chunk": c.l2_chunk, "batch_split": c.batch_split}


def sv_launch_count() -> int:
    return int(lib().sv_launch_count())


class State:
    """Owning wrapper: ``with State(n, SV_C128) as s: s.apply(gates)``."""

    def __init__(self, n: int, dtype: int = SV_C64, tensor=None, stream=None):
        self.n, self.dtype = n, dtype
        self._tensor = tensor
        if tensor is not None:  # adopt a torch CUDA buffer and stream
            nbytes = tensor.numel() * tensor.element_size()
            sptr = stream.cuda_stream if stream is not None else 0
            self.h = sv_create_on(n, dtype, tensor.data_ptr(), nbytes, sptr)
        else:
            self.h = sv_create(n, dtype)

    def apply(self, gates, cfg=None):
        sv_apply_circuit(self.h, gates, cfg)
        return self

    def stats(self):
        return sv_last_stats(self.h)

    def probabilities(self, mask):
        return sv_probabilities(self.h, mask)

    def measurements(self):
        return sv_last_measurements(self.h)

    def argmax(self, mask):
        return sv_argmax(self.h, mask)

    def sample(self, mask, u):
        return sv_sample(self.h, mask, u)

    def amplitudes(self):
        return sv_copy_out(self.h)

    def reset(self):
        sv_reset(self.h)

    def close(self):
        if self.h:
            sv_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
