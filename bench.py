#!/usr/bin/env python3
"""Benchmark: QPE n=28 circuit time and achieved HBM GB/s, partitioned vs per-gate.

One step = one whole QPE circuit on n = 28 qubits (t = 24 counting qubits,
4 eigenstate qubits, 436 gates, seeded phases) through the C ABI: reset to
|0...0>, sv_apply_circuit (planning, programme upload, tile passes) and
sv_argmax of the counting register (FP64 marginal, read back to the host).
The state (2 GiB complex64) is far larger than the 126 MiB L2, so every pass
streams from HBM and no L2 flush is needed between steps.

Prints one JSON line (rank 0).  Under torchrun every rank runs its own
replica on its own GPU (the workload has no exchange step); ``value`` is the
circuits/s of all ranks over the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle instead (the baseline arm),
each step a bounded prefix of the same circuit, extrapolated by gate count.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QPE n=28 circuit time & achieved HBM GB/s: partitioned/fused vs per-gate"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=28)
    ap.add_argument("--dtype", choices=["c64", "c128"], default="c64")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--flags", type=int, default=0, help="SV_FLAG_* bits of the headline configuration "
                    "when it is given (--tile / --chunk / --no-autotune)")
    ap.add_argument("--no-pergate", action="store_true")
    ap.add_argument("--no-c128", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fused", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-paper", action="store_true")
    ap.add_argument("--no-other", action="store_true", help="skip the other tile kernel's timing")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-planner comparison")
    ap.add_argument("--no-sweep", action="store_true", help="skip the QPE n = 20..32 sweep")
    ap.add_argument("--no-random", action="store_true", help="skip the random-circuit n = 30, 32 timing")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the errors against the oracle")
    ap.add_argument("--no-l2", action="store_true", help="skip the L2 block group timing")
    ap.add_argument("--no-cpu-part", action="store_true", help="skip the partitioned CPU baseline")
    ap.add_argument("--l2-sweep", type=int, default=0, metavar="N",
                    help="only run QPE-N once per L2 block size (for an ncu capture) and print its launches")
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def sources_sha(paths) -> str:
    """SHA-256 (16 hex digits) of the concatenated files, in the given order."""
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel_src: str, workload: str):
    """Per-launch DRAM bytes from the committed ncu summary, if the sources
    the kernel and its programme are built from are unchanged since the
    capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d[workload]
        if ent.get("source") != kernel_src:
            return None
        if ent.get("sources_sha") != sources_sha(ent["sources"]):
            return None
        return float(ent["bytes_per_launch"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        loaded = [r for r in rows if (num(r[4]) or 0) >= 50] or rows
        sm = [num(r[1]) for r in loaded if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(rows[0][2]), "samples": len(rows), "samples_loaded": len(loaded),
                "power_w_max": max((num(r[3]) or 0) for r in rows), "reasons": reasons}


REF_STRIDE = 8  # strata of the circuit for the reference arm: one step = 1/8 of its gates


def oracle_strata(gates, stride: int):
    """Systematic sample of a circuit for timing the FP64 oracle: stratum s
    holds gates s, s + stride, s + 2 stride, ...  Consecutive strata cover every
    gate of the circuit exactly once after `stride` steps, so the time of a
    stratum is a sample of the whole circuit (every gate kind, every qubit), not
    of its prefix.  The oracle's cost per gate does not depend on the
    amplitudes, so the order in which strata are applied does not change it."""
    return [gates[s::stride] for s in range(stride)]


def oracle_time(n: int, gates, seconds: float):
    """Time the FP64 oracle on the circuit: the whole circuit once, in order,
    when n <= 28; above that, strata (oracle_strata, stride 8) until the time
    budget is spent.  Returns (seconds per circuit, gates applied, threads,
    description)."""
    from oracle import oracle

    oracle.build()
    threads = oracle.num_threads()
    psi = oracle.init(n)
    if n <= 28:
        t0 = time.perf_counter()
        oracle.apply(n, psi, gates)
        el = time.perf_counter() - t0
        del psi
        return el, len(gates), threads, (f"the whole {len(gates)}-gate circuit once, in order, "
                                         f"on the FP64 complex128 oracle")
    strata = oracle_strata(gates, REF_STRIDE)
    done, el = 0, 0.0
    for i in range(REF_STRIDE):
        t0 = time.perf_counter()
        oracle.apply(n, psi, strata[i])
        el += time.perf_counter() - t0
        done += len(strata[i])
        if el >= seconds:
            break
    del psi
    return el / done * len(gates), done, threads, (
        f"{done} of {len(gates)} gates (strata of every {REF_STRIDE}th gate) on the FP64 "
        f"complex128 oracle, scaled by gate count")


def run_reference(args, world, rank):
    """The oracle as the reference arm: each step applies one stratum of the
    QPE circuit (every 8th gate, a different offset each step), so 8
    consecutive steps apply the whole circuit once.  ms_per_step is the
    measured time of one such step; value converts it to circuits/s by the
    fraction of the circuit's gates the timed steps applied."""
    if rank != 0:
        return
    from paper_2605_15098_gb300 import circuits as C

    n = args.n
    gates, _, _ = C.qpe(n)
    from oracle import oracle

    oracle.build()
    threads = oracle.num_threads()
    psi = oracle.init(n)
    strata = oracle_strata(gates, REF_STRIDE)

    def step(i):
        sl = strata[i % REF_STRIDE]
        t0 = time.perf_counter()
        oracle.apply(n, psi, sl)
        return time.perf_counter() - t0, len(sl)

    for i in range(args.warmup):
        step(i)
    tot, ng = 0.0, 0
    for i in range(args.steps):
        dt, g = step(args.warmup + i)
        tot += dt
        ng += g
    circuits = ng / len(gates)
    value = circuits / tot
    sample = (f"each step one stratum of the QPE n={n} circuit (every {REF_STRIDE}th gate, offset "
              f"advancing by one per step, so {REF_STRIDE} steps apply all {len(gates)} gates); "
              f"{args.steps} timed steps applied {ng} gates = {circuits:.3f} circuits on the FP64 "
              f"complex128 oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": f"QPE-{n} circuits/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot / max(args.steps, 1) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded QPE circuit)",
        "config": {"workload": f"QPE n={n}, t={n - 4} counting + 4 eigenstate qubits, "
                               f"{len(gates)} gates", "n": n,
                   "circuit_fraction_per_step": 1.0 / REF_STRIDE},
        "cpu_baseline": {"value": value, "unit": f"QPE-{n} circuits/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": f"QPE-{n} circuits/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def replica_max(dist, x: float) -> float:
    """Max of a per-rank time over the replicas (each rank runs its own
    independent copy of the step: nothing else crosses ranks)."""
    if not dist:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: all replicas' steps over the slowest rank's time."""
    return world * steps / (max_ms / 1e3)


RANDOM_N = (30, 32)
RANDOM_PERGATE_C128_N = 30  # the per-gate complex128 baseline of the random circuits


def random_circuits(sv, C, stream, peak: float) -> dict:
    """Random circuits (layers of U3 on every qubit, then CZ on a random
    matching) at n = 30 and 32, depth 40, complex64: the register-stage passes
    (library defaults) and the fused tensor-core passes (SV_MODE_FUSED), one
    warm-up and one timed run each; at n = 30 also the per-gate kernel in
    complex128.  Every step ends with the argmax of the lowest 10 qubits, and
    all paths must agree on it."""
    import torch

    res = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for nn in RANDOM_N:
        g = C.random_circuit(nn, 40)
        buf = torch.empty(1 << nn, dtype=torch.complex64, device="cuda")
        h = sv.sv_create_on(nn, sv.SV_C64, buf.data_ptr(), (1 << nn) * 8, stream.cuda_stream)
        row = {"gates": int(len(g))}
        for mname, mode in (("partitioned", sv.SV_MODE_PARTITIONED), ("fused_tensor_cores", sv.SV_MODE_FUSED)):
            cfg = sv.make_config(mode)
            sv.sv_reset(h)
            sv.sv_apply_circuit(h, g, cfg)
            e0.record(stream)
            sv.sv_reset(h)
            sv.sv_apply_circuit(h, g, cfg)
            idx, p = sv.sv_argmax(h, (1 << 10) - 1)
            e1.record(stream)
            stream.synchronize()
            ms = e0.elapsed_time(e1)
            st = sv.sv_last_stats(h)
            gbs = st["sweep_bytes"] / (ms / 1e3) / 1e9
            row[mname] = {"circuit_ms": round(ms, 2), "passes": st["passes"],
                          "fused_blocks": st["fused_blocks"], "hbm_gbs_full_sweeps": round(gbs, 1),
                          "frac_of_measured_hbm": round(gbs / peak, 4), "argmax_low10": int(idx)}
        row["same_argmax"] = row["partitioned"]["argmax_low10"] == row["fused_tensor_cores"]["argmax_low10"]
        res[f"n{nn}_depth40"] = row
        sv.sv_destroy(h)
        del buf
        torch.cuda.empty_cache()
        if nn == RANDOM_PERGATE_C128_N:
            # the same circuit on the plain per-gate kernel in complex128 (FP64
            # arithmetic, one HBM sweep per gate): the baseline the complex64
            # tile paths are compared with; one run after a 64-gate warm-up
            buf = torch.empty(1 << nn, dtype=torch.complex128, device="cuda")
            h = sv.sv_create_on(nn, sv.SV_C128, buf.data_ptr(), (1 << nn) * 16, stream.cuda_stream)
            cfg = sv.make_config(sv.SV_MODE_PERGATE)
            sv.sv_apply_circuit(h, g[:64], cfg)
            sv.sv_reset(h)
            e0.record(stream)
            sv.sv_apply_circuit(h, g, cfg)
            idx, p = sv.sv_argmax(h, (1 << 10) - 1)
            e1.record(stream)
            stream.synchronize()
            ms = e0.elapsed_time(e1)
            st = sv.sv_last_stats(h)
            row["per_gate_c128"] = {"circuit_ms": round(ms, 2), "passes": st["passes"],
                                    "argmax_low10": int(idx),
                                    "same_argmax": int(idx) == row["partitioned"]["argmax_low10"]}
            for k in ("partitioned", "fused_tensor_cores"):
                row[f"{k}_speedup_over_per_gate_c128"] = round(ms / row[k]["circuit_ms"], 2)
            sv.sv_destroy(h)
            del buf
            torch.cuda.empty_cache()
    return res


L2_SWEEP = (0, 16, 18, 20, 22, 24)


def l2_sweep(n: int) -> None:
    """QPE-n, complex64, chunk 7: one run per L2 block size (0 = no groups,
    the one-level plan) after a reset, printing each run's launch records.
    Meant to run under ncu, one launch per kernel and block size."""
    from paper_2605_15098_gb300 import build as B
    from paper_2605_15098_gb300 import circuits as C
    B.build()
    from paper_2605_15098_gb300 import sv
    g, _, info = C.qpe(n)
    h = sv.sv_create(n, sv.SV_C64)
    rows = []
    for l2 in L2_SWEEP:
        flags = sv.SV_FLAG_L2_BLOCKS if l2 else 0
        cfg = sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=7, flags=flags, l2_qubits=l2, l2_chunk=2)
        sv.sv_profile(h, True)
        sv.sv_reset(h)
        sv.sv_apply_circuit(h, g, cfg)
        idx, _ = sv.sv_argmax(h, info["mask"])
        recs = sv.sv_profile_read(h)
        sv.sv_profile(h, False)
        rows.append({"l2_qubits": l2, "outcome_ok": idx == info["y"],
                     "launches": [{"kind": r["kind"], "k": r["k"], "passes": r["nops"],
                                   "ms": round(r["ms"], 4), "bytes": r["bytes"]} for r in recs]})
    sv.sv_destroy(h)
    print(json.dumps({"l2_sweep": f"QPE n={n} complex64 chunk 7", "rows": rows}))


def l2_blocks(sv, C, stream) -> dict:
    """Two-level blocking through L2 against the one-level plan: QPE-28
    (chunk 7) and a random circuit at n = 30, depth 40, complex64.  Each
    configuration: one warm-up, then the median of three (QPE) or one (random)
    timed run of reset + apply + argmax under CUDA events."""
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for name, nn, g, chunk, mask, reps in (
            ("qpe28", 28, C.qpe(28)[0], 7, C.qpe(28)[2]["mask"], 3),
            ("random_n30_depth40", 30, C.random_circuit(30, 40), 0, (1 << 10) - 1, 1)):
        buf = torch.empty(1 << nn, dtype=torch.complex64, device="cuda")
        h = sv.sv_create_on(nn, sv.SV_C64, buf.data_ptr(), (1 << nn) * 8, stream.cuda_stream)
        row = {}
        for label, l2, l2c in (("one_level", 0, 0), ("l2_20_chunk4", 20, 4), ("l2_22_chunk4", 22, 4)):
            cfg = sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=chunk,
                                 flags=sv.SV_FLAG_L2_BLOCKS if l2 else 0, l2_qubits=l2, l2_chunk=l2c)
            sv.sv_reset(h)
            sv.sv_apply_circuit(h, g, cfg)
            times, idxs = [], []
            for _ in range(reps):
                e0.record(stream)
                sv.sv_reset(h)
                sv.sv_apply_circuit(h, g, cfg)
                idx, _ = sv.sv_argmax(h, mask)
                e1.record(stream)
                stream.synchronize()
                times.append(e0.elapsed_time(e1))
                idxs.append(int(idx))
            st = sv.sv_last_stats(h)
            row[label] = {"circuit_ms": round(sorted(times)[len(times) // 2], 3), "kernels": st["kernels"],
                          "passes": st["passes"], "argmax": idxs[0]}
        row["same_argmax"] = len({v["argmax"] for v in row.values()}) == 1
        res[name] = row
        sv.sv_destroy(h)
        del buf
        torch.cuda.empty_cache()
    return res


SWEEP_N = (20, 24, 28, 30, 32)


def cpu_partitioned(C) -> dict:
    """The paper's CPU finding (partitioning does not pay on a CPU), on the
    host cores: QPE n = 22 (64 MiB in FP64), the whole circuit, with the
    oracle's plain Algorithm 1 (one sweep per gate) and with the partitioned
    CPU program at block sizes of 2^12 .. 2^20 amplitudes (cpupart.c).  Both
    use every host thread; the two states must agree within 1e-12."""
    from oracle import oracle as orc
    from paper_2605_15098_gb300 import cpupart

    n = 22
    g, _, _ = C.qpe(n)
    t0 = time.perf_counter()
    ref = orc.run(n, g)
    t_plain = time.perf_counter() - t0
    rows = {}
    for l in (12, 16, 18, 20):
        t0 = time.perf_counter()
        got, st = cpupart.run(n, g, l)
        dt_ = time.perf_counter() - t0
        rows[f"block_2^{l}"] = {"ms": round(dt_ * 1e3, 2), "flushes": st["passes"], "swaps": st["swaps"],
                                "max_abs_err_vs_oracle": float(np.max(np.abs(got - ref))),
                                "speedup_vs_plain": round(t_plain / dt_, 3)}
    return {"workload": f"QPE n={n} complex128 ({len(g)} gates), host CPU", "threads": cpupart.num_threads(),
            "plain_algorithm1_ms": round(t_plain * 1e3, 2), "partitioned": rows}


def qpe_sweep(sv, C, stream, peak: float, no_pergate: bool, cfgs: dict) -> dict:
    """QPE circuit time at n = 20 .. 32 in complex64 and complex128, on the
    partitioned path (the autotuner's measured choice; library defaults for
    complex128 above n = 28, where each candidate takes seconds) and the
    per-gate path.  HBM bytes follow the full-sweep convention
    2 x passes x 2^n x sizeof(amplitude) for the partitioned path; a per-gate
    row's fraction counts the bytes each gate touches (a CP moves a quarter of
    the state, a SWAP half), its full-sweep rate is printed beside it.  Each
    chosen configuration is stored in `cfgs` under (n, dtype)."""
    import torch

    res = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for nn in SWEEP_N:
        g, _, info = C.qpe(nn)
        for dname, dcode, tdt, ab in (("c64", sv.SV_C64, torch.complex64, 8),
                                      ("c128", sv.SV_C128, torch.complex128, 16)):
            buf = torch.empty(1 << nn, dtype=tdt, device="cuda")
            h = sv.sv_create_on(nn, dcode, buf.data_ptr(), (1 << nn) * ab, stream.cuda_stream)
            row = {}
            for mname, mode in (("partitioned", sv.SV_MODE_PARTITIONED), ("per_gate", sv.SV_MODE_PERGATE)):
                if mname == "per_gate" and no_pergate:
                    continue
                cfg, tuned = sv.make_config(mode), False
                if mname == "partitioned" and (dname == "c64" or nn <= 28):
                    cfg, _ = sv.sv_autotune(h, g)  # measured choice of tile, chunk and kernel
                    tuned = True
                    cfgs[(nn, dname)] = cfg
                reps = 10 if nn <= 24 else 3 if nn <= 28 else 1
                if mname == "partitioned" or nn <= 28:  # warm-up: plan, compile, upload, read-out
                    sv.sv_reset(h)
                    sv.sv_apply_circuit(h, g, cfg)
                    sv.sv_argmax(h, info["mask"])
                e0.record(stream)
                for _ in range(reps):
                    sv.sv_reset(h)
                    sv.sv_apply_circuit(h, g, cfg)
                    idx, p = sv.sv_argmax(h, info["mask"])
                e1.record(stream)
                stream.synchronize()
                ms = e0.elapsed_time(e1) / reps
                st = sv.sv_last_stats(h)
                gbs = st["sweep_bytes"] / (ms / 1e3) / 1e9
                row[mname] = {"circuit_ms": round(ms, 3), "passes": st["passes"],
                              "hbm_gbs_full_sweeps": round(gbs, 1),
                              "outcome_ok": bool(idx == info["y"] and abs(p - 1) < 1e-5),
                              "qpe_outcome_prob_err": float(abs(1.0 - p)),
                              "config": sv.config_dict(cfg) if tuned else "library defaults"}
                if mname == "per_gate":
                    tgbs = st["touched_bytes"] / (ms / 1e3) / 1e9
                    row[mname]["hbm_gbs_touched"] = round(tgbs, 1)
                    row[mname]["frac_of_measured_hbm"] = round(tgbs / peak, 4)
                    row[mname]["frac_basis"] = "bytes each gate touches"
                else:
                    row[mname]["frac_of_measured_hbm"] = round(gbs / peak, 4)
            if "per_gate" in row:
                row["speedup_partitioned"] = round(row["per_gate"]["circuit_ms"] /
                                                   row["partitioned"]["circuit_ms"], 2)
            res[f"n{nn}_{dname}"] = row
            sv.sv_destroy(h)
            del buf
            torch.cuda.empty_cache()
    return res


ACC_QPE_N = (20, 24)
ACC_RANDOM_N = (20, 22, 24, 26)
ACC_BATCH_SAMPLE = 32


def accuracy_rows(sv, C, sweep_cfgs, batch_res) -> dict:
    """Error of each result against the FP64 oracle, at the sizes the oracle
    finishes in seconds: QPE n = 20 and 24 (complex64 and complex128, each
    timed path), random circuits n = 20..26 at depth 40 (complex64,
    register-stage and fused tensor-core passes), and a sample of the batched
    instances.  Per row: max |amp - amp_oracle|, fidelity |<psi_oracle|psi>|^2
    and, for QPE, |p(y) - p_oracle(y)| of the expected outcome y.  Part of the
    CPU-baseline leg: the oracle runs on the host cores."""
    from oracle import oracle as orc

    def compare(ref, got):
        d = np.abs(got.astype(np.complex128) - ref)
        fid = abs(np.vdot(ref, got.astype(np.complex128))) ** 2
        return {"max_abs_err": float(d.max()), "fidelity": float(fid),
                "one_minus_fidelity": float(1.0 - fid)}

    rows = {}
    for nn in ACC_QPE_N:
        g, _, info = C.qpe(nn)
        ref = orc.run(nn, g)
        p_ref = float(orc.marginal(nn, ref, info["mask"])[info["y"]])
        for dname, dt, modes in (
                ("c64", sv.SV_C64, (("partitioned", sv.SV_MODE_PARTITIONED),
                                    ("fused_tensor_cores", sv.SV_MODE_FUSED),
                                    ("per_gate", sv.SV_MODE_PERGATE))),
                ("c128", sv.SV_C128, (("partitioned", sv.SV_MODE_PARTITIONED),
                                      ("per_gate", sv.SV_MODE_PERGATE)))):
            for mname, mode in modes:
                cfg = sweep_cfgs.get((nn, dname)) if mname == "partitioned" else None
                cfg = cfg or sv.make_config(mode)
                with sv.State(nn, dt) as s:
                    s.apply(g, cfg)
                    got = s.amplitudes()
                    idx, p = s.argmax(info["mask"])
                r = compare(ref, got)
                r["qpe_outcome_prob_err"] = float(abs(p - p_ref))
                r["outcome_ok"] = bool(idx == info["y"])
                r["config"] = sv.config_dict(cfg)
                rows[f"qpe_n{nn}_{dname}_{mname}"] = r
        del ref
    for nn in ACC_RANDOM_N:
        g = C.random_circuit(nn, 40)
        ref = orc.run(nn, g)
        for mname, mode in (("partitioned", sv.SV_MODE_PARTITIONED),
                            ("fused_tensor_cores", sv.SV_MODE_FUSED)):
            with sv.State(nn, sv.SV_C64) as s:
                s.apply(g, sv.make_config(mode))
                got = s.amplitudes()
            r = compare(ref, got)
            r["gates"] = int(len(g))
            rows[f"random_n{nn}_depth40_c64_{mname}"] = r
            del got
        del ref
    if batch_res is not None:
        work, bidx, bp = batch_res
        step = max(1, len(work) // ACC_BATCH_SAMPLE)
        errs, same, sampled = [], 0, 0
        for i in range(0, len(work), step):
            nn, g, mask, y = work[i]
            ref = orc.run(nn, g)
            pm = orc.marginal(nn, ref, mask)
            oi, op = orc.argmax(pm)
            same += int(int(bidx[i]) == oi)
            errs.append(abs(float(bp[i]) - op))
            sampled += 1
        rows["batched_sample"] = {
            "instances_sampled": sampled, "of": len(work),
            "outcomes_equal_oracle": same == sampled,
            "max_qpe_outcome_prob_err": float(max(errs)) if errs else None}
    return {"tolerance": {"c128_max_abs_err": 1e-12, "c64_max_abs_err": 2e-5,
                          "c64_min_fidelity": 1 - 1e-6},
            "rows": rows}


def run_ours(args, world, rank, local):
    import torch

    if world > 1:
        # the single-GPU side measurements (other kernel, per-gate, paper
        # scheme, complex128, sweep, batch) run at N = 1 only, so that an
        # N-GPU run holds its GPUs for the replicated step and e2e alone
        args.no_other = args.no_pergate = args.no_paper = True
        args.no_c128 = args.no_sweep = args.no_batch = args.no_random = args.no_l2 = True

    from paper_2605_15098_gb300 import build as B
    from paper_2605_15098_gb300 import circuits as C

    torch.cuda.set_device(local)
    B.build()
    from paper_2605_15098_gb300 import sv

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")

    def barrier():
        if dist:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return replica_max(dist, x)

    n = args.n
    dt = sv.SV_C64 if args.dtype == "c64" else sv.SV_C128
    amp_bytes = 8 if dt == sv.SV_C64 else 16
    gates, expected, info = C.qpe(n)
    mask = info["mask"]
    stream = torch.cuda.Stream()
    buf = torch.empty(1 << n, dtype=torch.complex64 if dt == sv.SV_C64 else torch.complex128,
                      device="cuda")
    state_bytes = (1 << n) * amp_bytes
    h = sv.sv_create_on(n, dt, buf.data_ptr(), state_bytes, stream.cuda_stream)
    # configuration chosen by the library's autotuner (mode x chunk width x tile width)
    if args.tile or args.chunk or args.flags or args.no_autotune:
        mode = sv.SV_MODE_FUSED if (dt == sv.SV_C64 and not args.no_fused) else sv.SV_MODE_PARTITIONED
        cfg = sv.make_config(mode, tile_qubits=args.tile, chunk_qubits=args.chunk, flags=args.flags)
        tuned = None
    else:
        cfg, tuned_ms = sv.sv_autotune(h, gates)
        mode = cfg.mode
        tuned = {"chosen": sv.config_dict(cfg), "median_ms": tuned_ms}

    def step(c=cfg):
        sv.sv_reset(h)
        sv.sv_apply_circuit(h, gates, c)
        return sv.sv_argmax(h, mask)

    for _ in range(max(args.warmup, 0)):
        idx, p = step()
    idx, p = step()
    ok = idx == info["y"] and abs(p - 1.0) < (1e-4 if dt == sv.SV_C64 else 1e-12)
    st = sv.sv_last_stats(h)

    # ---- timed region (device time, CUDA events on the library's stream) ----
    launches0 = sv.sv_launch_count()
    sv.sv_profile(h, True)
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    elapsed_ms = e0.elapsed_time(e1)
    launches = sv.sv_launch_count() - launches0
    recs = sv.sv_profile_read(h)
    sv.sv_profile(h, False)
    max_ms = max_over_ranks(elapsed_ms)
    value = replica_value(world, args.steps, max_ms)

    tile = [r for r in recs if r["kind"] in (sv.SV_KERNEL_TILE, sv.SV_KERNEL_FUSED)]
    kinds = [r["gate_kind"] for r in tile]
    if kinds.count(-3) * 2 >= len(kinds):
        kname, ksrc = "k_tile3 (fused tile pass, tcgen05 blocks)", "paper_2605_15098_gb300/csrc/tile3.cu"
    elif kinds.count(-2) * 2 >= len(kinds):
        kname, ksrc = "k_tile2 (register-stage tile pass)", "paper_2605_15098_gb300/csrc/tile2.cu"
    else:
        kname, ksrc = "k_tile (generic tile pass)", "paper_2605_15098_gb300/csrc/tile.cu"
    tile_ms = [r["ms"] for r in tile]
    tile_avg_ms = sum(tile_ms) / len(tile_ms) if tile_ms else float("nan")
    # algorithmic bytes of each launch (2 x state; a pass that generates the
    # initial basis state writes it only)
    launch_bytes = sum(r["bytes"] for r in tile) / len(tile) if tile else 2.0 * state_bytes
    achieved = sum(r["bytes"] for r in tile) / (sum(tile_ms) / 1e3) / 1e9 if tile_ms else None
    peak, peak_kind = peaks()
    kern_share = sum(tile_ms) / max(max_ms if world == 1 else elapsed_ms, 1e-9)
    circuit_ms = max_ms / args.steps
    alg_gbs = st["sweep_bytes"] / (circuit_ms / 1e3) / 1e9

    out = {
        "metric": METRIC, "value": value, "unit": f"QPE-{n} circuits/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": circuit_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if dt == sv.SV_C64 else "f64",
        "data": f"synthetic: seeded QPE circuit (splitmix64 seed {C.DEFAULT_SEED}, a_i={info['a']})",
        "config": {
            "workload": f"QPE n={n} ({n - 4} counting + 4 eigenstate qubits, {len(gates)} gates), "
                        f"{'complex64' if dt == sv.SV_C64 else 'complex128'}, {sv.config_dict(cfg)['mode']} tile passes",
            "n": n, "gates": len(gates), "mode": sv.config_dict(cfg)["mode"],
            "passes": st["passes"], "fused_blocks": st["fused_blocks"],
            "relabels": st["relabels"],
            "tile_qubits": cfg.tile_qubits or (13 if dt == sv.SV_C64 else 12),
            "chunk_qubits": cfg.chunk_qubits or (5 if dt == sv.SV_C64 else 4),
            "state_bytes": state_bytes,
            "l2": "state (2^n amplitudes) exceeds the 126 MiB L2; no flush between steps",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "step": "reset + sv_apply_circuit + sv_argmax(counting register)",
            "outcome_ok": bool(ok),
            "qpe_outcome_prob_err": float(abs(1.0 - p)),
        },
        "hbm_gbs_algorithmic": alg_gbs,
        "autotune": tuned,
        "roofline": {
            "kernel": kname, "bound": "hbm", "achieved": achieved, "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic_for(ksrc, f"qpe{n}_{args.dtype}"),
            "algorithmic_bytes_per_launch": launch_bytes, "launches": len(tile_ms),
            "avg_launch_ms": tile_avg_ms, "share_of_step_time": kern_share,
        },
        "gpu_launches": launches,
        "clocks": clk,
    }

    # ---- the other tile kernel on the same circuit (fused <-> CUDA-core) ----
    if dt == sv.SV_C64 and mode in (sv.SV_MODE_FUSED, sv.SV_MODE_PARTITIONED) and not args.no_other:
        other = sv.SV_MODE_PARTITIONED if mode == sv.SV_MODE_FUSED else sv.SV_MODE_FUSED
        pc = sv.make_config(other, chunk_qubits=cfg.chunk_qubits)
        step(pc)
        e0.record(stream)
        for _ in range(3):
            step(pc)
        e1.record(stream)
        stream.synchronize()
        pms = e0.elapsed_time(e1) / 3
        pst = sv.sv_last_stats(h)
        out["fused_tensor_cores" if other == sv.SV_MODE_FUSED else "partitioned_cuda_cores"] = {
            "circuit_ms": pms, "passes": pst["passes"],
            "hbm_gbs_full_sweeps": pst["sweep_bytes"] / (pms / 1e3) / 1e9}

    # ---- per-gate comparison (same circuit, one HBM sweep per gate) ----
    if not args.no_pergate:
        pg = sv.make_config(sv.SV_MODE_PERGATE)
        step(pg)
        k = 2
        e0.record(stream)
        for _ in range(k):
            step(pg)
        e1.record(stream)
        stream.synchronize()
        pst = sv.sv_last_stats(h)
        pms = e0.elapsed_time(e1) / k
        out["per_gate"] = {
            "circuit_ms": pms, "passes": pst["passes"],
            "hbm_gbs_full_sweeps": pst["sweep_bytes"] / (pms / 1e3) / 1e9,
            "hbm_gbs_touched": pst["touched_bytes"] / (pms / 1e3) / 1e9,
            "frac_touched_of_measured_hbm": pst["touched_bytes"] / (pms / 1e3) / 1e9 / peak,
            "speedup_partitioned_over_pergate": pms / circuit_ms,
        }
    # ---- the paper's own scheme: contiguous 2^13 blocks + explicit LRU remaps ----
    if not args.no_paper:
        pp = sv.make_config(sv.SV_MODE_PARTITIONED, flags=sv.SV_FLAG_PAPER_SWAP)
        pidx, pprob = step(pp)
        sv.sv_profile(h, True)
        e0.record(stream)
        for _ in range(2):
            step(pp)
        e1.record(stream)
        stream.synchronize()
        precs = sv.sv_profile_read(h)
        sv.sv_profile(h, False)
        pst = sv.sv_last_stats(h)
        pms = e0.elapsed_time(e1) / 2
        rm = [r for r in precs if r["kind"] == sv.SV_KERNEL_REMAP]
        rm_ms = sum(r["ms"] for r in rm) / len(rm) if rm else None
        rm_bytes = sum(r["bytes"] for r in rm) / len(rm) if rm else None
        out["paper_remap"] = {
            "scheme": "local = 13 lowest physical qubits (contiguous 64 KiB blocks); a gate on a "
                      "global target is preceded by a remap pass with the LRU local qubit",
            "circuit_ms": pms, "passes": pst["passes"], "remaps": pst["remaps"],
            "remap_avg_ms": rm_ms,
            "remap_gbs": (rm_bytes / (rm_ms / 1e3) / 1e9) if rm else None,
            "remap_share": (sum(r["ms"] for r in rm) / 2 / pms) if rm else None,
            "slowdown_vs_chosen": pms / circuit_ms,
            "outcome_ok": bool(pidx == info["y"] and abs(pprob - 1.0) < 1e-4)}
    sv.sv_destroy(h)
    del buf

    # ---- complex128 (FP64 arithmetic) at the same n, both paths ----
    if not args.no_c128 and dt == sv.SV_C64:
        buf2 = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
        h2 = sv.sv_create_on(n, sv.SV_C128, buf2.data_ptr(), (1 << n) * 16, stream.cuda_stream)
        res = {}
        for name, c2, reps in (("partitioned", sv.make_config(sv.SV_MODE_PARTITIONED), 3),
                               ("per_gate", sv.make_config(sv.SV_MODE_PERGATE), 1)):
            if name == "per_gate" and args.no_pergate:
                continue
            sv.sv_reset(h2)
            sv.sv_apply_circuit(h2, gates, c2)
            e0.record(stream)
            for _ in range(reps):
                sv.sv_reset(h2)
                sv.sv_apply_circuit(h2, gates, c2)
                i2, p2 = sv.sv_argmax(h2, mask)
            e1.record(stream)
            stream.synchronize()
            ms = e0.elapsed_time(e1) / reps
            s2 = sv.sv_last_stats(h2)
            res[name] = {"circuit_ms": ms, "passes": s2["passes"],
                         "hbm_gbs_full_sweeps": s2["sweep_bytes"] / (ms / 1e3) / 1e9,
                         "outcome_ok": bool(i2 == info["y"] and abs(p2 - 1) < 1e-12)}
        out["c128"] = res
        sv.sv_destroy(h2)
        del buf2

    # ---- random circuits, n = 30 and 32, depth 40, complex64: CUDA-core vs tensor-core passes ----
    if not args.no_random and dt == sv.SV_C64:
        out["random_circuits"] = random_circuits(sv, C, stream, peak)

    # ---- two-level blocking through L2 against the one-level plan ----
    if not args.no_l2 and dt == sv.SV_C64:
        out["l2_blocks"] = l2_blocks(sv, C, stream)

    sweep_cfgs, batch_res = {}, None
    # ---- QPE sweep: n = 20 .. 32, complex64 and complex128, partitioned vs per-gate ----
    if not args.no_sweep and dt == sv.SV_C64:
        out["qpe_sweep"] = qpe_sweep(sv, C, stream, peak, args.no_pergate, sweep_cfgs)

    # ---- batched QPE (4096 instances, n uniform in 10..20): one graph launch ----
    if not args.no_batch:
        work = C.qpe_batch(args.batch)
        items = [(nn, gg, mm) for nn, gg, mm, _ in work]
        bcfg, _ = sv.sv_batch_autotune(items)
        t0 = time.perf_counter()
        bh = sv.sv_batch_create(items, bcfg)
        t_create = time.perf_counter() - t0
        sv.sv_batch_run(bh, len(work))
        runs = [sv.sv_batch_run(bh, len(work)) for _ in range(3)]
        binfo = sv.sv_batch_info(bh)
        sv.sv_batch_destroy(bh)
        bidx = runs[-1][0]
        batch_res = (work, runs[-1][0], runs[-1][1])
        bms = statistics.median(r[2] for r in runs)
        out["batched"] = {
            "instances": len(work), "n_range": [10, 20], "launch_ms": bms,
            "instances_per_s": len(work) / (bms / 1e3), "passes": binfo["passes"],
            "l2_gbs_algorithmic": binfo["sweep_bytes"] / (bms / 1e3) / 1e9,
            "host_plan_s": t_create, "chunk_qubits": bcfg.chunk_qubits, "config": sv.config_dict(bcfg),
            "outcomes_ok": bool(all(int(bidx[i]) == w[3] for i, w in enumerate(work)))}

    # ---- learned planner vs greedy: random circuit and QPE, n = 30, complex64 ----
    if not args.no_learned and rank == 0:
        model_path = os.path.join(ROOT, "paper_2605_15098_gb300", "data", "costmodel_gb300.svcm")
        res = {}
        if os.path.exists(model_path):
            model = sv.sv_cost_model_load(model_path)
            hl = sv.sv_create(30, sv.SV_C64)
            sv.sv_set_cost_model(hl, model)
            greedy_cfg = sv.make_config(sv.SV_MODE_PARTITIONED)
            learned_cfg = sv.make_config(sv.SV_MODE_PARTITIONED, planner=sv.SV_PLANNER_LEARNED)
            for name, g_l, mask_l in (("random n=30 depth 40", C.random_circuit(30, 40), (1 << 12) - 1),
                                      ("QPE n=30", C.qpe(30)[0], (1 << 26) - 1)):
                t0 = time.perf_counter()
                r = sv.sv_planner_judge(hl, g_l, greedy_cfg)
                r["judge_s"] = time.perf_counter() - t0
                outs = []
                for c_l in (greedy_cfg, learned_cfg):
                    sv.sv_reset(hl)
                    sv.sv_apply_circuit(hl, g_l, c_l)
                    outs.append((sv.sv_argmax(hl, mask_l),
                                 sv.sv_probabilities(hl, (1 << 10) - 1)))
                r["same_argmax"] = bool(outs[0][0][0] == outs[1][0][0])
                r["marginal10_max_abs_diff"] = float(np.max(np.abs(outs[0][1] - outs[1][1])))
                r["gain_over_greedy"] = r["greedy_ms"] / min(r["greedy_ms"], r["learned_ms"])

                # the same step timed the same way for every configuration
                # (reset + apply + argmax, host clock, median of 3 after a
                # warm-up that also fills the programme cache): what the
                # network adds over the greedy rules at the chunk width it
                # chose, and, for QPE, over the autotuner's measured choice
                def wall_ms(c_w):
                    sv.sv_reset(hl)
                    sv.sv_apply_circuit(hl, g_l, c_w)
                    sv.sv_argmax(hl, 1)
                    ts = []
                    for _ in range(3):
                        t1 = time.perf_counter()
                        sv.sv_reset(hl)
                        sv.sv_apply_circuit(hl, g_l, c_w)
                        sv.sv_argmax(hl, 1)
                        ts.append(time.perf_counter() - t1)
                    return statistics.median(ts) * 1e3
                wall = {"greedy_default": wall_ms(greedy_cfg),
                        "greedy_at_learned_chunk": wall_ms(sv.make_config(
                            sv.SV_MODE_PARTITIONED, chunk_qubits=int(r["chunk_qubits"]))),
                        "learned": wall_ms(learned_cfg)}
                if name.startswith("QPE"):
                    tuned_cfg, _ = sv.sv_autotune(hl, g_l)
                    wall["autotuned"] = wall_ms(tuned_cfg)
                    r["autotuned_config"] = sv.config_dict(tuned_cfg)
                r["wall_ms"] = {k: round(v, 3) for k, v in wall.items()}
                for k in wall:
                    if k != "learned":
                        r[f"learned_gain_over_{k}"] = round(wall[k] / wall["learned"], 3)
                res[name] = r
            sv.sv_destroy(hl)
            sv.sv_cost_model_destroy(model)
        out["learned_planner"] = res or {"unavailable": "no trained cost model file"}

    # ---- end to end through the public API with host buffers ----
    # every step plans, compiles and uploads the circuit's programme again
    # (the handle's programme cache is bypassed), as for a circuit seen once
    he = sv.sv_create(n, dt)
    cfg_e2e = sv.make_config(cfg.mode, tile_qubits=cfg.tile_qubits, chunk_qubits=cfg.chunk_qubits,
                             fuse_qubits=cfg.fuse_qubits, planner=cfg.planner,
                             flags=cfg.flags | sv.SV_FLAG_NO_PLAN_CACHE)
    step_e2e = lambda: (sv.sv_reset(he), sv.sv_apply_circuit(he, gates, cfg_e2e),
                        sv.sv_argmax(he, mask))
    for _ in range(2):
        step_e2e()
    ke = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        step_e2e()
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    est = sv.sv_last_stats(he)
    sv.sv_destroy(he)
    out["e2e"] = {"value": world * ke / t_e2e, "unit": f"QPE-{n} circuits/s",
                  "h2d_bytes_per_step": int(est["h2d_bytes"]),
                  "d2h_bytes_per_step": 16,
                  "gate_list_bytes": int(gates.nbytes),
                  "step": "sv_create'd handle: reset + sv_apply_circuit(host gate list; planned, "
                          "compiled and its programme uploaded every step) + sv_argmax (host result)"}

    # ---- CPU-baseline leg (rank 0, N = 1): the FP64 oracle on the host cores,
    # timed on the same circuit, then the error of each small result against it ----
    if rank == 0 and world == 1 and not args.no_cpu:
        cs, done, threads, sample = oracle_time(n, gates, args.cpu_seconds)
        out["cpu_baseline"] = {
            "value": 1.0 / cs, "unit": f"QPE-{n} circuits/s", "cores": threads, "kind": "oracle",
            "sample": sample}
        if dt == sv.SV_C64 and not args.no_accuracy:
            out["accuracy"] = accuracy_rows(sv, C, sweep_cfgs, batch_res)
        if not args.no_cpu_part:
            out["cpu_partitioned"] = cpu_partitioned(C)
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.l2_sweep:
        if rank == 0:
            l2_sweep(args.l2_sweep)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
