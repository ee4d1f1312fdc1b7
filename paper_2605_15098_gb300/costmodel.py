"""Training data and training of the planner's cost model, through the C ABI.

The library records every launch of a profiled ``sv_apply_circuit`` (kernel
family, tile layout, programme size, measured time).  This module runs
seeded synthetic circuits (n = 24..30) under many plan options, turns the
records into feature vectors with ``sv_cost_features`` and targets
ln(ms per algorithmic GB), and trains the MLP with the library's own
kernels.  Usage on a GPU:

    python -m paper_2605_15098_gb300.costmodel --out model.svcm --summary model.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import circuits as C
from . import sv

SEED = 2605150980


def _layered(n: int, depth: int, g: C.SplitMix64, mix: int) -> np.ndarray:
    """Random layered circuits with different gate mixtures (mix selects one)."""
    recs = []
    two_pi = 2.0 * np.pi
    for _ in range(depth):
        qs = list(range(n))
        for i in range(n - 1, 0, -1):
            j = g.next() % (i + 1)
            qs[i], qs[j] = qs[j], qs[i]
        width = 1 + g.next() % n
        for q in qs[:width]:
            if mix == 0:
                recs.append(C.u3(q, *(two_pi * g.uniform() for _ in range(3))))
            elif mix == 1:
                recs.append(C.h(q))
            else:
                recs.append(C.u3(q, two_pi * g.uniform(), 0.0, 0.0) if g.next() % 2 else C.h(q))
        pairs = 1 + g.next() % max(1, n // 2)
        for m in range(min(pairs, n // 2)):
            a, b = qs[2 * m], qs[2 * m + 1]
            k = g.next() % 3
            if k == 0:
                recs.append(C.cz(a, b))
            elif k == 1:
                recs.append(C.cpk(a, b, int(g.next() % 1024), 10))
            else:
                recs.append(C.swap(a, b))
    return C.gates(recs)


def workloads(seed: int, n_lo: int = 24, n_hi: int = 30):
    """Endless seeded stream of (name, n, gates): random circuits of the
    benchmark's construction, layered mixtures and QPE, n in [n_lo, n_hi]."""
    g = C.SplitMix64(seed)
    i = 0
    while True:
        n = n_lo + g.next() % (n_hi - n_lo + 1)
        kind = g.next() % 4
        if kind == 0:
            depth = 2 + g.next() % 20
            yield f"random{n}x{depth}", n, C.random_circuit(n, depth, seed + i)
        elif kind == 3:
            yield f"qpe{n}", n, C.qpe(n, seed + i)[0]
        else:
            depth = 2 + g.next() % 16
            yield f"layered{kind}_{n}x{depth}", n, _layered(n, depth, g, kind - 1)
        i += 1


CONFIGS = [("t2c%d" % c, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=c)) for c in (4, 5, 6, 7)]
CONFIGS += [("t3c%d" % c, sv.make_config(sv.SV_MODE_FUSED, chunk_qubits=c)) for c in (4, 5, 6, 7)]
CONFIGS += [("t2k14c%d" % c, sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=14, chunk_qubits=c))
            for c in (4, 7)]
CONFIGS += [("paper", sv.make_config(sv.SV_MODE_PARTITIONED, flags=sv.SV_FLAG_PAPER_SWAP)),
            ("paper_t3", sv.make_config(sv.SV_MODE_FUSED, flags=sv.SV_FLAG_PAPER_SWAP)),
            ("generic", sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=5,
                                       flags=sv.SV_FLAG_GENERIC_TILE))]
CONFIGS += [("t2c%dnarrow" % c, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=c,
                                               flags=sv.SV_FLAG_NARROW_FIRST)) for c in (6, 7, 8, 9)]
# complex128 runs on the generic tile kernel; sampled on smaller states
CONFIGS128 = [("c128k%dc%d" % (k, c), sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=k,
                                                     chunk_qubits=c))
              for k in (11, 12, 13) for c in (3, 4, 5)]
CONFIGS128 += [("c128paper", sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=12,
                                            flags=sv.SV_FLAG_PAPER_SWAP))]


def collect(target: int, seed: int = SEED, max_seconds: float = 600.0, n_lo: int = 24,
            n_hi: int = 30, log=print):
    """Profile seeded workloads until `target` launch records are collected.
    Returns X (N, F) float32, T (N,) float32 and the group (workload index)
    of each record."""
    X, T, grp = [], [], []
    handles = {}
    t0 = time.time()
    wi = 0
    stream = workloads(seed, n_lo, n_hi)
    try:
        while len(T) < target and time.time() - t0 < max_seconds:
            name, n, gates = next(stream)
            runs = [(sv.SV_C64, n, c) for c in CONFIGS]
            if wi % 5 == 0:  # a complex128 sample on 2^20..2^23 amplitudes
                n2 = 20 + n % 4
                g2 = gates[(gates["target"] < n2) & (gates["control"] < n2)]
                runs += [(sv.SV_C128, n2, c) for c in CONFIGS128]
            for dt, nn, (cname, cfg) in runs:
                g_run = gates if nn == n else g2
                if (nn, dt) not in handles:
                    handles[(nn, dt)] = sv.sv_create(nn, dt)
                h = handles[(nn, dt)]
                sv.sv_reset(h)
                sv.sv_profile(h, True)
                sv.sv_apply_circuit(h, g_run, cfg)
                recs = sv.sv_profile_read(h)
                sv.sv_profile(h, False)
                for r in recs:
                    if r["kind"] == sv.SV_KERNEL_PERGATE or r["ms"] <= 0:
                        continue
                    X.append(sv.sv_cost_features(r))
                    T.append(sv.cost_target(r))
                    grp.append(wi)
            wi += 1
            if wi % 20 == 0:
                log(f"  {wi} workloads, {len(T)} records, {time.time() - t0:.0f} s")
    finally:
        for h in handles.values():
            sv.sv_destroy(h)
    return (np.array(X, dtype=np.float32).reshape(-1, sv.SV_COST_FEATURES),
            np.array(T, dtype=np.float32), np.array(grp, dtype=np.int64))


def split(grp: np.ndarray, frac: float = 0.8):
    """Train / held-out masks by workload (every fifth workload is held out)."""
    test = (grp % 5) == 4 if frac == 0.8 else (grp % 100) >= int(frac * 100)
    return ~test, test


def train(X, T, grp, seed: int = SEED, epochs: int = 300, batch: int = 1024, lr: float = 2e-3):
    tr, te = split(grp)
    m = sv.sv_cost_model_create(seed)
    losses = sv.sv_cost_model_train(m, X[tr], T[tr], epochs=epochs, batch=batch, lr=lr, seed=seed)
    pred = sv.sv_cost_model_predict(m, X[te]) if te.any() else np.zeros(0)
    mse = float(np.mean((pred - T[te]) ** 2)) if te.any() else float("nan")
    base = float(np.mean((T[te] - T[tr].mean()) ** 2)) if te.any() else float("nan")
    summary = {
        "samples": int(len(T)), "train": int(tr.sum()), "held_out": int(te.sum()),
        "workloads": int(grp.max() + 1) if len(grp) else 0,
        "epochs": epochs, "batch": batch, "lr": lr, "seed": seed,
        "final_train_loss": float(losses[-1]), "held_out_mse": mse,
        "held_out_mse_of_mean_predictor": base,
        "held_out_rel_time_error_median": float(np.median(np.abs(np.exp(pred - T[te]) - 1.0)))
        if te.any() else float("nan"),
    }
    return m, summary, losses


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=50000)
    ap.add_argument("--seconds", type=float, default=900.0)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--seed", type=int, default=SEED)
    ap.add_argument("--out", required=True)
    ap.add_argument("--summary")
    ap.add_argument("--data", help="save the collected samples (.npz)")
    args = ap.parse_args()
    from . import build as B
    B.build()
    t0 = time.time()
    X, T, grp = collect(args.samples, args.seed, args.seconds)
    t_collect = time.time() - t0
    m, summary, losses = train(X, T, grp, args.seed, args.epochs)
    summary["collect_seconds"] = t_collect
    summary["train_seconds"] = time.time() - t0 - t_collect
    summary["loss_curve"] = [float(v) for v in losses[:: max(1, len(losses) // 30)]]
    sv.sv_cost_model_save(m, args.out)
    sv.sv_cost_model_destroy(m)
    if args.data:
        np.savez_compressed(args.data, X=X, T=T, grp=grp)
    if args.summary:
        with open(args.summary, "w") as f:
            json.dump(summary, f, indent=1)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
