"""Planner and stage compiler, checked on the CPU.

The programme the library would run (sv_plan_export, host only) is executed
by an independent NumPy executor of the documented step semantics and
compared with the FP64 oracle.  Register-stage programmes carry float32
gate matrices and 32-bit phases, hence the looser bound there.
"""
import numpy as np
import pytest

import planemu
from gen import fold_leading, mixed_circuit
from paper_2605_15098_gb300 import build as B
from paper_2605_15098_gb300 import circuits as C


@pytest.fixture(scope="module")
def sv():
    B.build()
    from paper_2605_15098_gb300 import sv as mod
    return mod


def check(sv, orc, n, g, cfg, dtype, tol):
    """Both variants of the first pass (generating |0...0> in registers, as
    the library does from a recorded basis state, and reading the state)
    against the oracle."""
    plan = sv.sv_plan_export(n, dtype, g, cfg)
    ref = orc.run(n, g)
    for use_gen in (True, False):
        got = planemu.run_plan(n, plan, use_gen=use_gen)
        err = float(np.max(np.abs(got - ref)))
        assert err <= tol, (use_gen, err)
    return plan


@pytest.mark.parametrize("n,seed", [(14, 1), (15, 2), (16, 3)])
def test_t2_mixed(sv, orc, n, seed):
    g = mixed_circuit(n, 150, seed)
    check(sv, orc, n, g, sv.make_config(sv.SV_MODE_PARTITIONED), sv.SV_C64, 2e-5)
    g = mixed_circuit(n, 150, seed, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 9, 10))  # no CU
    plan = check(sv, orc, n, g, sv.make_config(sv.SV_MODE_PARTITIONED), sv.SV_C64, 2e-5)
    assert all(p["kernel"] == "t2" for p in plan["passes"])


@pytest.mark.parametrize("n", [14, 15, 16])
def test_t2_qpe(sv, orc, n):
    g, expected, _ = C.qpe(n, seed=n)
    plan = check(sv, orc, n, g, sv.make_config(sv.SV_MODE_PARTITIONED), sv.SV_C64, 1e-5)
    assert all(p["kernel"] == "t2" for p in plan["passes"])
    # inverse-QFT steps on register bits run as phased butterflies
    assert planemu.T2_HPH in t2_ops(plan)


@pytest.mark.parametrize("chunk", [4, 5, 6, 7])
def test_t2_random_layers(sv, orc, chunk):
    n = 15
    g = C.random_circuit(n, 4, 99 + chunk)
    check(sv, orc, n, g, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=chunk), sv.SV_C64, 2e-5)


def t2_ops(plan):
    ops = []
    for p in plan["passes"]:
        if p.get("t2"):
            ops += [ins["op"] for ins in p["t2"]["ins"]]
    return ops


@pytest.mark.parametrize("n,depth", [(14, 3), (16, 4)])
def test_u3_split_real_rotations(sv, orc, n, depth):
    """In complex64 a U3 runs as P(phi) RY(theta) P(lambda): every
    non-diagonal step is a real rotation (a shear triple on a register bit,
    a real 2x2 on a lane bit), the phases join
    diagonal runs, the amplitudes still match the oracle and the pass gate
    counts still add up to the circuit's gates."""
    g = C.random_circuit(n, depth, 5 + n)
    plan = check(sv, orc, n, g, sv.make_config(sv.SV_MODE_PARTITIONED), sv.SV_C64, 2e-5)
    ops = t2_ops(plan)
    # register-bit rotations run as shear triples (planemu.T2_ROT), lane-bit ones as real 2x2
    assert ops.count(planemu.T2_RGATE) + ops.count(planemu.T2_ROT) == n * depth
    assert ops.count(planemu.T2_ROT) > 0
    assert planemu.T2_GATE not in ops
    assert sum(p["ngates"] for p in plan["passes"]) + plan["relabels"] == len(g)
    # complex128 keeps the general matrices
    plan128 = check(sv, orc, n, g, sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=10,
                                                  chunk_qubits=3), sv.SV_C128, 1e-12)
    assert sum(p["ngates"] for p in plan128["passes"]) + plan128["relabels"] == len(g)


def test_diagonal_runs_are_fewest():
    """Diagonal gates go to the fewest runs their windows allow: a layer of
    U3 on every qubit of one tile needs one run before the rotations (the
    lambda phases) and one after them (the phi phases), not one per qubit."""
    B.build()
    from paper_2605_15098_gb300 import sv as S
    def kinds(plan):
        return [op["type"] for p in plan["passes"] for op in p["ops"]]

    n = 12
    g = C.gates([C.u3(q, 0.3 + q, 1.1, 2.2) for q in range(n)])
    plan = S.sv_plan_export(n, S.SV_C64, g, S.make_config(S.SV_MODE_PARTITIONED))
    assert len(plan["passes"]) == 1
    assert kinds(plan).count(planemu.TOP_DIAG) == 2
    assert kinds(plan).count(planemu.TOP_GATE) == n
    # QFT: one run feeds each Hadamard after the first
    t = 10
    g = C.gates(C.qft(t))
    plan = S.sv_plan_export(t, S.SV_C64, g, S.make_config(S.SV_MODE_PARTITIONED))
    assert kinds(plan).count(planemu.TOP_DIAG) == t - 1


@pytest.mark.parametrize("n", [15, 17])
def test_diagonal_gates_move_to_their_successors_pass(sv, orc, n):
    """By default a diagonal gate runs in the pass of the first later gate it
    does not commute with (SV_FLAG_EARLY_DIAG keeps it in its first ready
    pass).  Both plans match the oracle; QPE's controlled powers then leave
    the early passes without diagonal runs and the whole plan has fewer."""
    g, _, _ = C.qpe(n, seed=n + 2)
    greedy = sv.SV_FLAG_GREEDY_ONLY  # the pass structure of the plain list scheduling
    late = check(sv, orc, n, g, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=5, flags=greedy),
                 sv.SV_C64, 1e-5)
    early = check(sv, orc, n, g, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=5,
                                                flags=greedy | sv.SV_FLAG_EARLY_DIAG), sv.SV_C64, 1e-5)
    runs = lambda plan: sum(1 for op in t2_ops(plan) if op in (planemu.T2_DIAG, planemu.T2_HPH))
    assert len(late["passes"]) == len(early["passes"]) > 1
    assert runs(late) < runs(early)
    first = [ins["op"] for ins in late["passes"][0]["t2"]["ins"]]
    assert planemu.T2_DIAG not in first and planemu.T2_HPH not in first
    g = C.random_circuit(n, 4, n)
    for flags in (0, sv.SV_FLAG_EARLY_DIAG):
        check(sv, orc, n, g, sv.make_config(sv.SV_MODE_PARTITIONED, flags=flags), sv.SV_C64, 2e-5)


@pytest.mark.parametrize("n,kind", [(16, "qpe"), (18, "qpe"), (16, "random"), (17, "mixed")])
def test_local_qubit_search(sv, orc, n, kind):
    """The default planner (local search of each pass's local qubits, the
    greedy plan kept when it has fewer passes) never needs more passes than
    the greedy list scheduling alone, and its plans match the oracle."""
    if kind == "qpe":
        g = C.qpe(n, seed=n)[0]
    elif kind == "random":
        g = C.random_circuit(n, 12, n)
    else:
        g = mixed_circuit(n, 200, n, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 9, 10))
    for c in (4, 5):
        searched = check(sv, orc, n, g, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=c),
                         sv.SV_C64, 2e-5)
        greedy = sv.sv_plan_export(n, sv.SV_C64, g, sv.make_config(
            sv.SV_MODE_PARTITIONED, chunk_qubits=c, flags=sv.SV_FLAG_GREEDY_ONLY))
        assert len(searched["passes"]) <= len(greedy["passes"])


def test_default_plan_never_has_more_passes_than_greedy(sv):
    """On seeded mixed circuits the default planner (search, greedy plan kept
    when shorter) never needs more passes than the greedy scheduling alone."""
    better = 0
    for seed in range(120):
        n = 9 + seed % 10
        kinds = (0, 1, 2, 3, 4, 5, 6, 7, 9, 10) if seed % 2 else (1, 2, 3, 4, 6)
        g = mixed_circuit(n, 40 + (seed * 7) % 200, seed, kinds=kinds)
        for c in (3, 4, 5):
            cfg = dict(tile_qubits=8, chunk_qubits=c)
            a = len(sv.sv_plan_export(n, sv.SV_C64, g, sv.make_config(sv.SV_MODE_PARTITIONED, **cfg))["passes"])
            b = len(sv.sv_plan_export(n, sv.SV_C64, g, sv.make_config(
                sv.SV_MODE_PARTITIONED, flags=sv.SV_FLAG_GREEDY_ONLY, **cfg))["passes"])
            assert a <= b, (seed, n, c, a, b)
            better += a < b
    assert better > 0


def test_search_shortens_qpe28():
    """QPE n=28: 3 passes with the search against 5 for the greedy scheduling (c = 7)."""
    B.build()
    from paper_2605_15098_gb300 import sv as S
    g, _, _ = C.qpe(28)
    n_s = len(S.sv_plan_export(28, S.SV_C64, g, S.make_config(S.SV_MODE_PARTITIONED, chunk_qubits=7))["passes"])
    n_g = len(S.sv_plan_export(28, S.SV_C64, g, S.make_config(
        S.SV_MODE_PARTITIONED, chunk_qubits=7, flags=S.SV_FLAG_GREEDY_ONLY))["passes"])
    assert n_s < n_g


def test_fusion_and_prefix_rules(sv, orc):
    """A diagonal run that also acts off the Hadamard's bit stays a separate
    run (no phased butterfly); a repeated Hadamard ends the generated prefix.
    Both programmes still match the oracle."""
    n = 14
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED)
    # the run before H(8) holds CP(8, 9) and CP(10, 11): not the identity where bit 8 is 0
    g = C.gates([C.h(q) for q in range(n)] + [C.cpk(8, 9, 1, 3), C.cpk(10, 11, 1, 4), C.h(8), C.h(10)])
    plan = check(sv, orc, n, g, cfg, sv.SV_C64, 1e-5)
    ops = t2_ops(plan)
    assert planemu.T2_HPH not in ops and planemu.T2_DIAG in ops
    # 14 leading Hadamards (13 on the first pass's local qubits), then H(3)
    # again: the generated prefix stops there, and the generated-state variant
    # of the first pass keeps exactly that one Hadamard step
    g = C.gates([C.h(q) for q in range(n)] + [C.h(3), C.cpk(3, 4, 1, 2)])
    plan = check(sv, orc, n, g, cfg, sv.SV_C64, 1e-5)
    gen = plan["passes"][0]["t2gen"]
    assert bin(gen["gen_hmask"]).count("1") == 13
    ops = [i["op"] for i in gen["ins"]]
    assert ops.count(planemu.T2_H) + ops.count(planemu.T2_HPH) == 1


@pytest.mark.parametrize("flags", [0, 1, 4, 5])
def test_generic_plan(sv, orc, flags):
    n = 13
    g = mixed_circuit(n, 120, 40 + flags)
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=8, chunk_qubits=3,
                         flags=flags | sv.SV_FLAG_GENERIC_TILE)
    plan = check(sv, orc, n, g, cfg, sv.SV_C128, 1e-12)
    assert all(p["kernel"] == "generic" for p in plan["passes"])


def test_pass_count_qpe28(sv):
    """QPE n=28 needs a handful of HBM sweeps instead of one per gate."""
    g, _, _ = C.qpe(28)
    plan = sv.sv_plan_export(28, sv.SV_C64, g, sv.make_config(sv.SV_MODE_PARTITIONED))
    assert len(plan["passes"]) <= 6
    assert sum(p["ngates"] for p in plan["passes"]) + plan["relabels"] == len(g)


@pytest.mark.parametrize("n,seed", [(14, 11), (16, 12)])
def test_fused_mixed(sv, orc, n, seed):
    g = mixed_circuit(n, 150, seed)
    plan = check(sv, orc, n, g, sv.make_config(sv.SV_MODE_FUSED), sv.SV_C64, 2e-5)
    assert any(p["kernel"] == "t3" for p in plan["passes"])


@pytest.mark.parametrize("n", [14, 16, 17])
def test_fused_qpe(sv, orc, n):
    g, _, _ = C.qpe(n, seed=n + 1)
    plan = check(sv, orc, n, g, sv.make_config(sv.SV_MODE_FUSED), sv.SV_C64, 1e-5)
    assert all(p["kernel"] == "t3" for p in plan["passes"])


@pytest.mark.parametrize("depth", [2, 5])
def test_fused_random_layers(sv, orc, depth):
    n = 15
    g = C.random_circuit(n, depth, 300 + depth)
    plan = check(sv, orc, n, g, sv.make_config(sv.SV_MODE_FUSED), sv.SV_C64, 2e-5)
    assert sum(len(p["t2"]["blocks"]) for p in plan["passes"] if p["kernel"] == "t3") >= 1


def lru_remap_pairs(n, k, g):
    """Remap pairs under Sec. III-B's rule, restated independently: the local
    qubits are the k lowest physical bits; a gate whose target is global
    exchanges it with the least recently used local bit (ties: the lowest)
    that the gate does not use; circuit SWAPs relabel the map."""
    phys = list(range(n))
    last = [-1] * k
    pairs, clock = [], 0
    for r in g:
        kind, t, c = int(r["kind"]), int(r["target"]), int(r["control"])
        if kind == C.SWAP:
            phys[t], phys[c] = phys[c], phys[t]
            continue
        ctrl = kind in (C.CP, C.CZ, C.CU, C.CPK)
        busy = {phys[t]} | ({phys[c]} if ctrl else set())
        if phys[t] >= k:
            v = min((p for p in range(k) if p not in busy), key=lambda p: (last[p], p))
            gq = phys[t]
            lq = phys.index(v)
            phys[lq], phys[t] = gq, v
            pairs.append((v, gq))
        last[phys[t]] = clock
        if ctrl and phys[c] < k:
            last[phys[c]] = clock
        clock += 1
    return pairs, phys


@pytest.mark.parametrize("flags", [0, 1, 4])
def test_paper_remap_plan_generic(sv, orc, flags):
    """Explicit remap passes (SV_FLAG_PAPER_SWAP): the block is the k lowest
    physical bits, every remap exchanges one local and one global bit, and
    the programme equals the oracle in FP64."""
    n, k = 13, 8
    g = mixed_circuit(n, 150, 70 + flags)
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=k,
                         flags=flags | sv.SV_FLAG_PAPER_SWAP | sv.SV_FLAG_GENERIC_TILE)
    plan = check(sv, orc, n, g, cfg, sv.SV_C128, 1e-12)
    assert plan["remaps"] > 0
    assert plan["remaps"] == sum(len(p["remap_before"]) for p in plan["passes"])
    for p in plan["passes"]:
        assert p["slot_phys"] == list(range(k)) and p["c"] == k
        for a, b in p["remap_before"]:
            assert a < k <= b
        bits = [b for pr in p["remap_before"] for b in pr]
        assert len(bits) == len(set(bits))


def test_paper_remap_plan_register_stage(sv, orc):
    n = 15
    g, _, _ = C.qpe(n, seed=4)
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, flags=sv.SV_FLAG_PAPER_SWAP)
    plan = check(sv, orc, n, g, cfg, sv.SV_C64, 1e-5)
    assert plan["remaps"] > 0
    assert any(p["kernel"] == "t2" for p in plan["passes"])


@pytest.mark.parametrize("n,seed", [(16, 1), (24, 2)])
def test_paper_remaps_follow_lru(sv, n, seed):
    g, _, _ = C.qpe(n, seed=seed)
    g2 = mixed_circuit(n, 200, seed, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10))
    for gates in (g, g2):
        for k in (8, 11, 13):
            cfg = sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=k, flags=sv.SV_FLAG_PAPER_SWAP)
            plan = sv.sv_plan_export(n, sv.SV_C128 if k != 13 else sv.SV_C64, gates, cfg)
            pairs, phys = lru_remap_pairs(n, k, gates)
            assert [tuple(pr) for p in plan["passes"] for pr in p["remap_before"]] == pairs
            assert plan["phys"] == phys


def test_paper_swap_count_falls_with_block_size(sv):
    """The trade-off the paper measures: fewer remaps as the block grows, and
    many more state sweeps than the gathering planner needs."""
    n = 24
    g, _, _ = C.qpe(n)
    counts = []
    for k in range(8, 15):
        cfg = sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=k, flags=sv.SV_FLAG_PAPER_SWAP)
        counts.append(sv.sv_plan_export(n, sv.SV_C64, g, cfg)["remaps"])
    assert all(a >= b for a, b in zip(counts, counts[1:])) and counts[0] > counts[-1]
    gather = sv.sv_plan_export(n, sv.SV_C64, g, sv.make_config(sv.SV_MODE_PARTITIONED))
    assert len(gather["passes"]) * 4 < counts[-1]


@pytest.mark.parametrize("n,seed,tile,chunk", [(16, 5, 0, 5), (16, 5, 14, 7), (18, 1, 0, 7), (20, 3, 0, 4)])
def test_generated_product_state(sv, orc, n, seed, tile, chunk):
    """After the fold of leading X and H gates, the first pass generates
    H^{hq}|b> (Hadamards on global qubits included) and its programme may
    still begin with Hadamards on qubits that carry a folded one (QPE's first
    inverse-QFT step after zero-phase controlled phases): those cancel.  The
    generated-state variant, emulated from the recorded state, matches the
    oracle on the whole list."""
    g, _, _ = C.qpe(n, seed=seed)
    mixed = C.gates([C.h(q) for q in range(0, n, 2)] + [C.x(1), C.h(1), C.x(3)] +
                    list(mixed_circuit(n, 40, seed, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 9, 10))) +
                    [C.h(0), C.h(2)])
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=tile, chunk_qubits=chunk)
    for circ in (g, mixed):
        ref = orc.run(n, circ)
        basis, hq, rest = fold_leading(circ)
        assert hq and len(rest) < len(circ)
        plan = sv.sv_plan_export(n, sv.SV_C64, rest, cfg)
        assert "t2gen" in plan["passes"][0]
        got = planemu.run_plan(n, plan, use_gen=True, basis=basis, hq=hq)
        assert float(np.max(np.abs(got - ref))) <= 2e-5


@pytest.mark.parametrize("n,seed", [(14, 3), (16, 4)])
def test_general_gates_split_the_plan(sv, orc, n, seed):
    """MCU, U2Q and MEASURE become steps of their own between tile passes
    (run on the per-gate path); the plan around them still matches the
    oracle, measurement outcomes included."""
    from gen import general_circuit
    g = general_circuit(n, 60, seed, orc)
    kinds = set(int(k) for k in g["kind"])
    assert {C.MCU, C.U2Q, C.MEASURE} <= kinds
    plan = sv.sv_plan_export(n, sv.SV_C64, g, sv.make_config(sv.SV_MODE_PARTITIONED))
    steps = [p for p in plan["passes"] if p.get("general")]
    assert len(steps) == sum(1 for k in g["kind"] if int(k) in (C.MCU, C.U2Q, C.MEASURE))
    assert sum(p["ngates"] for p in plan["passes"]) + plan["relabels"] == len(g)
    psi = orc.init(n)
    orc.apply_measured(n, psi, g)
    got = planemu.run_plan(n, plan, use_gen=False)
    assert float(np.max(np.abs(got - psi))) <= 2e-5


@pytest.mark.parametrize("n,kind", [(16, "qpe"), (15, "mixed"), (15, "random")])
def test_phased_butterfly_fields_match_their_run(sv, n, kind):
    """A phased butterfly step names its run's table record, static row and
    slot itself (read by the complex64 and complex128 kernels instead of the
    run's factor records); they must be exactly those of the records the step
    also keeps (read by the emulator above)."""
    K_DIRECT, FAC_TABLE = 0x40, 1 << 28
    K_SHARED = 0x41  # the same, with shared twiddles (tileprog.h: kT2HphShared)
    g = (C.qpe(n, seed=n)[0] if kind == "qpe" else mixed_circuit(n, 150, 7) if kind == "mixed"
         else C.random_circuit(n, 4, 5))
    found = 0
    for dtype in (sv.SV_C64, sv.SV_C128):
        plan = sv.sv_plan_export(n, dtype, g, sv.make_config(sv.SV_MODE_PARTITIONED))
        for p in plan["passes"]:
            for t2 in [p[k] for k in ("t2", "t2gen", "t2d", "t2dgen") if k in p]:
                fac = t2["fac2"]
                for ins in t2["ins"]:
                    if ins["op"] != planemu.T2_HPH:
                        continue
                    found += 1
                    trec, row, slot = -1, -1, -1
                    for f in fac[ins["e0"]:ins["e1"]]:
                        if f["w0"] & FAC_TABLE:
                            trec = f["row"]
                        else:
                            row, slot = f["row"], f["slot"]
                    assert ins["ccls"] in (K_DIRECT, K_SHARED)
                    assert (ins["aux"] & 0xffff) - 1 == trec
                    assert ((ins["aux"] >> 16) & 0xffff) - 1 == row
                    assert ins["cidx"] == slot
    if kind == "qpe":
        assert found > 0


@pytest.mark.parametrize("n,kind,chunk", [(16, "qpe", 7), (17, "qpe", 6), (15, "mixed", 7), (16, "random", 6)])
def test_narrow_first_pass(sv, orc, n, kind, chunk):
    """SV_FLAG_NARROW_FIRST: the list's first pass gathers 16-amplitude chunks
    (4 chunk qubits), the others the configured width; the programme matches
    the oracle whether the first pass generates |0...0> or reads it."""
    g = (C.qpe(n, seed=n)[0] if kind == "qpe" else mixed_circuit(n, 150, 11) if kind == "mixed"
         else C.random_circuit(n, 4, 21))
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=chunk, flags=sv.SV_FLAG_NARROW_FIRST)
    plan = check(sv, orc, n, g, cfg, sv.SV_C64, 2e-5)
    cs = [p["c"] for p in plan["passes"] if "c" in p]
    assert cs[0] == 4 and all(c == chunk for c in cs[1:]), cs
    # the first pass's tile holds its 4 chunk qubits and k - 4 free ones
    assert plan["passes"][0]["slot_phys"][:4] == [0, 1, 2, 3]


def test_programme_independent_of_earlier_compilations(sv):
    """The compiler keeps a per-thread memo of FP32 phase exponentials.  A
    programme must not depend on what was compiled before it: the same
    circuit exported before and after others (continuous rotation angles
    and dyadic QPE phases, both dtypes) gives the same bytes."""
    import json

    n = 16
    a = C.qpe(n, seed=4)[0]
    others = [C.random_circuit(n, 12, seed=s) for s in (1, 2, 3)] + [C.qpe(n, seed=9)[0]]
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=5)
    first = json.dumps(sv.sv_plan_export(n, sv.SV_C64, a, cfg), sort_keys=True)
    for g in others:
        sv.sv_plan_export(n, sv.SV_C64, g, cfg)
        sv.sv_plan_export(n, sv.SV_C128, g, cfg)
    again = json.dumps(sv.sv_plan_export(n, sv.SV_C64, a, cfg), sort_keys=True)
    assert first == again


@pytest.mark.parametrize("kind", ["qpe", "random"])
def test_shared_twiddle_flag_holds(sv, kind):
    """A phased butterfly marked kT2HphShared (control-class 0x41) on register
    bit j has a table whose packed entries q1 (bit j - 1 of q1 set) depend only
    on the bits of q1 below j - 1: the kernel then forms the 2^(j-1) products
    of the thread factor and the table once.  Checked entry by entry on the
    exported FP32 tables; QPE's inverse QFT has such steps."""
    if kind == "qpe":
        n, g = 24, fold_leading(C.qpe(24, seed=2)[0])[2]
    else:
        n, g = 18, C.random_circuit(18, 10, seed=3)
    flagged = 0
    for chunk in (5, 7, 9):
        cfg = sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=chunk, flags=sv.SV_FLAG_NARROW_FIRST)
        plan = sv.sv_plan_export(n, sv.SV_C64, g, cfg)
        for p in plan["passes"]:
            for t2 in (p.get("t2"), p.get("t2gen")):
                if not t2:
                    continue
                mats = np.array(t2["mats"], dtype=np.float32).reshape(-1)
                for ins in t2["ins"]:
                    if ins["op"] != 9 or ins["ccls"] != 0x41:
                        continue
                    flagged += 1
                    j, trec = ins["idx"], (ins["aux"] & 0xFFFF) - 1
                    assert 1 <= j <= 3 and trec >= 0
                    entry = lambda q: mats[8 * trec + 4 * q:8 * trec + 4 * q + 4]
                    hb = 1 << (j - 1)
                    for q1 in range(16):
                        if q1 & hb:
                            assert np.array_equal(entry(q1), entry((q1 & (hb - 1)) | hb))
    if kind == "qpe":
        assert flagged > 0


def test_shared_twiddle_flag_holds_c128(sv):
    """The complex128 form: a step marked 0x41 on register bit j = 0..3 has a
    32-entry FP64 table whose entries x (bit j of x set) depend only on the
    bits of x below j.  QPE's complex128 programmes run on the FP64
    register-stage kernel (exported as t2d) and have such steps."""
    n, g = 22, fold_leading(C.qpe(22, seed=5)[0])[2]
    flagged = 0
    for chunk in (5, 6, 7):
        cfg = sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=13, chunk_qubits=chunk)
        plan = sv.sv_plan_export(n, sv.SV_C128, g, cfg)
        assert all(p["kernel"] == "t2d" for p in plan["passes"] if p["ops"])
        for p in plan["passes"]:
            for t2 in (p.get("t2d"), p.get("t2dgen")):
                if not t2:
                    continue
                mats = np.array(t2["mats"], dtype=np.float64).reshape(-1)
                for ins in t2["ins"]:
                    if ins["op"] != planemu.T2_HPH or ins["ccls"] != 0x41:
                        continue
                    flagged += 1
                    j, trec = ins["idx"], (ins["aux"] & 0xFFFF) - 1
                    assert 0 <= j <= 3 and trec >= 0
                    entry = lambda x: mats[8 * trec + 2 * x:8 * trec + 2 * x + 2]
                    hb = 1 << j
                    for x in range(32):
                        if x & hb:
                            assert np.array_equal(entry(x), entry((x & (hb - 1)) | hb))
    assert flagged > 0
