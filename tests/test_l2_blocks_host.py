"""Two-level blocking (Sec. III-B: the block sized by the last-level cache),
checked on the CPU.

The groups that sv_plan_export reports with SV_FLAG_L2_BLOCKS are checked for
their structure (consecutive register-stage passes whose tile qubits lie in
the block, every (block, pass) segment once, each pass of a block after the
block's previous pass in claim order), and the programme is executed segment
by segment in that claim order by the NumPy executor and compared with the
FP64 oracle.
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


def bits(qs):
    m = 0
    for q in qs:
        m |= 1 << q
    return m


def check_structure(plan, n):
    for g in plan["l2_groups"]:
        passes = plan["passes"][g["first"]:g["first"] + g["count"]]
        assert 2 <= g["count"] <= 4
        assert all(p["kernel"] == "t2" and p["k"] == 13 and p["ops"] for p in passes)
        assert all(not p["remap_before"] and not p.get("general") for p in passes[1:])
        union = 0
        for p in passes:
            union |= bits(p["slot_phys"])
        assert union & ~g["bmask"] == 0
        assert bin(g["bmask"]).count("1") == g["l"] == min(g["l"], n)
        nblocks = 1 << (n - g["l"])
        pos = {}
        for i, s in enumerate(g["segs"]):
            key = (s >> 3, s & 7)
            assert key not in pos
            pos[key] = i
        assert len(pos) == nblocks * g["count"]
        assert set(pos) == {(b, j) for b in range(nblocks) for j in range(g["count"])}
        for (b, j), i in pos.items():
            if j:
                assert pos[(b, j - 1)] < i  # claim order is a topological order
        # away from the ends a step holds every pass once: a block's passes
        # lie lag * count segments apart
        full = [pos[(b, 1)] - pos[(b, 0)] for b in range(nblocks)
                if g["lag"] * (g["count"] - 1) <= b < nblocks - g["lag"] * (g["count"] - 1)]
        assert all(d == g["lag"] * g["count"] + 1 for d in full)


def test_groups_of_qpe_plans(sv):
    """QPE plans at n = 20..30: groups are formed within the cap, and their
    structure holds for every block size of the sweep."""
    for n in (20, 24, 28, 30):
        g, _, _ = C.qpe(n, seed=n)
        counts = []
        for l2 in (0, 14, 16, 18, 20, 22):
            cfg = sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=7, flags=sv.SV_FLAG_L2_BLOCKS,
                                 l2_qubits=l2)
            plan = sv.sv_plan_export(n, sv.SV_C64, g, cfg)
            check_structure(plan, n)
            for gr in plan["l2_groups"]:
                assert gr["l"] == min(l2 or 20, n)
            counts.append(sum(gr["count"] for gr in plan["l2_groups"]))
        assert max(counts) >= 2  # some block size groups passes
        # no flag: no groups
        plan = sv.sv_plan_export(n, sv.SV_C64, g, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=7))
        assert "l2_groups" not in plan


def test_rejects_bad_block_size(sv):
    g, _, _ = C.qpe(16, seed=1)
    with pytest.raises(sv.SvError):
        sv.sv_plan_export(16, sv.SV_C64, g, sv.make_config(sv.SV_MODE_PARTITIONED, flags=sv.SV_FLAG_L2_BLOCKS,
                                                            l2_qubits=13))


@pytest.mark.parametrize("case", ["mixed16_l15", "random16_l16", "qpe18_l18_folded"])
def test_grouped_execution_matches_oracle(sv, orc, case):
    """The grouped programme, run (block, pass) segment by segment in claim
    order, equals the oracle; several blocks, and a first pass that
    generates the recorded product state."""
    basis, hq = 0, 0
    if case == "mixed16_l15":
        n, l2 = 16, 15
        g = mixed_circuit(n, 200, 5, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 9, 10))
        rest = g
    elif case == "random16_l16":
        n, l2 = 16, 16
        g = C.random_circuit(n, 6, 7)
        rest = g
    else:
        n, l2 = 18, 18
        g, _, _ = C.qpe(n, seed=3)
        basis, hq, rest = fold_leading(g)
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, flags=sv.SV_FLAG_L2_BLOCKS, l2_qubits=l2)
    plan = sv.sv_plan_export(n, sv.SV_C64, rest, cfg)
    check_structure(plan, n)
    assert plan["l2_groups"], case
    ref = orc.run(n, g)
    got = planemu.run_plan(n, plan, use_gen=True, basis=basis, hq=hq, l2_groups=True)
    assert float(np.max(np.abs(got - ref))) <= 2e-5
    if case == "mixed16_l15":
        assert any((1 << (n - gr["l"])) > 1 for gr in plan["l2_groups"])
