"""Learned planner (GPU): the cost model only chooses among plans of the
same gate list, so amplitudes agree with the greedy plan's (within the
complex64 tolerance, reading A12) and outcomes are identical; sv_planner_judge
keeps whichever plan measured faster."""
import os

import numpy as np
import pytest

from gen import mixed_circuit
from paper_2605_15098_gb300 import circuits as C

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
MODEL = os.path.join(os.path.dirname(HERE), "paper_2605_15098_gb300", "data", "costmodel_gb300.svcm")


@pytest.fixture(scope="module")
def sv():
    import torch

    assert torch.cuda.is_available()
    from paper_2605_15098_gb300 import build as B
    B.build()
    from paper_2605_15098_gb300 import sv as mod
    return mod


def fidelity(a, b):
    return abs(np.vdot(a.astype(np.complex128), b.astype(np.complex128))) ** 2


@pytest.fixture(scope="module")
def model(sv):
    """The committed trained model when present, else a freshly initialised
    one (the planner must stay correct whatever the model predicts)."""
    m = sv.sv_cost_model_load(MODEL) if os.path.exists(MODEL) else sv.sv_cost_model_create(3)
    yield m
    sv.sv_cost_model_destroy(m)


@pytest.mark.parametrize("n,kind", [(18, "qpe"), (20, "random"), (19, "mixed")])
def test_learned_plan_parity(sv, orc, model, n, kind):
    if kind == "qpe":
        g, _, info = C.qpe(n, seed=n)
        mask = info["mask"]
    elif kind == "random":
        g, mask = C.random_circuit(n, 6, seed=n), (1 << n) - 1
    else:
        g, mask = mixed_circuit(n, 150, n, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 9, 10)), (1 << n) - 1
    ref = orc.run(n, g)
    with sv.State(n, sv.SV_C64) as s:
        sv.sv_set_cost_model(s.h, model)
        choice = sv.sv_learned_plan(s.h, g, sv.make_config(sv.SV_MODE_PARTITIONED))
        assert choice["candidates"] > 0 and choice["predicted_ms"] > 0
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED, planner=sv.SV_PLANNER_LEARNED))
        st = s.stats()
        assert st["planner"] == sv.SV_PLANNER_LEARNED
        assert st["predicted_ms"] == pytest.approx(choice["predicted_ms"])
        got = s.amplitudes()
        idx_l, _ = s.argmax(mask)
        s.reset()
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED))
        assert s.stats()["planner"] == sv.SV_PLANNER_GREEDY
        greedy = s.amplitudes()
        idx_g, _ = s.argmax(mask)
    assert 1.0 - fidelity(ref, got) <= 1e-6
    assert np.max(np.abs(got - ref)) <= 2e-5
    assert 1.0 - fidelity(greedy, got) <= 1e-6
    assert idx_l == idx_g


def test_learned_plan_c128_is_fp64_exact(sv, orc, model):
    n = 16
    g = mixed_circuit(n, 120, 77)
    ref = orc.run(n, g)
    with sv.State(n, sv.SV_C128) as s:
        sv.sv_set_cost_model(s.h, model)
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED, planner=sv.SV_PLANNER_LEARNED))
        assert s.stats()["planner"] == sv.SV_PLANNER_LEARNED
        got = s.amplitudes()
    assert np.max(np.abs(got - ref)) <= 1e-12


def test_no_model_falls_back_to_greedy(sv):
    n = 16
    g, _, _ = C.qpe(n)
    with sv.State(n, sv.SV_C64) as s:
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED, planner=sv.SV_PLANNER_LEARNED))
        assert s.stats()["planner"] == sv.SV_PLANNER_GREEDY
        with pytest.raises(sv.SvError) as e:
            sv.sv_learned_plan(s.h, g)
        assert e.value.code == sv.SV_ERR_STATE


def test_judge_keeps_the_faster_plan(sv, model):
    n = 24
    g = C.random_circuit(n, 8, seed=5)
    with sv.State(n, sv.SV_C64) as s:
        sv.sv_set_cost_model(s.h, model)
        res = sv.sv_planner_judge(s.h, g, sv.make_config(sv.SV_MODE_PARTITIONED))
        assert res["learned_ms"] > 0 and res["greedy_ms"] > 0
        want = sv.SV_PLANNER_LEARNED if res["learned_ms"] < res["greedy_ms"] else sv.SV_PLANNER_GREEDY
        assert res["verdict"] == want
        s.reset()
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED, planner=sv.SV_PLANNER_LEARNED))
        assert s.stats()["planner"] == want


def circuit_ms(sv, s, g, cfg, reps=3):
    """Median over `reps` runs of the summed launch times of one apply."""
    times = []
    for _ in range(reps + 1):
        sv.sv_profile(s.h, True)
        s.reset()
        s.apply(g, cfg)
        recs = sv.sv_profile_read(s.h)
        sv.sv_profile(s.h, False)
        times.append(sum(r["ms"] for r in recs))
    return sorted(times[1:])[reps // 2]


# held out from the training stream (random circuits of depth 2..21, layered
# mixtures of depth 2..17, QPE; n = 24..30): deeper random circuits
HELD_OUT = [("random n=26 depth 40", 26, 40, 91), ("random n=27 depth 32", 27, 32, 92)]


def test_learned_gain_is_measured(sv, model):
    """What the learned planner adds, by measurement: against the greedy plan
    of the default configuration (what sv_planner_judge compares), against
    the greedy plan at the chunk and tile width the learned plan chose (what
    the per-pass kernel choice, diagonal placement and remaps add), and
    against the autotuned greedy configuration.  The judge never keeps the
    slower plan, and on at least one held-out workload the learned plan is
    strictly faster than the default greedy plan."""
    rows = []
    for name, n, depth, seed in HELD_OUT:
        g = C.random_circuit(n, depth, seed)
        with sv.State(n, sv.SV_C64) as s:
            sv.sv_set_cost_model(s.h, model)
            res = sv.sv_planner_judge(s.h, g, sv.make_config(sv.SV_MODE_PARTITIONED))
            same = circuit_ms(sv, s, g, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=res["chunk_qubits"]))
            tuned, _ = sv.sv_autotune(s.h, g)
            tuned.planner = sv.SV_PLANNER_GREEDY
            tuned_ms = circuit_ms(sv, s, g, tuned)
        kept = min(res["learned_ms"], res["greedy_ms"])
        rows.append((name, res["learned_ms"], res["greedy_ms"], same, tuned_ms, res["verdict"]))
        print(f"{name}: learned {res['learned_ms']:.3f} ms, greedy default {res['greedy_ms']:.3f}, "
              f"greedy at c={res['chunk_qubits']} {same:.3f}, greedy autotuned {tuned_ms:.3f}, "
              f"rule kernels at the learned options {res['rule_ms']:.3f} (kept: {res['rule_kernels']}), "
              f"verdict {res['verdict']}")
        assert kept <= res["greedy_ms"]
        if res["rule_ms"] > 0:  # the judge kept the faster kernel choice for the learned options
            assert res["learned_ms"] <= res["rule_ms"]
        want = sv.SV_PLANNER_LEARNED if res["learned_ms"] < res["greedy_ms"] else sv.SV_PLANNER_GREEDY
        assert res["verdict"] == want
    assert any(r[1] < 0.97 * r[2] for r in rows), rows
