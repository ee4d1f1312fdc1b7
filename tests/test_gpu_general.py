"""The general gate set on the GPU against the FP64 oracle: multi-controlled
U, two-qubit unitaries and collapsing measurements mixed with the paper's
gates, on the per-gate path and in partitioned plans (where each of them is a
step between tile passes).  complex128 within 1e-12, complex64 within the
complex64 bounds; measurement outcomes equal the oracle's (every u is chosen
half-way inside its outcome, see gen.general_circuit)."""
import numpy as np
import pytest

from gen import general_circuit
from paper_2605_15098_gb300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch

    assert torch.cuda.is_available()
    from paper_2605_15098_gb300 import build as B
    B.build()
    from paper_2605_15098_gb300 import sv as mod
    return mod


def oracle_run(orc, n, g):
    psi = orc.init(n)
    out = orc.apply_measured(n, psi, g)
    return psi, out


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n,seed", [(5, 1), (12, 2), (15, 3), (18, 4)])
def test_general_gates_match_oracle(sv, orc, n, seed, dt):
    g = general_circuit(n, 70, 10 * n + seed, orc)
    ref, outs = oracle_run(orc, n, g)
    modes = [sv.SV_MODE_PERGATE, sv.SV_MODE_PARTITIONED] + ([sv.SV_MODE_FUSED] if dt == 0 else [])
    for mode in modes:
        with sv.State(n, dt) as s:
            s.apply(g, sv.make_config(mode))
            got = s.amplitudes()
            meas = s.measurements()
        assert list(meas) == list(outs), (mode, meas, outs)
        if dt == sv.SV_C128:
            assert np.max(np.abs(got - ref)) <= 1e-12, mode
        else:
            assert np.max(np.abs(got - ref)) <= 2e-5, mode
            assert abs(np.vdot(ref, got.astype(np.complex128))) ** 2 >= 1 - 1e-6


def test_mcu_with_all_other_qubits_as_controls(sv, orc):
    """A controlled U whose controls are every other qubit acts on exactly
    one pair of amplitudes."""
    n = 16
    rng = np.random.default_rng(5)
    m = C.random_unitary(rng)
    g = C.gates([C.h(q) for q in range(n)] + [C.mcu([q for q in range(n) if q != 7], 7, m)])
    ref = orc.run(n, g)
    for mode in (sv.SV_MODE_PERGATE, sv.SV_MODE_PARTITIONED):
        with sv.State(n, sv.SV_C128) as s:
            s.apply(g, sv.make_config(mode))
            assert np.max(np.abs(s.amplitudes() - ref)) <= 1e-12


def test_measurements_collapse_and_repeat(sv, orc):
    """Measuring every qubit of a QPE register in turn reads its closed-form
    outcome bit by bit (p = 1 each), and the state becomes that basis state."""
    n = 14
    g, expected, info = C.qpe(n, seed=9)
    meas = C.gates(list(g) + [C.measure(q, 0.37) for q in range(n)])
    with sv.State(n, sv.SV_C64) as s:
        s.apply(meas, sv.make_config(sv.SV_MODE_PARTITIONED))
        bits = s.measurements()
        amps = s.amplitudes()
    assert sum(int(b) << q for q, b in enumerate(bits)) == expected
    assert abs(abs(amps[expected]) - 1.0) <= 1e-6


def test_general_gates_rejected_where_invalid(sv):
    n = 6
    bad = [
        C.gates(C.u2q(0, 1, np.eye(4))[:2]),            # rows missing
        C.gates([C.u2q(0, 1, np.eye(4))[1]]),            # a row alone
        C.gates([C.mcu([2, 3], 3, np.eye(2))]),          # target among the controls
        C.gates([C.measure(0, 1.5)]),                    # u outside [0, 1)
    ]
    for g in bad:
        with sv.State(n, sv.SV_C64) as s:
            with pytest.raises(sv.SvError) as e:
                s.apply(g)
            assert e.value.code == sv.SV_ERR_ARG
    with pytest.raises(sv.SvError) as e:
        sv.sv_apply_circuit_batch([(6, C.gates([C.h(0), C.measure(0, 0.5)]), 1)])
    assert e.value.code == sv.SV_ERR_UNSUPPORTED
