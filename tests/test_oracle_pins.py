"""The FP64 oracle against facts fixed outside it (CPU only).

Every check here derives its expected value from the paper (worked examples
in tests/golden/), from a closed form, from an identity, or from a brute-force
Kronecker product; none re-runs the oracle's own formula.  The last test
builds the oracle with planted mistakes and requires each to fail a pin.
"""
import os

import numpy as np
import pytest

import pins
from paper_2605_15098_gb300 import circuits as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _runner(orc, mutation=0):
    def run(n, g):
        return orc.run(n, g, mutation)
    return run


def _fixture(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.mark.parametrize("pin", pins.ALL_PINS)
def test_pin(orc, pin):
    bad = getattr(pins, pin)(_runner(orc))
    assert not bad, bad


def test_paper_qpe_golden(orc):
    rows = [(int(r[0]), r[1], float(r[2])) for r in _fixture("paper_qpe.txt")]
    bad = pins.pin_paper_qpe(_runner(orc), rows)
    assert not bad, bad


def test_alg1_pairs_golden(orc):
    """Fig. 1: X on qubit 1 of 3 qubits maps each basis state to its Alg. 1 partner."""
    for row in _fixture("alg1_pairs.txt"):
        n, t = int(row[0]), int(row[1])
        pairs = [tuple(int(v) for v in p.split(",")) for p in row[2:]]
        for a, b in pairs:
            for src, dst in ((a, b), (b, a)):
                recs = [C.x(q) for q in range(n) if (src >> q) & 1] + [C.x(t)]
                psi = orc.run(n, C.gates(recs))
                assert abs(psi[dst] - 1.0) < 1e-15, (src, dst)
        covered = sorted(v for p in pairs for v in p)
        assert covered == list(range(1 << n))


def test_fig2_block_classes(orc):
    """Fig. 2: with blocks of 2^l amplitudes, a gate on qubit q pairs within a
    block iff q < l.  Checked by observing which amplitudes X(q) exchanges."""
    for row in _fixture("fig2_blocks.txt"):
        n, l, q, cls = int(row[0]), int(row[1]), int(row[2]), row[3]
        pairs = [tuple(int(v) for v in p.split(",")) for p in row[4:]]
        for a, b in pairs:
            recs = [C.x(k) for k in range(n) if (a >> k) & 1] + [C.x(q)]
            psi = orc.run(n, C.gates(recs))
            assert abs(psi[b] - 1.0) < 1e-15
            same_block = (a >> l) == (b >> l)
            assert same_block == (cls == "local")


def test_controlled_rule(orc):
    """Sec. III-A: the inner iteration runs only when the control bit is 1."""
    n = 3
    for basis in range(1 << n):
        recs = [C.x(k) for k in range(n) if (basis >> k) & 1]
        recs.append(C.cu(2, 0, [[0, 1], [1, 0]]))
        psi = orc.run(n, C.gates(recs))
        expect = basis ^ 1 if (basis >> 2) & 1 else basis
        assert abs(psi[expect] - 1.0) < 1e-15


def test_marginal_and_norm(orc):
    n = 6
    g = C.random_circuit(n, 3, 11)
    psi = orc.run(n, g)
    full = orc.marginal(n, psi, (1 << n) - 1)
    assert np.max(np.abs(full - np.abs(psi) ** 2)) < 1e-15
    # marginal over {1, 4}: brute-force sum over the other bits
    m = orc.marginal(n, psi, 0b010010)
    ref = np.zeros(4)
    for xi in range(1 << n):
        ref[((xi >> 1) & 1) | (((xi >> 4) & 1) << 1)] += abs(psi[xi]) ** 2
    assert np.max(np.abs(m - ref / ref.sum())) < 1e-15
    # product state: marginal of qubit 0 after U3 is (cos^2, sin^2)(theta/2)
    psi = orc.run(2, C.gates([C.u3(0, 1.2, 0.3, 0.1)]))
    m0 = orc.marginal(2, psi, 1)
    assert abs(m0[0] - np.cos(0.6) ** 2) < 1e-15 and abs(m0[1] - np.sin(0.6) ** 2) < 1e-15


def test_sampling_inverse_cdf(orc):
    p = np.array([0.1, 0.2, 0.3, 0.4])
    u = np.array([0.0, 0.05, 0.15, 0.31, 0.61, 0.999999])
    out, margin = orc.sample(p, u)
    assert list(out) == [0, 0, 1, 2, 3, 3]
    assert np.all(margin >= 0)
    # block order over > 1024 outcomes: C_i = prefix of block sums + in-block prefix
    rng = np.random.default_rng(3)
    q = rng.random(3000)
    c = orc.cdf(q)
    ref = np.empty_like(q)
    before = 0.0
    for b0 in range(0, q.size, 1024):
        run = 0.0
        for i in range(b0, min(b0 + 1024, q.size)):
            run += q[i]
            ref[i] = before + run
        before += run
    assert np.array_equal(c, ref)
    uu = rng.random(200)
    out, _ = orc.sample(q, uu)
    ref_out = [int(np.argmax(c > v * c[-1])) for v in uu]
    assert list(out) == ref_out


def test_argmax_lowest_tie(orc):
    assert orc.argmax(np.array([0.1, 0.4, 0.1, 0.4])) == (1, 0.4)
    assert orc.argmax(np.array([0.5]))[0] == 0


def test_rejects_bad_gates(orc):
    with pytest.raises(ValueError):
        orc.run(3, C.gates([C.h(3)]))
    with pytest.raises(ValueError):
        orc.run(3, C.gates([C.cz(1, 1)]))
    with pytest.raises(ValueError):
        orc.run(3, C.gates([C.swap(0, 0)]))


def test_rejects_bad_general_gates(orc):
    """A MAT record outside a U2Q, a U2Q without its three rows, a control
    mask that holds the target or is empty, and u outside [0, 1)."""
    m4 = np.eye(4)
    bad_lists = [
        C.gates(C.u2q(0, 1, m4)[1:2]),
        C.gates(C.u2q(0, 1, m4)[:3]),
        C.gates([C.mcu([0, 2], 2, np.eye(2))]),
        C.gates([C.mcu([], 1, np.eye(2))]),
        C.gates([C.measure(0, 1.0)]),
        C.gates([C.measure(0, -0.1)]),
    ]
    for g in bad_lists:
        with pytest.raises(ValueError):
            orc.run(3, g)


def test_measure_outcomes_reported(orc):
    """Outcomes come back in list order: |1> on qubit 1 always measures 1,
    |0> on qubit 0 always 0, and H then u = 0.7 gives 1."""
    g = C.gates([C.x(1), C.measure(1, 0.0), C.measure(0, 0.99), C.h(2), C.measure(2, 0.7)])
    psi = orc.init(3)
    assert list(orc.apply_measured(3, psi, g)) == [1, 0, 1]


@pytest.mark.parametrize("mutation", [1, 2, 3, 4, 5, 6, 7, 8])
def test_planted_mistake_is_caught(orc, mutation):
    """A build of the oracle with a planted mistake must fail at least one pin."""
    orc.build(mutation)
    run = _runner(orc, mutation)
    rows = [(int(r[0]), r[1], float(r[2])) for r in _fixture("paper_qpe.txt")]
    failures = pins.pin_paper_qpe(run, rows)
    for name in pins.ALL_PINS:
        failures += getattr(pins, name)(run)
    assert failures, f"mutation {mutation} passed every pin"
