"""The complex128 register-stage kernel (GPU): the format-2 programme with
64-bit phases and FP64 values, on 2^13-amplitude tiles.  Every case against
the FP64 oracle within 1e-12, the complex128 bar of the parity suite."""
import numpy as np
import pytest

from gen import mixed_circuit
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


def run(sv, n, g, chunk=5, flags=0, records=False):
    with sv.State(n, sv.SV_C128) as s:
        if records:
            sv.sv_profile(s.h, True)
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=13, chunk_qubits=chunk, flags=flags))
        recs = sv.sv_profile_read(s.h) if records else []
        st = s.stats()
        return s.amplitudes(), st, recs


@pytest.mark.parametrize("n", [13, 16, 20])
def test_qpe(sv, orc, n):
    g, _, info = C.qpe(n, seed=n)
    ref = orc.run(n, g)
    got, st, recs = run(sv, n, g, records=True)
    assert np.max(np.abs(got - ref)) <= 1e-12
    # the register-stage kernel ran every pass (gate_kind -2), one CTA per SM
    assert recs and all(r["gate_kind"] == -2 for r in recs if r["kind"] == sv.SV_KERNEL_TILE)
    assert st["ctas_per_sm"] == 1


@pytest.mark.parametrize("n,seed,chunk", [(14, 1, 4), (16, 2, 5), (18, 3, 7)])
def test_mixed(sv, orc, n, seed, chunk):
    g = mixed_circuit(n, 300, seed, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 9, 10))
    ref = orc.run(n, g)
    got, _, _ = run(sv, n, g, chunk=chunk)
    assert np.max(np.abs(got - ref)) <= 1e-12


@pytest.mark.parametrize("n,depth", [(15, 10), (19, 8)])
def test_random_layers(sv, orc, n, depth):
    g = C.random_circuit(n, depth, 100 + n)
    ref = orc.run(n, g)
    got, _, _ = run(sv, n, g)
    assert np.max(np.abs(got - ref)) <= 1e-12


def test_product_state_prefix_and_controls(sv, orc):
    """Leading X and H fold into the generated first pass; controlled gates
    on register, thread and global bits."""
    n = 17
    rng = np.random.default_rng(5)
    recs = [C.x(2), C.h(0), C.h(5), C.x(9), C.h(9), C.h(16)]
    for _ in range(200):
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        k = rng.integers(4)
        if k == 0:
            recs.append(C.cu(a, b, C.random_unitary(rng)))
        elif k == 1:
            recs.append(C.cp(a, b, float(rng.uniform(0, 6.3))))
        elif k == 2:
            recs.append(C.u3(a, *rng.uniform(0, 6.3, 3)))
        else:
            recs.append(C.h(a))
    g = C.gates(recs)
    ref = orc.run(n, g)
    got, _, _ = run(sv, n, g)
    assert np.max(np.abs(got - ref)) <= 1e-12
