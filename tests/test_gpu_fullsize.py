"""Full-size configurations (GPU): QPE up to n = 32 in both dtypes, and the
depth-40 random circuit at n = 30.  The oracle cannot run these sizes, so
the checks are properties that hold at any size: QPE's closed-form outcome
(Eq. 2-3), a random circuit followed by its inverse returning to |0...0>,
and agreement between the per-gate and partitioned paths."""
import numpy as np
import pytest

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


def inverse(g):
    """Gates in reverse order, each replaced by its inverse (U3 and CZ here)."""
    recs = []
    for r in g[::-1]:
        kind, t = int(r["kind"]), int(r["target"])
        if kind == C.U3:
            th, ph, la = (float(v) for v in r["p"][:3])
            recs.append(C.u3(t, -th, -la, -ph))
        elif kind == C.CZ:
            recs.append(C.cz(int(r["control"]), t))
        else:
            raise ValueError(kind)
    return C.gates(recs)


@pytest.mark.parametrize("n,dtype", [(32, 0), (30, 1), (32, 1)])
def test_qpe_largest_sizes(sv, n, dtype):
    g, expected, info = C.qpe(n)
    with sv.State(n, dtype) as s:
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=7 if dtype == 0 else 0))
        idx, p = s.argmax(info["mask"])
    assert idx == info["y"]
    assert abs(p - 1.0) <= (1e-12 if dtype == sv.SV_C128 else 1e-5)


@pytest.mark.parametrize("mode", [2, 3])
def test_random30_then_inverse_is_identity(sv, mode):
    """U then U^-1 on |0...0>: the full state returns to e_0 (complex64, n = 30,
    register-stage (2) and fused tensor-core (3) paths)."""
    n = 30
    g = C.random_circuit(n, 40)
    gi = inverse(g)
    with sv.State(n, sv.SV_C64) as s:
        cfg = sv.make_config(mode, chunk_qubits=7)
        s.apply(g, cfg)
        s.apply(gi, cfg)
        psi = s.amplitudes()
    assert abs(abs(complex(psi[0])) ** 2 - 1.0) <= 2e-5
    rest = 0.0
    step = 1 << 24
    for i in range(0, psi.size, step):
        chunk = psi[i:i + step].astype(np.complex128)
        if i == 0:
            chunk[0] = 0
        rest += float(np.sum(chunk.real ** 2 + chunk.imag ** 2))
    assert rest <= 2e-5


def test_random30_pergate_and_partitioned_agree(sv):
    n = 30
    g = C.random_circuit(n, 40, seed=11)
    mask = (1 << 16) - 1 << 7          # 16 qubits in the middle
    out = []
    for mode in (sv.SV_MODE_PERGATE, sv.SV_MODE_PARTITIONED):
        with sv.State(n, sv.SV_C64) as s:
            s.apply(g, sv.make_config(mode))
            out.append(s.probabilities(mask))
    assert np.max(np.abs(out[0] - out[1])) <= 1e-6
    assert abs(out[1].sum() - 1.0) <= 1e-9
