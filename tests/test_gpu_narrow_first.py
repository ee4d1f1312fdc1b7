"""SV_FLAG_NARROW_FIRST on the GPU: the list's first pass gathers 16-amplitude
chunks and generates the recorded |0...0> in registers, the later passes use
the configured width; amplitudes against the FP64 oracle (complex64 and the
complex128 register-stage kernel), and the QPE outcome exact."""
import numpy as np
import pytest

from gen import mixed_circuit
from paper_2605_15098_gb300 import circuits as C

pytestmark = pytest.mark.gpu

TOL128 = 1e-12
FID64 = 1e-6
ERR64 = 2e-5


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


@pytest.mark.parametrize("n,chunk", [(20, 7), (22, 6), (22, 8), (24, 7), (26, 7), (26, 9)])
def test_qpe_c64(sv, orc, n, chunk):
    g, expected, info = C.qpe(n, seed=n)
    ref = orc.run(n, g)
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=chunk, flags=sv.SV_FLAG_NARROW_FIRST)
    plan = sv.sv_plan_export(n, sv.SV_C64, g, cfg)
    assert plan["passes"][0]["c"] == 4
    with sv.State(n, sv.SV_C64) as s:
        s.apply(g, cfg)
        got = s.amplitudes()
        idx, p = s.argmax(info["mask"])
    assert idx == info["y"] and abs(p - 1.0) <= 1e-5
    assert np.max(np.abs(got - ref)) <= ERR64
    assert fidelity(ref, got) >= 1 - FID64


@pytest.mark.parametrize("n,seed", [(16, 1), (18, 2)])
def test_mixed_c64_and_c128(sv, orc, n, seed):
    g = mixed_circuit(n, 200, 31 * n + seed)
    ref = orc.run(n, g)
    for dtype, chunk in ((sv.SV_C64, 7), (sv.SV_C64, 9), (sv.SV_C128, 6)):
        cfg = sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=13, chunk_qubits=chunk,
                             flags=sv.SV_FLAG_NARROW_FIRST)
        with sv.State(n, dtype) as s:
            s.apply(g, cfg)
            got = s.amplitudes()
            s.reset()
            s.apply(g, cfg)  # a second call from the recorded state, from the programme cache
            again = s.amplitudes()
        if dtype == sv.SV_C128:
            assert np.max(np.abs(got - ref)) <= TOL128
        else:
            assert np.max(np.abs(got - ref)) <= ERR64 and fidelity(ref, got) >= 1 - FID64
        assert np.array_equal(got, again)


def test_reading_first_pass(sv, orc):
    """The narrow pass also runs when the state is not a recorded basis state
    (it then reads its tile in 16-amplitude chunks)."""
    n = 20
    g, expected, info = C.qpe(n, seed=3)
    pre = C.gates([C.p(0, 0.7)])  # leaves |0...0>, written out by the per-gate kernel
    ref = orc.run(n, g)
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=7, flags=sv.SV_FLAG_NARROW_FIRST)
    with sv.State(n, sv.SV_C64) as s:
        s.apply(pre, sv.make_config(sv.SV_MODE_PERGATE))
        s.apply(g, cfg)
        got = s.amplitudes()
        idx, p = s.argmax(info["mask"])
    assert idx == info["y"]
    assert np.max(np.abs(got - ref)) <= ERR64


def test_with_l2_blocks_identical_to_one_level(sv, orc):
    """A narrow first pass inside an L2 block group: the group kernel computes
    the tiles' slot values itself, the one-level kernel receives them from
    k_slotv; the same sums and products, so the amplitudes are bit-identical."""
    n = 22
    g, expected, info = C.qpe(n, seed=5)
    ref = orc.run(n, g)
    outs = []
    for flags, l2 in ((sv.SV_FLAG_NARROW_FIRST, 0), (sv.SV_FLAG_NARROW_FIRST | sv.SV_FLAG_L2_BLOCKS, 18)):
        cfg = sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=7, flags=flags, l2_qubits=l2, l2_chunk=2)
        with sv.State(n, sv.SV_C64) as s:
            s.apply(g, cfg)
            outs.append(s.amplitudes())
            idx, p = s.argmax(info["mask"])
        assert idx == info["y"]
        assert np.max(np.abs(outs[-1] - ref)) <= ERR64
    assert np.array_equal(outs[0], outs[1])
