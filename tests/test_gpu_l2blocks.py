"""Two-level blocking on the GPU (Sec. III-B: blocks sized by the last-level
cache, here L2): with SV_FLAG_L2_BLOCKS the passes of a group run in one
launch, block by block.  Checked against the FP64 oracle and against the
one-level plan, which runs the same per-tile arithmetic, so the amplitudes
must be identical bit for bit."""
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


def run(sv, n, g, cfg, records=False):
    with sv.State(n, sv.SV_C64) as s:
        if records:
            sv.sv_profile(s.h, True)
        s.apply(g, cfg)
        st = s.stats()
        amps = s.amplitudes()
        recs = sv.sv_profile_read(s.h) if records else []
    return amps, st, recs


@pytest.mark.parametrize("n,l2", [(18, 15), (20, 16), (20, 18), (22, 18), (22, 0), (24, 20), (26, 0)])
def test_qpe_parity_and_identical_to_one_level(sv, orc, n, l2):
    g, expected, _ = C.qpe(n, seed=n)
    ref = orc.run(n, g)
    one, st1, _ = run(sv, n, g, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=7))
    two, st2, recs = run(sv, n, g, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=7,
                                                  flags=sv.SV_FLAG_L2_BLOCKS, l2_qubits=l2), records=True)
    assert float(np.max(np.abs(two - ref))) <= 2e-5
    assert np.array_equal(one, two)
    assert st2["passes"] == st1["passes"]
    # two CTAs of the 2^13-amplitude tile kernels per SM, grouped or not
    assert st1["ctas_per_sm"] == 2 and st2["ctas_per_sm"] == 2
    # one launch per group: nops passes, a block of 2^k amplitudes
    grouped = [r for r in recs if r["kind"] == sv.SV_KERNEL_L2BLOCK]
    assert st2["kernels"] == st1["kernels"] - sum(r["nops"] - 1 for r in grouped)
    # the default block size follows the device's L2 size
    assert all(2 <= r["nops"] <= 4 and r["k"] == (min(l2, n) if l2 else min(r["k"], n)) and r["k"] >= 14
               for r in grouped)


@pytest.mark.parametrize("n,seed,l2", [(20, 1, 16), (22, 2, 18), (24, 3, 20)])
def test_random_layers_parity(sv, orc, n, seed, l2):
    g = C.random_circuit(n, 12, seed)
    ref = orc.run(n, g)
    one, _, _ = run(sv, n, g, sv.make_config(sv.SV_MODE_PARTITIONED))
    two, _, recs = run(sv, n, g, sv.make_config(sv.SV_MODE_PARTITIONED, flags=sv.SV_FLAG_L2_BLOCKS,
                                                l2_qubits=l2), records=True)
    assert float(np.max(np.abs(two - ref))) <= 2e-5
    assert np.array_equal(one, two)


@pytest.mark.parametrize("n,seed", [(17, 4), (19, 5)])
def test_mixed_gates_and_sweep(sv, orc, n, seed):
    """Every gate kind of the register-stage kernel, over a sweep of block sizes."""
    g = mixed_circuit(n, 300, seed, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 9, 10))
    ref = orc.run(n, g)
    one, _, _ = run(sv, n, g, sv.make_config(sv.SV_MODE_PARTITIONED))
    groups = 0
    for l2 in (14, 15, 16, 17, n):
        for chunk in (1, 4):
            two, _, recs = run(sv, n, g, sv.make_config(sv.SV_MODE_PARTITIONED, flags=sv.SV_FLAG_L2_BLOCKS,
                                                        l2_qubits=l2, l2_chunk=chunk), records=True)
            assert float(np.max(np.abs(two - ref))) <= 2e-5
            assert np.array_equal(one, two), (l2, chunk)
            groups += sum(r["kind"] == sv.SV_KERNEL_L2BLOCK for r in recs)
    assert groups > 0


def test_readout_after_groups(sv, orc):
    """QPE's read-out after a grouped run: the expected outcome."""
    n = 24
    g, expected, info = C.qpe(n, seed=11)
    with sv.State(n, sv.SV_C64) as s:
        sv.sv_profile(s.h, True)
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=7, flags=sv.SV_FLAG_L2_BLOCKS))
        idx, p = s.argmax(info["mask"])
        recs = sv.sv_profile_read(s.h)
    assert idx == info["y"] and p > 0.99
    assert any(r["kind"] == sv.SV_KERNEL_L2BLOCK for r in recs)


def test_autotune_with_l2_candidates(sv, tmp_path):
    """A state larger than L2: the autotuner also measures L2 block groups;
    whatever it picks reproduces the QPE outcome and comes back from its
    cache with the same flags."""
    n = 24
    g, _, info = C.qpe(n, seed=2)
    cache = str(tmp_path / "tune.txt")
    with sv.State(n, sv.SV_C64) as s:
        best, ms = sv.sv_autotune(s.h, g, cache)
        best2, _ = sv.sv_autotune(s.h, g, cache)
        assert (best2.flags, best2.l2_chunk, best2.chunk_qubits) == (best.flags, best.l2_chunk, best.chunk_qubits)
        s.apply(g, best)
        idx, p = s.argmax(info["mask"])
    assert idx == info["y"] and p > 0.99
