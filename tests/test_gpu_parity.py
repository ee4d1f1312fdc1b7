"""CUDA path against the FP64 oracle, element by element (GPU).

Tolerances:
  * complex128: max |amp_gpu - amp_oracle| <= 1e-12 (both sides FP64; the
    difference is rounding order and the device's own cos/sin).
  * complex64: fidelity |<psi_oracle|psi_gpu>|^2 >= 1 - 1e-6 and
    max |amp error| <= 2e-5 (FP32 storage: ~6e-8 relative per operation,
    grown by the gate count).
  * Integer outcomes (argmax, samples) are compared exactly; a differing
    sample is accepted only where the oracle's own CDF puts u*C_last within
    1e-12 of an outcome boundary (a genuine tie that FP64 rounding decides).
"""
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


def run_gpu(sv, n, gates, dtype, cfg=None):
    with sv.State(n, dtype) as s:
        s.apply(gates, cfg)
        return s.amplitudes(), s.stats()


def fidelity(a, b):
    return abs(np.vdot(a.astype(np.complex128), b.astype(np.complex128))) ** 2


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11, 14])
def test_pergate_c128_all_kinds(sv, orc, n):
    for seed in (1, 2):
        g = mixed_circuit(n, 60, 100 * n + seed)
        ref = orc.run(n, g)
        got, st = run_gpu(sv, n, g, sv.SV_C128, sv.make_config(sv.SV_MODE_PERGATE))
        assert np.max(np.abs(got - ref)) <= TOL128
        assert st["passes"] == len(g)


@pytest.mark.parametrize("n,k,c", [(6, 12, 4), (12, 8, 3), (14, 10, 4), (16, 8, 2), (17, 12, 5),
                                   (18, 13, 4)])
def test_partitioned_c128_all_kinds(sv, orc, n, k, c):
    g = mixed_circuit(n, 120, 7 * n + k)
    ref = orc.run(n, g)
    got, st = run_gpu(sv, n, g, sv.SV_C128,
                      sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=min(k, 13), chunk_qubits=c))
    assert np.max(np.abs(got - ref)) <= TOL128
    assert st["passes"] < len(g)


@pytest.mark.parametrize("flags", [0, 1, 4, 5])
def test_partitioned_flags(sv, orc, flags):
    n = 15
    g = mixed_circuit(n, 90, 31 + flags)
    ref = orc.run(n, g)
    got, _ = run_gpu(sv, n, g, sv.SV_C128,
                     sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=9, chunk_qubits=3, flags=flags))
    assert np.max(np.abs(got - ref)) <= TOL128


def test_qpe12_c128(sv, orc):
    """QPE, 12 qubits, complex128: amplitudes, P(expected) = 1, argmax exact."""
    n = 12
    g, expected, info = C.qpe(n)
    ref = orc.run(n, g)
    for mode in (sv.SV_MODE_PERGATE, sv.SV_MODE_PARTITIONED):
        with sv.State(n, sv.SV_C128) as s:
            s.apply(g, sv.make_config(mode, tile_qubits=8, chunk_qubits=3))
            got = s.amplitudes()
            assert np.max(np.abs(got - ref)) <= TOL128
            idx, p = s.argmax(info["mask"])
            assert idx == info["y"]
            assert abs(p - 1.0) <= 1e-12
            idx_full, p_full = s.argmax((1 << n) - 1)
            assert idx_full == expected


@pytest.mark.parametrize("n", [16, 20, 22])
def test_qpe_sweep_c128_parity(sv, orc, n):
    g, expected, info = C.qpe(n, seed=n)
    ref = orc.run(n, g)
    for mode in (sv.SV_MODE_PERGATE, sv.SV_MODE_PARTITIONED):
        got, _ = run_gpu(sv, n, g, sv.SV_C128, sv.make_config(mode))
        assert np.max(np.abs(got - ref)) <= TOL128


@pytest.mark.parametrize("n,dtype,chunk,flags", [(28, 0, 0, 0), (28, 1, 0, 0), (30, 0, 0, 0),
                                                   (28, 0, 9, 256), (30, 0, 9, 256)])
def test_qpe_full_size_closed_form(sv, n, dtype, chunk, flags):
    """Full-size QPE in the library's default configuration and in the one the
    autotuner picks for complex64 QPE-28/30 (chunk 9, narrow first pass): the
    counting register reads y = sum(a_i) mod 2^t with probability 1 (Eq. 2-3)."""
    g, expected, info = C.qpe(n)
    with sv.State(n, dtype) as s:
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=chunk, flags=flags))
        idx, p = s.argmax(info["mask"])
        assert idx == info["y"]
        assert abs(p - 1.0) <= (1e-12 if dtype == sv.SV_C128 else 1e-5)
        idx_full, _ = s.argmax((1 << n) - 1)
        assert idx_full == expected


@pytest.mark.parametrize("mode", [1, 2])
def test_c64_random_fidelity(sv, orc, mode):
    n = 16
    g = mixed_circuit(n, 150, 55 + mode)
    ref = orc.run(n, g)
    got, _ = run_gpu(sv, n, g, sv.SV_C64, sv.make_config(mode, tile_qubits=10, chunk_qubits=3))
    assert 1.0 - fidelity(ref, got) <= FID64
    assert np.max(np.abs(got - ref)) <= ERR64


def test_c64_qpe(sv, orc):
    n = 20
    g, expected, info = C.qpe(n, seed=3)
    ref = orc.run(n, g)
    for mode in (sv.SV_MODE_PERGATE, sv.SV_MODE_PARTITIONED):
        with sv.State(n, sv.SV_C64) as s:
            s.apply(g, sv.make_config(mode))
            got = s.amplitudes()
            assert 1.0 - fidelity(ref, got) <= FID64
            idx, p = s.argmax(info["mask"])
            assert idx == info["y"] and abs(p - 1.0) <= 1e-5


@pytest.mark.parametrize("mask_kind", ["low", "high", "mixed", "single_high", "full", "single_low"])
def test_readout_parity(sv, orc, mask_kind):
    n = 13
    g = mixed_circuit(n, 80, 9)
    psi = orc.run(n, g)
    masks = {"low": 0b111111, "high": 0b1111100000000, "mixed": 0b1010011001010,
             "single_high": 1 << 12, "full": (1 << n) - 1, "single_low": 1}
    mask = masks[mask_kind]
    with sv.State(n, sv.SV_C128) as s:
        # partitioned so that the qubit map is not the identity (SWAP relabels)
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=8, chunk_qubits=2))
        p = s.probabilities(mask)
        ref = orc.marginal(n, psi, mask)
        assert np.max(np.abs(p - ref)) <= 1e-13
        idx, pm = s.argmax(mask)
        ridx, rpm = orc.argmax(ref)
        if idx != ridx:
            assert abs(ref[idx] - rpm) <= 1e-13  # a genuine near-tie
        gen = C.SplitMix64(1234)
        u = np.array([gen.uniform() for _ in range(500)])
        got = s.sample(mask, u)
        want, margin = orc.sample(ref, u)
        bad = (got != want) & (margin > 1e-12)
        assert not bad.any()


def test_edge_cases(sv, orc):
    # empty circuit
    with sv.State(4, sv.SV_C128) as s:
        s.apply(C.gates([]))
        a = s.amplitudes()
        assert a[0] == 1 and np.all(a[1:] == 0)
    # n = 1, every single-qubit kind, both paths, both dtypes
    g = C.gates([C.h(0), C.x(0), C.p(0, 0.3), C.pk(0, 3, 3), C.u3(0, 1, 2, 3),
                 C.u(0, [[0, 1j], [1j, 0]])])
    ref = orc.run(1, g)
    for dt in (sv.SV_C64, sv.SV_C128):
        for mode in (1, 2):
            got, _ = run_gpu(sv, 1, g, dt, sv.make_config(mode))
            assert np.max(np.abs(got - ref)) <= (TOL128 if dt else ERR64)
    # invalid gate: error, state untouched
    with sv.State(3, sv.SV_C128) as s:
        s.apply(C.gates([C.h(1)]))
        before = s.amplitudes()
        with pytest.raises(sv.SvError):
            s.apply(C.gates([C.h(0), C.cz(2, 2)]))
        with pytest.raises(sv.SvError):
            s.apply(C.gates([C.h(3)]))
        assert np.array_equal(before, s.amplitudes())
        with pytest.raises(sv.SvError):
            s.sample(1, np.array([1.0]))
        with pytest.raises(sv.SvError):
            s.probabilities(1 << 3)


def test_create_on_torch_buffer(sv, orc):
    import torch

    n = 14
    buf = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    stream = torch.cuda.Stream()
    g = mixed_circuit(n, 50, 77)
    ref = orc.run(n, g)
    with sv.State(n, sv.SV_C128, tensor=buf, stream=stream) as s:
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=9, chunk_qubits=3))
        # the caller's tensor holds the state in physical order
        phys = sv.sv_qubit_map(s.h)
        stream.synchronize()
        dev = buf.cpu().numpy()
        perm = np.zeros(1 << n, dtype=np.int64)
        for x in range(1 << n):
            y = 0
            for q in range(n):
                y |= ((x >> q) & 1) << phys[q]
            perm[x] = y
        assert np.max(np.abs(dev[perm] - ref)) <= TOL128


@pytest.mark.parametrize("n,chunk", [(14, 5), (16, 4), (17, 6), (18, 7), (19, 5)])
def test_c64_register_stage_kernel(sv, orc, n, chunk):
    """complex64 passes on the register-stage kernel (tiles of 2^13, bulk copies).
    CU gates are left out: a pass with a register-controlled CU runs on the
    generic tile kernel (covered by the partitioned tests above)."""
    g = mixed_circuit(n, 160, 500 + n, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 9, 10))
    ref = orc.run(n, g)
    with sv.State(n, sv.SV_C64) as s:
        sv.sv_profile(s.h, True)
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED, chunk_qubits=chunk))
        recs = sv.sv_profile_read(s.h)
        got = s.amplitudes()
    assert any(r["gate_kind"] == -2 for r in recs)  # register-stage launches
    assert 1.0 - fidelity(ref, got) <= FID64
    assert np.max(np.abs(got - ref)) <= ERR64


@pytest.mark.parametrize("n,chunk,kind", [(15, 4, "mixed"), (17, 7, "mixed"), (18, 5, "qpe"),
                                          (20, 4, "random")])
def test_c64_wide_tiles(sv, orc, n, chunk, kind):
    """2^14-amplitude tiles (512 threads, one CTA per SM) on the register-stage kernel."""
    if kind == "qpe":
        g = C.qpe(n, seed=n)[0]
    elif kind == "random":
        g = C.random_circuit(n, 8, seed=n)
    else:
        g = mixed_circuit(n, 150, n + 3, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 9, 10))
    ref = orc.run(n, g)
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=14, chunk_qubits=chunk)
    plan = sv.sv_plan_export(n, sv.SV_C64, g, cfg)
    assert all(p["kernel"] == "t2" and p["t2"]["threads"] == 512 for p in plan["passes"] if p["ops"])
    with sv.State(n, sv.SV_C64) as s:
        s.apply(g, cfg)
        got = s.amplitudes()
    assert 1.0 - fidelity(ref, got) <= FID64
    assert np.max(np.abs(got - ref)) <= ERR64


def test_c64_register_stage_vs_generic(sv):
    """Same circuit through both tile kernels: equal up to float32 rounding."""
    n = 18
    g = C.random_circuit(n, 6, 77)
    a, _ = run_gpu(sv, n, g, sv.SV_C64, sv.make_config(sv.SV_MODE_PARTITIONED))
    b, _ = run_gpu(sv, n, g, sv.SV_C64,
                   sv.make_config(sv.SV_MODE_PARTITIONED, flags=sv.SV_FLAG_GENERIC_TILE))
    assert 1.0 - fidelity(a, b) <= FID64


FUSED_FID = 1e-6


@pytest.mark.parametrize("n,seed", [(14, 1), (16, 2), (18, 3)])
def test_fused_mixed(sv, orc, n, seed):
    """Tensor-core fused blocks (tcgen05, TF32 split three-pass) on every gate kind
    (CU controlled by another in-tile qubit folds into the blocks)."""
    g = mixed_circuit(n, 160, 900 + seed, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 9, 10))
    ref = orc.run(n, g)
    with sv.State(n, sv.SV_C64) as s:
        sv.sv_profile(s.h, True)
        s.apply(g, sv.make_config(sv.SV_MODE_FUSED))
        recs = sv.sv_profile_read(s.h)
        st = s.stats()
        got = s.amplitudes()
    assert any(r["kind"] == sv.SV_KERNEL_FUSED for r in recs)
    assert st["fused_blocks"] > 0
    assert 1.0 - fidelity(ref, got) <= FUSED_FID
    assert np.max(np.abs(got - ref)) <= ERR64


def test_fused_random_streamed_blocks(sv, orc):
    """Random U3 + CZ layers: passes with more blocks than shared-memory slots."""
    n = 20
    g = C.random_circuit(n, 8, 4321)
    ref = orc.run(n, g)
    got, st = run_gpu(sv, n, g, sv.SV_C64, sv.make_config(sv.SV_MODE_FUSED))
    assert st["fused_blocks"] > 0  # blocks were used
    assert 1.0 - fidelity(ref, got) <= FUSED_FID
    assert np.max(np.abs(got - ref)) <= ERR64


def test_random_depth40_both_paths(sv, orc):
    """The random-circuit workload at depth 40 (U3 layers and CZ matchings),
    n = 24: register-stage passes and fused tensor-core passes both within
    the complex64 tolerances of the FP64 oracle."""
    n = 24
    g = C.random_circuit(n, 40, 2605)
    ref = orc.run(n, g)
    for mode in (sv.SV_MODE_PARTITIONED, sv.SV_MODE_FUSED):
        got, st = run_gpu(sv, n, g, sv.SV_C64, sv.make_config(mode))
        if mode == sv.SV_MODE_FUSED:
            assert st["fused_blocks"] > 0
        assert 1.0 - fidelity(ref, got) <= FUSED_FID
        assert np.max(np.abs(got - ref)) <= ERR64


@pytest.mark.parametrize("n", [16, 20])
def test_fused_qpe(sv, orc, n):
    g, expected, info = C.qpe(n, seed=n + 7)
    ref = orc.run(n, g)
    with sv.State(n, sv.SV_C64) as s:
        s.apply(g, sv.make_config(sv.SV_MODE_FUSED))
        got = s.amplitudes()
        idx, p = s.argmax(info["mask"])
    assert 1.0 - fidelity(ref, got) <= FUSED_FID
    assert idx == info["y"] and abs(p - 1.0) <= 1e-5


@pytest.mark.parametrize("n", [28, 30])
def test_fused_qpe_full_size(sv, n):
    g, expected, info = C.qpe(n)
    with sv.State(n, sv.SV_C64) as s:
        s.apply(g, sv.make_config(sv.SV_MODE_FUSED))
        idx, p = s.argmax(info["mask"])
        assert idx == info["y"] and abs(p - 1.0) <= 1e-5
        assert s.argmax((1 << n) - 1)[0] == expected


@pytest.mark.parametrize("flags", [0, 32, 64, 96, 256])
def test_batch_qpe_outcomes(sv, orc, flags):
    """Batched QPE instances (n uniform in 10..20) in one graph-captured launch:
    every outcome equals the oracle's argmax (small n) and the closed form,
    with each planner option (diagonal placement, local search, a first pass
    of 16-amplitude chunks at chunk width 7)."""
    work = C.qpe_batch(96, seed=777)
    cfg = None
    if flags:
        cfg = sv.make_config(sv.SV_MODE_PARTITIONED, flags=flags,
                             chunk_qubits=7 if flags & sv.SV_FLAG_NARROW_FIRST else 0)
    b = sv.sv_batch_create([(n, g, m) for n, g, m, _ in work], cfg)
    try:
        idx, p, ms = sv.sv_batch_run(b, len(work))
        idx2, p2, _ = sv.sv_batch_run(b, len(work))  # replay gives the same results
        info = sv.sv_batch_info(b)
    finally:
        sv.sv_batch_destroy(b)
    assert np.array_equal(idx, idx2) and np.array_equal(p, p2)
    assert info["count"] == len(work) and info["passes"] >= len(work)
    for i, (n, g, mask, y) in enumerate(work):
        assert int(idx[i]) == y, (i, n)
        assert abs(p[i] - 1.0) <= 1e-5
        if n <= 14:
            ref = orc.marginal(n, orc.run(n, g), mask)
            assert int(idx[i]) == orc.argmax(ref)[0]


def test_batch_mixed_circuits_match_single(sv):
    """Batch read-outs equal those of the single-state API on the same circuits."""
    from gen import mixed_circuit
    rng = np.random.default_rng(3)
    circ = []
    for i in range(24):
        n = int(rng.integers(5, 17))
        g = mixed_circuit(n, 40, 60 + i, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 9, 10))
        circ.append((n, g, (1 << n) - 1))
    idx, p = sv.sv_apply_circuit_batch(circ)
    for i, (n, g, mask) in enumerate(circ):
        with sv.State(n, sv.SV_C128) as s:
            s.apply(g, sv.make_config(sv.SV_MODE_PERGATE))
            probs = s.probabilities(mask)
        top = np.sort(probs)[-2:]
        if top[1] - top[0] > 1e-5:  # a clear maximum: same index
            assert int(idx[i]) == int(np.argmax(probs))
        assert abs(p[i] - probs.max()) <= 1e-5


def test_autotune_picks_a_valid_config(sv, orc, tmp_path):
    n = 16
    g, expected, info = C.qpe(n, seed=5)
    cache = str(tmp_path / "tune.txt")
    with sv.State(n, sv.SV_C64) as s:
        best, ms = sv.sv_autotune(s.h, g, cache)
        assert ms > 0 and best.mode in (sv.SV_MODE_PARTITIONED, sv.SV_MODE_FUSED)
        best2, ms2 = sv.sv_autotune(s.h, g, cache)  # cache hit: same answer
        assert (best2.mode, best2.chunk_qubits, best2.tile_qubits, best2.flags, best2.l2_chunk) == \
            (best.mode, best.chunk_qubits, best.tile_qubits, best.flags, best.l2_chunk)
        assert abs(ms2 - ms) < 1e-3
        s.apply(g, best)
        idx, p = s.argmax(info["mask"])
        assert idx == info["y"] and abs(p - 1) < 1e-5
    # another circuit with the same structure (different angles) hits the same entry
    g2, _, _ = C.qpe(n, seed=6)
    with sv.State(n, sv.SV_C64) as s:
        best3, ms3 = sv.sv_autotune(s.h, g2, cache)
        assert abs(ms3 - ms) < 1e-3


def test_batch_autotune(sv):
    work = C.qpe_batch(64, seed=11)
    items = [(n, g, m) for n, g, m, _ in work]
    best, ms = sv.sv_batch_autotune(items)
    assert best.chunk_qubits in (4, 5, 6, 7) and best.batch_split in (0, 16) and ms > 0
    idx, p = sv.sv_apply_circuit_batch(items, best)
    assert all(int(idx[i]) == w[3] for i, w in enumerate(work))


def test_batch_product_state_prefixes(sv, orc):
    """Leading X and H gates of a batched instance fold into the product state
    that its first pass generates; instances made of such gates only (nothing
    left to generate the state) are planned as given.  Outcomes and their
    probabilities against the oracle."""
    from gen import mixed_circuit
    circ = [(5, C.gates([C.x(0), C.x(3)]), 31),
            (14, C.gates([C.h(0), C.h(1)]), 3),
            (14, C.gates([C.x(2), C.h(2)]), 4),
            (16, C.gates([C.x(1), C.h(1), C.x(1), C.h(4)] + list(mixed_circuit(16, 30, 9))), (1 << 16) - 1),
            (17, C.gates([C.h(q) for q in range(17)] + [C.x(16), C.cz(0, 16)] +
                         list(mixed_circuit(17, 40, 10, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 9, 10)))), (1 << 17) - 1)]
    idx, p = sv.sv_apply_circuit_batch(circ)
    for i, (n, g, mask) in enumerate(circ):
        probs = orc.marginal(n, orc.run(n, g), mask)
        top = np.sort(probs)[-2:]
        if top[1] - top[0] > 1e-5:
            assert int(idx[i]) == int(np.argmax(probs)), i
        else:  # ties: an index of the maximum
            assert probs[int(idx[i])] >= top[1] - 1e-5, i
        assert abs(p[i] - probs.max()) <= 1e-5, i


@pytest.mark.parametrize("split", [0, 14, 16, 19, 25])
def test_batch_split_instances(sv, split):
    """Instances of at least `split` qubits are shared out among CTAs pass by
    pass (25: none is): every outcome equals the closed form, and the
    probabilities equal those of the unsplit launch."""
    work = C.qpe_batch(160, seed=4242)
    items = [(n, g, m) for n, g, m, _ in work]
    idx, p = sv.sv_apply_circuit_batch(items, sv.make_config(sv.SV_MODE_PARTITIONED, batch_split=split))
    idx0, p0 = sv.sv_apply_circuit_batch(items, sv.make_config(sv.SV_MODE_PARTITIONED, batch_split=25))
    for i, (n, g, mask, y) in enumerate(work):
        assert int(idx[i]) == y, (i, n)
    assert np.array_equal(idx, idx0)
    assert np.max(np.abs(p - p0)) == 0.0  # same per-tile arithmetic and summation order
