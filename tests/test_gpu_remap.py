"""Remap passes on the GPU: the paper's explicit global-local SWAPs (Sec.
III-B, SV_FLAG_PAPER_SWAP) and the layout normalisation before a copy-out.

A remap moves amplitudes without arithmetic, so a state made only of
permutations is compared bit for bit; circuits with arithmetic use the
tolerances of the parity suite (complex128 1e-12, complex64 fidelity).
"""
import numpy as np
import pytest

from gen import mixed_circuit, without_leading_x
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


def fidelity(a, b):
    return abs(np.vdot(a.astype(np.complex128), b.astype(np.complex128))) ** 2


def swap_bits_np(state, a, b):
    x = np.arange(state.size)
    differ = ((x >> a) & 1) != ((x >> b) & 1)
    y = np.where(differ, x ^ ((1 << a) | (1 << b)), x)
    return state[y]


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [5, 12, 19])
def test_layout_normalisation_is_exact(sv, n, dtype):
    """SWAP gates are relabels in partitioned mode; the copy-out moves the
    amplitudes back to logical order with at most two multi-pair remap
    passes.  The result equals the permuted input bit for bit."""
    rng = np.random.default_rng(n + 10 * dtype)
    ctype = np.complex64 if dtype == sv.SV_C64 else np.complex128
    psi = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)).astype(ctype)
    recs, want = [], psi.copy()
    for _ in range(3 * n):
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        recs.append(C.swap(a, b))
        want = swap_bits_np(want, a, b)
    g = C.gates(recs)
    for mode in (sv.SV_MODE_PARTITIONED, sv.SV_MODE_PERGATE):
        with sv.State(n, dtype) as s:
            sv.sv_copy_in(s.h, psi)
            s.apply(g, sv.make_config(mode))
            st = s.stats()
            got = s.amplitudes()
            assert got.dtype == ctype
            assert np.array_equal(got, want)
            if mode == sv.SV_MODE_PARTITIONED:
                assert st["relabels"] == len(g) and st["passes"] == 0


@pytest.mark.parametrize("n,k", [(14, 8), (17, 10), (19, 12)])
def test_paper_mode_c128(sv, orc, n, k):
    g = mixed_circuit(n, 160, 3 * n + k)
    ref = orc.run(n, g)
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=k, flags=sv.SV_FLAG_PAPER_SWAP)
    plan = sv.sv_plan_export(n, sv.SV_C128, without_leading_x(g), cfg)
    with sv.State(n, sv.SV_C128) as s:
        s.apply(g, cfg)
        st = s.stats()
        got = s.amplitudes()
    assert np.max(np.abs(got - ref)) <= 1e-12
    assert st["remaps"] == plan["remaps"] > 0
    tile_passes = sum(1 for p in plan["passes"] if p["ops"])
    assert st["passes"] == st["remaps"] + tile_passes


@pytest.mark.parametrize("n", [16, 20])
def test_paper_mode_c64_qpe(sv, orc, n):
    g, expected, info = C.qpe(n, seed=n + 5)
    ref = orc.run(n, g)
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, flags=sv.SV_FLAG_PAPER_SWAP)
    with sv.State(n, sv.SV_C64) as s:
        s.apply(g, cfg)
        assert s.stats()["remaps"] > 0
        idx, p = s.argmax(info["mask"])
        assert idx == info["y"] and abs(p - 1.0) <= 1e-5
        got = s.amplitudes()
    assert 1.0 - fidelity(ref, got) <= 1e-6


def test_paper_mode_full_size_qpe(sv):
    """QPE-28 complex64 with the paper's explicit remaps: the counting
    register still reads its closed-form value (Eq. 2-3)."""
    n = 28
    g, expected, info = C.qpe(n)
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, flags=sv.SV_FLAG_PAPER_SWAP)
    with sv.State(n, sv.SV_C64) as s:
        s.apply(g, cfg)
        st = s.stats()
        idx, p = s.argmax(info["mask"])
    assert idx == info["y"] and abs(p - 1.0) <= 1e-5
    assert st["remaps"] == sv.sv_plan_export(n, sv.SV_C64, without_leading_x(g), cfg)["remaps"]


def window_circuit(n, windows, per, seed):
    """Non-diagonal gates (U, X, controlled U) inside qubit windows, one
    window after another: each window is one tile pass's local set.  Every
    gate acts on the qubit the previous gate ended on, so no planner can
    reorder them: floating-point results depend on the order of gates even
    where they commute.  No Hadamards: a tile pass scales its unnormalised
    Hadamards once, by a factor that depends on how many the pass holds."""
    rng = np.random.default_rng(seed)
    recs = []
    cur = 0
    for w in windows:
        if cur not in w:
            cur = w[0]
        for _ in range(per):
            r = rng.random()
            if r < 0.45:  # an explicit 2x2 (complex64 plans split U3 into phases and a rotation)
                recs.append(C.u(cur, C.random_unitary(rng)))
            elif r < 0.55:
                recs.append(C.x(cur))
            else:
                b = int(rng.choice([q for q in w if q != cur]))
                recs.append(C.cu(cur, b, C.random_unitary(rng)))
                cur = b
    return C.gates(recs)


@pytest.mark.parametrize("dt,flags", [(1, 0), (0, 8)])
def test_remap_points_do_not_change_amplitudes(sv, orc, dt, flags):
    """Reading A12: two plans of the same gates, in the same order, whose
    passes differ only in where the qubits are brought together - explicit
    remap passes before the passes (the paper's global-local SWAPs,
    SV_FLAG_PAPER_SWAP) or tiles gathered from the qubits where they lie -
    apply the same arithmetic to every amplitude, so the amplitudes are
    identical bit for bit (complex128 and complex64 on the generic tile
    kernel; no diagonal gates, whose grouping into phase factors may differ
    between the plans)."""
    n, k = 16, 12
    windows = [list(range(0, 11)) + [11 + p] for p in range(5)]
    g = window_circuit(n, windows, 40, 7 + dt)
    outs, stats = [], []
    for extra in (0, sv.SV_FLAG_PAPER_SWAP):
        with sv.State(n, dt) as s:
            s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=k, flags=flags | extra))
            stats.append(s.stats())
            outs.append(s.amplitudes())
    assert stats[0]["remaps"] == 0 and stats[1]["remaps"] > 0
    assert np.array_equal(outs[0], outs[1])
    ref = orc.run(n, g)
    assert np.max(np.abs(outs[0] - ref)) <= (1e-12 if dt == 1 else 2e-5)
