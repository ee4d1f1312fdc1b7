"""A reset records |0...0> without writing it; X and H gates that come first
on their qubit only change the recorded product state H^{hq}|b> (X flips a
bit of b, H toggles a qubit of hq), and the first register-stage pass
generates the state instead of reading it (GPU).  Checked against the FP64
oracle, including what the adopted device buffer holds."""
import numpy as np
import pytest

from gen import fold_leading, mixed_circuit, without_leading_x
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


def tol(sv, dt):
    return 1e-12 if dt == sv.SV_C128 else 2e-5


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [3, 14, 17])
def test_leading_x_gates(sv, orc, n, dt):
    rng = np.random.default_rng(n + 7 * dt)
    xs = [C.x(int(q)) for q in rng.choice(n, size=min(n, 5), replace=False)]
    body = mixed_circuit(n, 80, n + 1)
    g = C.gates(xs + list(body) + [C.x(0), C.x(n - 1)])  # trailing X are real gates
    ref = orc.run(n, g)
    for mode in (sv.SV_MODE_PARTITIONED, sv.SV_MODE_PERGATE):
        with sv.State(n, dt) as s:
            s.apply(g, sv.make_config(mode))
            got = s.amplitudes()
        assert np.max(np.abs(got - ref)) <= tol(sv, dt)


@pytest.mark.parametrize("dt", [0, 1])
def test_only_x_gates_stay_a_basis_state(sv, orc, dt):
    n = 16
    g = C.gates([C.x(1), C.x(7), C.swap(7, 9), C.x(15), C.x(1)])
    ref = orc.run(n, g)
    with sv.State(n, dt) as s:
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED))
        assert s.stats()["passes"] == 0
        idx, p = s.argmax((1 << n) - 1)
        assert idx == int(np.argmax(np.abs(ref))) and p == 1.0
        got = s.amplitudes()
    assert np.array_equal(got, ref.astype(got.dtype))


def test_adopted_buffer_after_reset(sv):
    """sv_info hands out the device pointer only after writing the state."""
    import torch

    n = 12
    buf = torch.full((1 << n,), 3.0 + 1j, dtype=torch.complex64, device="cuda")
    with sv.State(n, sv.SV_C64, tensor=buf) as s:
        s.reset()
        sv.sv_info(s.h)
        torch.cuda.synchronize()
        host = buf.cpu().numpy()
        assert host[0] == 1 and np.all(host[1:] == 0)


def test_qpe_first_pass_generates(sv, orc):
    n = 20
    g, expected, info = C.qpe(n, seed=2)
    ref = orc.run(n, g)
    with sv.State(n, sv.SV_C64) as s:
        sv.sv_profile(s.h, True)
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED))
        recs = sv.sv_profile_read(s.h)
        st = s.stats()
        got = s.amplitudes()
    tiles = [r for r in recs if r["kind"] == sv.SV_KERNEL_TILE]
    state_bytes = 8 * (1 << n)
    assert tiles[0]["bytes"] == state_bytes and all(r["bytes"] == 2 * state_bytes for r in tiles[1:])
    assert st["sweep_bytes"] == sum(r["bytes"] for r in tiles)
    fid = abs(np.vdot(ref, got.astype(np.complex128))) ** 2
    assert 1 - fid <= 1e-6


@pytest.mark.parametrize("n,seed", [(14, 1), (16, 2), (19, 3)])
def test_leading_hadamards_are_generated(sv, orc, n, seed):
    """Leading Hadamards (on local and global qubits alike) fold into the
    recorded state and the first pass generates H^{hq}|b>; the same list on a
    state that is not a recorded one applies them."""
    rng = np.random.default_rng(seed)
    xs = [int(q) for q in rng.choice(n, size=n // 2, replace=False)]
    hs = [int(q) for q in rng.choice(n, size=n - 3, replace=False)]
    body = mixed_circuit(n, 60, seed + 40, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 9, 10))  # no CU
    g = C.gates([C.x(q) for q in xs] + [C.h(q) for q in hs] + list(body) + [C.h(q) for q in hs])
    ref = orc.run(n, g)
    basis, hq, rest = fold_leading(g)
    hs_mask = sum(1 << q for q in hs)
    assert hq & hs_mask == hs_mask and len(rest) <= len(g) - len(xs) - len(hs)
    with sv.State(n, sv.SV_C64) as s:
        sv.sv_profile(s.h, True)
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED))
        recs = sv.sv_profile_read(s.h)
        got = s.amplitudes()
    tiles = [r for r in recs if r["kind"] == sv.SV_KERNEL_TILE]
    assert tiles and tiles[0]["bytes"] == 8 * (1 << n)  # generated: written, not read
    assert abs(np.vdot(ref, got.astype(np.complex128))) ** 2 >= 1.0 - 1e-6
    # the same list on a state that is not a basis state: the Hadamards run
    with sv.State(n, sv.SV_C64) as s:
        s.apply(C.gates([C.h(0)]), sv.make_config(sv.SV_MODE_PERGATE))
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED))
        got2 = s.amplitudes()
    ref2 = orc.run(n, np.concatenate([C.gates([C.h(0)]), g]))
    assert abs(np.vdot(ref2, got2.astype(np.complex128))) ** 2 >= 1.0 - 1e-6


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [5, 15, 18])
def test_recorded_product_state(sv, orc, n, dt):
    """Prefixes of X and H only (H on every qubit, H H on one, X then H, H
    then X, which stays a gate): the recorded state, written by the read-out
    or generated by a following pass, equals the oracle's; a prefix that
    folds entirely leaves no pass to run."""
    pre = [C.h(q) for q in range(n)] + [C.h(2), C.x(3)] + [C.x(1)]
    g_only = C.gates([C.x(0), C.h(0)] + pre[1:])
    body = mixed_circuit(n, 40, n + 3 * dt)
    for g in (g_only, C.gates(list(g_only) + list(body))):
        ref = orc.run(n, g)
        for mode in (sv.SV_MODE_PARTITIONED, sv.SV_MODE_FUSED) if dt == 0 else (sv.SV_MODE_PARTITIONED,):
            with sv.State(n, dt) as s:
                s.apply(g, sv.make_config(mode))
                st = s.stats()
                got = s.amplitudes()
            assert np.max(np.abs(got - ref)) <= tol(sv, dt)
            if len(g) == len(g_only):
                # every gate folds but the X on qubit 3, which follows its H
                assert st["passes"] >= 1 and st["gates"] == len(g)


