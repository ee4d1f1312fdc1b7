"""A reset records |0...0> without writing it; X gates that come first on
their qubit only flip the recorded basis index, and the first register-stage
pass generates the state instead of reading it (GPU).  Checked against the
FP64 oracle, including what the adopted device buffer holds."""
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
