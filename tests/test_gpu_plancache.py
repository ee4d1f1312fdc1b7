"""The handle's cache of compiled programmes (sv_apply_circuit, partitioned
modes): a repeated (gate list, configuration, qubit map) key reuses the
planned, compiled and uploaded programme, and every result still matches the
FP64 oracle (complex128 1e-12, complex64 fidelity >= 1 - 1e-6).
"""
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


def close(sv, dtype, got, ref):
    if dtype == sv.SV_C128:
        return float(np.max(np.abs(got - ref))) <= 1e-12
    f = abs(np.vdot(ref, got.astype(np.complex128))) ** 2
    return 1.0 - f <= 1e-6


@pytest.mark.parametrize("dtype", [0, 1])
def test_repeat_hits_and_matches(sv, orc, dtype):
    n = 17
    g = mixed_circuit(n, 200, 71 + dtype)
    ref = orc.run(n, g)
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=13 if dtype == sv.SV_C64 else 12)
    with sv.State(n, dtype) as s:
        s.apply(g, cfg)
        first = s.amplitudes()
        up1 = s.stats()["h2d_bytes"]
        s.reset()
        s.apply(g, cfg)
        second = s.amplitudes()
        up2 = s.stats()["h2d_bytes"]
    assert up1 > 0 and up2 == 0  # the second call uploads nothing
    assert np.array_equal(first, second)
    assert close(sv, dtype, second, ref)


def test_bypass_flag_recompiles(sv):
    n = 16
    g, _, _ = C.qpe(n)
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, flags=sv.SV_FLAG_NO_PLAN_CACHE)
    with sv.State(n, sv.SV_C64) as s:
        for _ in range(2):
            s.reset()
            s.apply(g, cfg)
            assert s.stats()["h2d_bytes"] > 0


def test_qubit_map_is_part_of_the_key(sv, orc):
    """A list with SWAPs changes the qubit map, so applying it again without
    a reset starts from another map: a different programme, and the result
    of both applications still matches the oracle."""
    n = 16
    g = C.gates([C.h(q) for q in range(n)] + [C.swap(0, 15), C.swap(3, 9)]
                + [C.cpk(q, (q + 5) % n, 1, 3 + q % 4) for q in range(n)] + [C.h(2), C.h(14)])
    ref = orc.run(n, np.concatenate([g, g]))
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED)
    with sv.State(n, sv.SV_C64) as s:
        s.apply(g, cfg)
        s.apply(g, cfg)
        assert s.stats()["h2d_bytes"] > 0  # not the first call's programme
        got = s.amplitudes()
    assert close(sv, sv.SV_C64, got, ref)


def test_many_keys_evict_and_stay_correct(sv, orc):
    """More distinct lists than the cache holds, then the first again."""
    n = 15
    circuits = [mixed_circuit(n, 80, 500 + i) for i in range(10)]
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED)
    with sv.State(n, sv.SV_C64) as s:
        for g in circuits + circuits[:2]:
            s.reset()
            s.apply(g, cfg)
            assert close(sv, sv.SV_C64, s.amplitudes(), orc.run(n, g))
