"""Failure paths, with every failure made on the host (GPU): an injected
allocation, programme-upload or launch failure returns SV_ERR_OOM or
SV_ERR_CUDA before any kernel writes the state, which stays as it was; the
device error word that a bounded wait sets when it gives up is raised from
the host, and the next read-out reports SV_ERR_TIMEOUT once.  No device wait
is made to run out and nothing faults."""
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
    yield mod
    for site in (mod.SV_FAULT_ALLOC, mod.SV_FAULT_UPLOAD, mod.SV_FAULT_LAUNCH):
        mod.sv_fault_inject(site, -1)


@pytest.fixture(autouse=True)
def disarm(sv):
    yield
    for site in (sv.SV_FAULT_ALLOC, sv.SV_FAULT_UPLOAD, sv.SV_FAULT_LAUNCH):
        sv.sv_fault_inject(site, -1)


def fails_with(sv, code, fn, *args):
    with pytest.raises(sv.SvError) as e:
        fn(*args)
    assert e.value.code == code, sv.sv_last_error()


def test_create_fails_on_allocation(sv):
    sv.sv_fault_inject(sv.SV_FAULT_ALLOC, 0)
    fails_with(sv, sv.SV_ERR_OOM, sv.sv_create, 14, sv.SV_C64)
    h = sv.sv_create(14, sv.SV_C64)  # the site is off again
    sv.sv_destroy(h)


@pytest.mark.parametrize("site,code", [(0, -2), (1, -3), (2, -3)])
@pytest.mark.parametrize("dt", [0, 1])
def test_failed_apply_leaves_the_state(sv, orc, site, code, dt):
    """From the recorded |0...0> (the leading X and H gates fold into it
    first) and from a written state: the failing call returns its code and
    the state reads back unchanged; the same call then succeeds."""
    n = 16
    g, _, info = C.qpe(n, seed=3)
    cfg = sv.make_config(sv.SV_MODE_PARTITIONED, flags=sv.SV_FLAG_NO_PLAN_CACHE)
    with sv.State(n, dt) as s:
        before = s.amplitudes()
        sv.sv_fault_inject(site, 0)
        fails_with(sv, code, s.apply, g, cfg)
        assert np.array_equal(s.amplitudes(), before)
        s.apply(g, cfg)
        ref = orc.run(n, g)
        got = s.amplitudes()
        assert np.max(np.abs(got - ref)) <= (1e-12 if dt == 1 else 2e-5)
        if site == sv.SV_FAULT_ALLOC:
            return  # the handle's buffers now fit: a further call allocates nothing
        # a written state (not a recorded one): unchanged too
        before = got
        sv.sv_fault_inject(site, 0)
        fails_with(sv, code, s.apply, C.gates([C.h(3), C.cz(2, 9)]), cfg)
        assert np.array_equal(s.amplitudes(), before)


def test_launch_failure_midway_and_recovery(sv, orc):
    """A launch refused after the first pass ran: SV_ERR_CUDA, then a reset
    and the same circuit give the right state."""
    n = 20
    g, _, info = C.qpe(n, seed=4)
    with sv.State(n, sv.SV_C64) as s:
        sv.sv_fault_inject(sv.SV_FAULT_LAUNCH, 1)
        fails_with(sv, sv.SV_ERR_CUDA, s.apply, g, sv.make_config(sv.SV_MODE_PARTITIONED))
        s.reset()
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED))
        idx, p = s.argmax(info["mask"])
        assert idx == info["y"] and abs(p - 1) < 1e-5


@pytest.mark.parametrize("readout", ["argmax", "probabilities", "copy_out", "sample", "measurements"])
def test_device_timeout_is_reported_once(sv, readout):
    n = 14
    g, _, info = C.qpe(n, seed=5)
    with sv.State(n, sv.SV_C64) as s:
        s.apply(g, sv.make_config(sv.SV_MODE_PARTITIONED))
        sv.sv_fault_raise_device_flag(s.h)
        calls = {
            "argmax": lambda: s.argmax(info["mask"]),
            "probabilities": lambda: s.probabilities(info["mask"]),
            "copy_out": lambda: s.amplitudes(),
            "sample": lambda: s.sample(info["mask"], np.array([0.25, 0.75])),
            "measurements": lambda: s.measurements(),
        }
        fails_with(sv, sv.SV_ERR_TIMEOUT, calls[readout])
        calls[readout]()  # the word was cleared: the next call succeeds


def test_unknown_site_rejected(sv):
    fails_with(sv, sv.SV_ERR_ARG, sv.sv_fault_inject, 7, 0)
