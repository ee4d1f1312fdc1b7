"""sv_marginal_noalloc: the read-out for callers that cannot allocate device memory.

Checks, through the C ABI, that the allocation-free marginal (partial sums in
a fixed device array compiled into the library) gives the same renormalised
probabilities as sv_probabilities_device, which allocates its own scratch,
on two calls in a row (the second call finds the first call's partial sums
still in the shared array).  Runs last so that a failure here leaves every
other test already run.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_15098_gb300 import circuits as C

pytestmark = pytest.mark.gpu

TOL = 1e-13  # same bound as the read-out parity tests


@pytest.fixture(scope="module")
def sv():
    import torch

    assert torch.cuda.is_available()
    from paper_2605_15098_gb300 import build as B
    B.build()
    from paper_2605_15098_gb300 import sv as mod
    return mod


def circuit(n):
    recs = list(C.random_circuit(n, 3, 4242))
    # SWAPs make the qubit map a non-trivial permutation in partitioned mode
    recs += [C.swap(0, n - 1), C.swap(2, n - 3), C.h(1), C.cp(1, n - 2, 0.37)]
    return C.gates(recs)


@pytest.mark.parametrize("dtype", [0, 1])
def test_noalloc_matches_allocating_readout(sv, dtype):
    import torch

    n = 15
    masks = [0b111111, (1 << n) - 1, 1 << (n - 1), 0b101000110010101, 1]
    with sv.State(n, dtype) as s:
        s.apply(circuit(n), sv.make_config(sv.SV_MODE_PARTITIONED, tile_qubits=9, chunk_qubits=3))
        n_, dt_, dev = sv.sv_info(s.h)
        phys = sv.sv_qubit_map(s.h)
        assert phys != list(range(n))
        for mask in masks:
            m = bin(mask).count("1")
            ref = torch.empty(1 << m, dtype=torch.float64, device="cuda")
            sv.sv_probabilities_device(s.h, mask, ref.data_ptr())
            torch.cuda.synchronize()
            ref_h = ref.cpu().numpy()
            assert abs(ref_h.sum() - 1.0) < 1e-12
            for call in range(2):
                out = torch.full((1 << m,), float("nan"), dtype=torch.float64, device="cuda")
                sv.sv_marginal_noalloc(dev, n, dt_, phys, mask, out.data_ptr(), 0)
                torch.cuda.synchronize()
                got = out.cpu().numpy()
                assert np.all(np.isfinite(got)), (mask, call)
                assert np.max(np.abs(got - ref_h)) <= TOL, (mask, call)


def test_noalloc_large_masks_and_no_allocation(sv):
    """n = 22 complex64 under a permuted qubit map: a 10-qubit mask that
    holds physical bit 0 (outcome bits low), a 6-qubit mask of high physical
    bits (outcome bits high, the warp-per-outcome kernel) and an 18-qubit
    mask (one group: the caller's buffer takes the sums directly), each
    against sv_probabilities_device on two calls in a row.  After a warm-up
    call, further calls leave the device's free memory unchanged."""
    import torch

    n = 22
    with sv.State(n, sv.SV_C64) as s:
        s.apply(circuit(n), sv.make_config(sv.SV_MODE_PARTITIONED))
        _, dt_, dev = sv.sv_info(s.h)
        phys = sv.sv_qubit_map(s.h)
        logical_of = {p: q for q, p in enumerate(phys)}

        def mask_of_phys(bits):
            return sum(1 << logical_of[b] for b in bits)

        masks = [mask_of_phys(range(10)), mask_of_phys(range(n - 6, n)),
                 mask_of_phys([b for b in range(n) if b not in (3, 7, 11, 19)])]
        outs = {}
        for mask in masks:
            m = bin(mask).count("1")
            ref = torch.empty(1 << m, dtype=torch.float64, device="cuda")
            sv.sv_probabilities_device(s.h, mask, ref.data_ptr())
            torch.cuda.synchronize()
            ref_h = ref.cpu().numpy()
            outs[mask] = torch.empty(1 << m, dtype=torch.float64, device="cuda")
            for call in range(2):
                outs[mask].fill_(float("nan"))
                sv.sv_marginal_noalloc(dev, n, dt_, phys, mask, outs[mask].data_ptr(), 0)
                torch.cuda.synchronize()
                got = outs[mask].cpu().numpy()
                assert np.all(np.isfinite(got)), (m, call)
                assert np.max(np.abs(got - ref_h)) <= TOL, (m, call)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            for mask in masks:
                sv.sv_marginal_noalloc(dev, n, dt_, phys, mask, outs[mask].data_ptr(), 0)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_bad_arguments(sv):
    import torch

    lib = sv.lib()
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    st = torch.empty(8, dtype=torch.complex64, device="cuda")
    bad_map = (ctypes.c_int * 3)(0, 0, 2)
    calls = [
        (None, 3, 0, None, 3, out.data_ptr()),          # NULL state
        (st.data_ptr(), 3, 0, None, 3, None),           # NULL output
        (st.data_ptr(), 3, 0, None, 0, out.data_ptr()),  # empty mask
        (st.data_ptr(), 3, 0, None, 1 << 3, out.data_ptr()),  # mask beyond n
        (st.data_ptr(), 3, 5, None, 3, out.data_ptr()),  # bad dtype
        (st.data_ptr(), 3, 0, bad_map, 3, out.data_ptr()),  # not a permutation
    ]
    for dev, n, dt, pm, mask, o in calls:
        rc = lib.sv_marginal_noalloc(ctypes.c_void_p(dev), n, dt, pm, mask, ctypes.c_void_p(o), None)
        assert rc == sv.SV_ERR_ARG, sv.sv_last_error()
