"""The paper's partitioned CPU simulation (Sec. III-B), the second CPU
baseline: against the FP64 oracle on the paper's gate kinds, over block sizes
from a few qubits to the whole state (CPU only)."""
import numpy as np
import pytest

from gen import mixed_circuit
from paper_2605_15098_gb300 import circuits as C
from paper_2605_15098_gb300 import cpupart


@pytest.mark.parametrize("n,l", [(8, 3), (10, 4), (12, 6), (12, 12)])
def test_qpe(orc, n, l):
    g, expected, info = C.qpe(n, seed=n)
    ref = orc.run(n, g)
    got, st = cpupart.run(n, g, l)
    assert np.max(np.abs(got - ref)) <= 1e-12
    if l < n - 4:  # counting qubits above the block: the eigenstate gates force swaps
        assert st["swaps"] > 0


@pytest.mark.parametrize("n,l,seed", [(9, 3, 1), (11, 5, 2), (13, 7, 3)])
def test_mixed(orc, n, l, seed):
    g = mixed_circuit(n, 200, seed, kinds=(0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10))
    ref = orc.run(n, g)
    got, st = cpupart.run(n, g, l)
    assert np.max(np.abs(got - ref)) <= 1e-12
    assert st["passes"] >= 1


def test_random_layers(orc):
    n, l = 12, 5
    g = C.random_circuit(n, 6, 3)
    ref = orc.run(n, g)
    got, _ = cpupart.run(n, g, l)
    assert np.max(np.abs(got - ref)) <= 1e-12


def test_rejects_general_gates():
    g = C.gates([C.h(0), C.mcu([1, 2], 0, np.eye(2))])
    with pytest.raises(ValueError):
        cpupart.run(4, g, 2)
