"""GB300-native dense state-vector simulation with state partitioning.

Re-design for one NVIDIA GB300 (sm_103a) of the method of arxiv 2605.15098
("Accelerating State-Vector Quantum Simulation on Integrated GPUs via Cache
Locality Optimization").  The compute path is the CUDA library ``libsv``
behind a C ABI (``include/sv.h``); ``paper_2605_15098_gb300.sv`` is its thin
ctypes binding and ``paper_2605_15098_gb300.circuits`` builds the seeded
benchmark circuits.
"""
__all__ = ["circuits", "sv"]
