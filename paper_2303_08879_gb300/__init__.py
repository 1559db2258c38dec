"""GB300-native Fock-amplitude recurrence (arXiv 2303.08879): diagonal
(Algorithm 1) and conditional (Algorithm 2) walks with reverse-mode VJPs,
behind the C ABI of include/fockdiag.h.

Submodules are imported lazily so that ``inputs`` (the seeded workload
generator) works without the compiled library; every compute entry point
raises ``FockError`` when libfockdiag.so is missing.
"""
__all__ = ["fockdiag", "autograd", "inputs", "build"]
