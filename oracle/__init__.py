"""FP64 CPU oracle of the Lagrange-flux scheme (arXiv:1607.08710).

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product package.
"""
