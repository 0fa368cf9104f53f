"""Serial oracle of the operator-split reaction-diffusion method.

TEST INFRASTRUCTURE ONLY: imported by the tests, the package smoke check and
the benchmark's CPU-baseline leg, never by the CUDA path.
"""
