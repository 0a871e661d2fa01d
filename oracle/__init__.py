"""CPU oracle of the discrete-continuous stereo method (test infrastructure only).

Imported only by the tests, the smoke check and the benchmark's CPU-baseline
leg; the CUDA product never uses it.
"""
