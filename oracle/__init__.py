"""FP64 CPU oracle of the moving-mesh hot path: TEST INFRASTRUCTURE ONLY.

Importable by the tests, the smoke check and the benchmark's CPU-baseline leg;
the product package never imports it.
"""
