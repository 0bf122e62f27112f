"""FP64 CPU oracle of the adaptive-force-update gravity path.

Test infrastructure only: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.
"""
