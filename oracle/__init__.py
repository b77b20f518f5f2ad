"""CPU oracle (FP64, numpy): test infrastructure only.

Imported by the tests, by the smoke check and by the benchmark's CPU
baseline.  The product library never imports it and it never imports the
product library.
"""
