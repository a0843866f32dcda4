"""CPU FP64 oracle of the H-matrix DD-BEM hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check in __graft_entry__ and the
benchmark's CPU-baseline leg may import anything in this package.  It shares no code
with the CUDA library and never imports it.
"""
