"""GB300-native H-matrix displacement-discontinuity BEM hot path.

libhmat.so (CUDA sm_103a + host C++) holds every step of the path; `hmat` is its thin
ctypes binding and `synth` the seeded synthetic-input generator.  Importing the
package does not load the library; `hmat.lib()` does, and raises if it is missing.
"""
