"""GB300-native (sm_103a) genetic algorithm step for Hadamard matrices
(Balogh & Ruiz, arXiv 2208.14961).

The compute lives in libhadga.so (CUDA, built by ``build.build()``) behind
the C ABI of include/hadga.h; ``hadga`` is its ctypes binding.
"""
