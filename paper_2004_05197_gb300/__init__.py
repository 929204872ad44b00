"""GB300 (sm_103a) surrogate-matrix IGA wave library.

The compute path lives in libiga.so (CUDA, C ABI in include/iga.h); ``iga`` is
its thin ctypes binding and ``workloads`` builds the synthetic workloads of the
benchmark from that binding.
"""
