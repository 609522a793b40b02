"""GB300-native stable LSD radix sort of 32-bit keys (optionally with 32-bit values).

The sort itself runs in hand-written CUDA kernels behind the C ABI of
``librs.so`` (declared in ``include/rs.h``); ``paper_1008_2849_gb300.rs`` is the
thin Python binding with the same names.  Submodules are imported on demand,
so that ``paper_1008_2849_gb300.inputs`` (seeded synthetic inputs) imports on
machines without a GPU.
"""
