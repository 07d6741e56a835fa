"""GB300-native (sm_103a CUDA) ray tracer for unified Gaussian primitives (arXiv 2406.09733).

The compute lives in ``libugp.so`` (C ABI in ``include/ugp.h``); ``ugp`` is its
thin Python binding and ``scenes`` draws seeded synthetic inputs.
"""
