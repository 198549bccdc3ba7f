"""GB300-native batched GCP-CROWN bound propagation (arXiv 2208.05740).

The compute path lives in ``libgcp.so`` (hand-written CUDA for sm_103a behind
the C ABI declared in ``include/gcp.h``); ``gcp`` is its thin Python binding.
"""
