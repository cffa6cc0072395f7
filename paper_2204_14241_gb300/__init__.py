"""GB300-native pseudofermion HMC hot path for the O(3) spin-fermion model
(arXiv:2204.14241). The compute path is the CUDA library ``libhmc`` behind a C ABI
(``include/hmc.h``); ``hmc`` is its thin Python binding. The library is loaded on
first use, and a missing library raises instead of falling back to anything else.
"""
