"""dexgb: GB300-native formal solution of the radiative transfer equation accelerated by
sparse block grids, variance-limited mipmapping and hierarchical DDA (arxiv 2511.08498).

The compute path is ``libdexgb.so`` (hand-written CUDA for sm_103a behind the C ABI in
``include/dexgb.h``); ``paper_2511_08498_gb300.api`` is its ctypes binding.  Importing
this package loads nothing; the first API call loads the library and raises if it cannot.
"""
