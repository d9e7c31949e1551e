"""B300-native (sm_103a) chunk-coding hot path of the paper "Ultra-Fast Neural Video Compression".

The compute lives in ``libufvc.so`` (C ABI declared in ``include/ufvc.h``); :mod:`.ufvc` is its thin
ctypes binding.  Import :mod:`paper_2606_04410_b300.ufvc` to load the library (it fails loudly if the
library is missing).
"""
