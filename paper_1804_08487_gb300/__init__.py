"""GB300-native global Curveball super step (Carstens et al., "Parallel and
I/O-efficient Randomisation of Massive Networks using Global Curveball Trades").

The hot path runs in the CUDA library ``lib/libcb.so`` (sm_103a) behind the
C ABI declared in ``include/cb.h``; :mod:`.cb` is its thin Python binding and
:mod:`.synth` builds seeded synthetic input graphs.
"""
