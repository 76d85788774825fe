"""GB300-native hot path of randomized DOT inversion with simultaneous sources and detectors.

The compute path lives in a C-ABI shared library (libdot.so, hand-written CUDA for
sm_103a); `paper_1706_05586_gb300.dot` is the thin ctypes binding over it.  Importing
this package does not load the library; the binding does, and fails loudly if the
library is missing.
"""
