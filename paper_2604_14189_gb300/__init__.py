"""GB300-native 2D finite-difference wave solvers (acoustic + elastic) with
exact discrete adjoints, after SWEEP (Wang & Alkhalifah).

The compute path is the C-ABI library ``libsweep.so`` (hand-written CUDA for
sm_103a, declared in ``include/sweep.h``); ``sweep`` is its thin ctypes
binding.  Import ``paper_2604_14189_gb300.sweep`` to load the library; this
package initialiser loads nothing so that ``inputs`` can be used on its own.
"""
