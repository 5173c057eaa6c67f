"""GB300-native encrypted quadratic-gradient NAG logistic-regression training.

The compute path is the CUDA library ``libhelr.so`` (built from ``csrc/``) behind
the C ABI declared in ``include/he_lr.h``; ``binding`` marshals arguments to it.
"""
