"""GB300-native prior-predictive Monte Carlo (ABC rejection and Bayesian
p-values), after Warne, Sisson & Drovandi, arXiv:1902.09046.

The compute path is the C-ABI library ``libppabc.so`` built from ``csrc/``
(hand-written sm_103a CUDA kernels); ``binding`` marshals torch tensors into
it.  Importing this package does not load the library: the first call into
``binding`` does, and it raises if the library is missing or no GB300-class
device is present.  There is no CPU fallback.
"""

__all__ = ["binding", "workloads"]
