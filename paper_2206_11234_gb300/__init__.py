"""GB300-native importance-sampled first-passage-time simulation.

Hot path of arXiv:2206.11234 (§2): biased Euler–Maruyama runs of the
slow-roll stochastic-inflation Langevin equation until first passage, with
Girsanov log-weights and weighted histograms of the first-passage time, as
hand-written sm_103a CUDA kernels behind the C ABI declared in include/fpt.h.

Importing this package loads nothing; ``paper_2206_11234_gb300.native``
loads the CUDA library and raises if it is missing.
"""
__all__ = ["native", "workloads"]
