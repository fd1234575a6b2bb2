"""GB300-native Kronecker payoff products for poker river endgames.

Implements the data-parallel hot path of Farina & Sandholm, "Fast Payoff
Matrix Sparsification Techniques for Structured Extensive-Form Games"
(AAAI-22): the products A*y and A^T*x of Prop. 1, evaluated in Kronecker form
by hand-written sm_103a kernels behind the C ABI of ``include/kps.h``.
"""
__all__ = ["kps", "synth", "build"]
