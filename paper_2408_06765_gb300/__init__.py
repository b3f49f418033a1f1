"""GB300-native (sm_103a) hot path of the QMC Rayleigh-Sommerfeld-integral
(RSI) beam model (arXiv 2408.06765): scrambled-Sobol points, piston and RSI
stage sums, interface transmission and field images, behind the C ABI in
``include/rsi.h``.  The binding is imported lazily so that ``workloads``
can be used without a built library."""

__all__ = ["workloads"]
