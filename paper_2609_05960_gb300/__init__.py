"""GB300-native engine for gate-level time-based power analysis.

The compute path is the CUDA library ``libgtpower.so`` (sources in ``csrc/``,
C ABI in ``include/gtpower.h``); ``gtpower`` is its ctypes binding and
``autograd`` wraps the adjoint for PyTorch.
"""
from .gtpower import Engine, GtpError, load  # noqa: F401
from .autograd import peak_loss, power_waveform  # noqa: F401

__all__ = ["Engine", "GtpError", "load", "power_waveform", "peak_loss"]
