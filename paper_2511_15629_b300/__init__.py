"""B300-native discretized stochastic DP for energy-storage arbitrage.

The compute path is the CUDA library ``libesdp.so`` (built from ``csrc/``)
behind a C ABI; ``esdp`` is its thin ctypes binding and ``autograd`` the
torch.autograd.Function over the solve and its adjoint.  Importing the package does not load the library.
"""
__all__ = ["instances", "esdp", "autograd"]
