"""GB300-native (sm_103a) library for the hot path of "High-order Differentiable
Autoencoder for Nonlinear Model Reduction" (Shen et al.): decoder derivatives by
stacked complex-step columns, complex-step backpropagation, cubature-weighted
reduced assembly and the reduced implicit-Euler Newton step.

``paper_2102_11026_gb300.dae`` is the ctypes binding of the C-ABI library
(``include/dae.h``); ``synth`` builds seeded synthetic inputs.  Importing the
package does not load the CUDA library; the binding loads it on first use and
raises if it is missing.
"""
__all__ = ["dae", "synth"]
