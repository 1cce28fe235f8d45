"""Paraexp direct-adjoint gradients on GB300 (Skene, Eggl & Schmid, arXiv 2004.00546).

The compute path is the C-ABI library ``libpxa.so`` (hand-written CUDA for
sm_103a); ``paper_2004_00546_gb300.pxa`` is its ctypes binding. Importing this
package does not load the library; ``pxa.load()`` does, and fails loudly when it
is missing.
"""
__all__ = ["inputs"]
