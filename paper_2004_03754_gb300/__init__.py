"""GB300-native electromagnetic PIC step with the customised dual-stencil
field solver of Li et al. (arXiv:2004.03754).

The compute path lives in the CUDA library ``libpic.so`` (see ``include/pic.h``);
``paper_2004_03754_gb300.pic`` is its thin Python binding.
"""
__all__ = ["pic", "inputs", "coeffs"]
