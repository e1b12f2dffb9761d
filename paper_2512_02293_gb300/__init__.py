"""GB300-native differentiable Gaussian-splatting mapping step (VIGS-SLAM, Sec. 3.3).

The compute path is the C-ABI library ``libgs`` (CUDA for sm_103a, built from
``csrc/``); :mod:`.gs` is its thin Python binding.  Importing the package does
not load the library: the first call into :mod:`.gs` does, and raises if the
library is missing.
"""
__all__ = ["gs", "synth"]
