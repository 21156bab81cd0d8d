"""GB300 (sm_103a) thermocapillary central-moment phase-field LBM.

``lbm`` is the ctypes binding of the CUDA library (``include/lbm.h``);
``build`` compiles it in-tree.  See Holzer et al., arXiv 2401.03041.
"""
__all__ = ["lbm", "build"]
