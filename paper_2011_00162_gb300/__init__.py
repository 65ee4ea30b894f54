"""GB300 (sm_103a) implementation of the OD2P frame update and ADMM iteration.

Method: Chang, Glowinski, Marchesini, Tai, Wang, Zeng, "Overlapping Domain
Decomposition Methods for Ptychographic Imaging", arXiv:2011.00162.

The compute path is the CUDA library ``libod2p.so`` (C ABI in include/od2p.h);
:mod:`.api` marshals torch tensors to it, :mod:`.autograd` wraps the ST-AGM
loss as a differentiable function, :mod:`.synth` makes seeded inputs and
:mod:`.autotune` picks the frame update's launch shape per workload and caches
it on disk; :mod:`.adaptive` rebalances the consensus penalty between
iterations.
"""
from .api import *  # noqa: F401,F403
from .api import __all__ as _api_all
from . import adaptive, autotune  # noqa: F401

__all__ = list(_api_all)
