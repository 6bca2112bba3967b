"""GB300-native vectorized Sparrow environment step (paper arxiv 2305.04180).

The simulator, the fused Q-network rollout and the TD learner run in the CUDA
library ``libsparrowgb.so`` (``csrc/``, C ABI in ``include/sparrow_gb.h``).
This package is its Python binding: it marshals arguments, uses PyTorch only
for device memory and streams, and has no CPU fallback.
"""

from .qnet import QNet, Replay
from .sim import Sim, make_config

__all__ = ["Sim", "make_config", "QNet", "Replay"]
