"""GB300-native differentiable splatting of meshgrid Gaussian surfels (RoGs, arXiv 2405.14342).

The hot path (projection, binning and sorting, compositing, backward, pose
initialisation) runs in hand-written CUDA kernels for sm_103a behind the C-ABI
library ``librogs.so`` (declared in ``include/rogs.h``).  The Python modules
here only marshal arguments:

* ``rogs``      -- ctypes binding with the C-ABI's names
* ``render``    -- ``torch.autograd.Function`` over fwd/bwd and the fused loss
* ``scenes``    -- seeded synthetic inputs (no method arithmetic)
"""
