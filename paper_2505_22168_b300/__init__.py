"""B300-native GMNN energies, forces and parameter gradients (libgm, sm_103a).

The compute path is libgm.so (CUDA kernels behind the C ABI of include/gm.h); this
package only marshals PyTorch device buffers and streams into it.
"""
from ._lib import GmError, load  # noqa: F401
from .gmnn import (GMNN, DeviceSystem, GMNNFunction, MDParams, MDState, NeighborList, pack_theta,  # noqa: F401
                   unpack_theta)
