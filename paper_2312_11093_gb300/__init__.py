"""GB300-native MGCNN solver hot path (arXiv 2312.11093).

The compute path lives in the CUDA library `libmgcnn.so` (sources under
`csrc/`, C ABI in `include/mgcnn.h`); `mgcnn` is its thin ctypes binding.
Submodules are imported lazily so that `inputs` can be used without the
library.
"""
