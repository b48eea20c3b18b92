// FP64 instantiation of the device path.
#include "pflbm_launch.cuh"

namespace pflbm {
PFLBM_INSTANTIATE(double)
}  // namespace pflbm
