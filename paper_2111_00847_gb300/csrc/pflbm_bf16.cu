// BF16-deviation storage instantiation of the device path (FP32 arithmetic).
#include "pflbm_launch.cuh"

namespace pflbm {
PFLBM_INSTANTIATE_DEV(PopDev<__nv_bfloat16>)
}  // namespace pflbm
