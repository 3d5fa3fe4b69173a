// Persistent fused AJ kernel, PolF32 precision policy.
#define AJ_POL PolF32
#define AJ_SUFFIX f32
#include "aj_kern_inst.cuh"
