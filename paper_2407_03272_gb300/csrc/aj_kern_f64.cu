// Persistent fused AJ kernel, PolF64 precision policy.
#define AJ_POL PolF64
#define AJ_SUFFIX f64
#include "aj_kern_inst.cuh"
