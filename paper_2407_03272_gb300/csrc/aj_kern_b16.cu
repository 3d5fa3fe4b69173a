// Persistent fused AJ kernel, PolB16 precision policy.
#define AJ_POL PolB16
#define AJ_SUFFIX b16
#include "aj_kern_inst.cuh"
