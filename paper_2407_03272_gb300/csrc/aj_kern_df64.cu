// Persistent fused AJ kernel, PolDF64 precision policy.
#define AJ_POL PolDF64
#define AJ_SUFFIX df64
#include "aj_kern_inst.cuh"
