// step_f32dev.cu -- the step kernels and launchers for FP32 deviation storage (one translation unit
// per storage format, compiled in parallel)
#include "lbcg_internal.h"
#define LBCG_STEP_PREC LBCG_FP32_DEV
#include "step_kernels.cuh"
