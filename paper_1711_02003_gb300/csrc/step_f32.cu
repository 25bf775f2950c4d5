// step_f32.cu -- the step kernels and launchers for FP32 storage (one translation unit
// per storage format, compiled in parallel)
#include "lbcg_internal.h"
#define LBCG_STEP_PREC LBCG_FP32
#include "step_kernels.cuh"
