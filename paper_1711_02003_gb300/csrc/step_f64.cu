// step_f64.cu -- the step kernels and launchers for FP64 storage (one translation unit
// per storage format, compiled in parallel)
#include "lbcg_internal.h"
#define LBCG_STEP_PREC LBCG_FP64
#include "step_kernels.cuh"
