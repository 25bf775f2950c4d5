// step_f16.cu -- the step kernels and launchers for scaled FP16 storage (one translation unit
// per storage format, compiled in parallel)
#include "lbcg_internal.h"
#define LBCG_STEP_PREC LBCG_FP16_SCALED
#include "step_kernels.cuh"
