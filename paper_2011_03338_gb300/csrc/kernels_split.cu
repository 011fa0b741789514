// FP32-split instantiation of the kernels in blend_kernels.cuh (namespace
// sesc::split): reconstruction, nodal and interface fluxes and operator passes in
// FP32 accumulated in FP32; the indicator ratio, the squeezing formula, the
// permissibility checks of face states, the flux-difference assembly and the RK
// stage in FP64 (the state stays FP64).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <atomic>

#include "kparams.h"
#include "opgen.h"

#define SESC_REAL float
#define SESC_NS split
#include "blend_kernels.cuh"
#include "adjoint_kernels.cuh"
