// FP64 instantiation of the kernels in blend_kernels.cuh (namespace sesc::fp64):
// every operation of the right-hand side in double precision; and the adjoint
// kernels of adjoint_kernels.cuh (FP64 only).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <atomic>

#include "kparams.h"
#include "opgen.h"

#define SESC_REAL double
#define SESC_NS fp64
#include "blend_kernels.cuh"
#include "adjoint_kernels.cuh"
