// grad_kernels.cu -- adjoint-sweep pass kernels (grad_kernel<...>) of both precisions, one
// translation unit.
#include "kernels.cuh"

#define QAOA_OWN_GRAD
#include "instances.h"
#undef QAOA_INSTANCE
#define QAOA_INSTANCE template
QAOA_GRAD_INSTANCES(float, 12, 4)
QAOA_GRAD_INSTANCES(double, 12, 4)
