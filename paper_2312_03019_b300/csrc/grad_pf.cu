// grad_pf.cu -- the persistent prefetching forms of the compiled complex64 sweep programs
// (grad_pf_kernel<12, 4, false, grad_recipe(r)..., grad_masks(r, v)>), unit weights, one
// translation unit.
#include "kernels.cuh"

#define QAOA_OWN_GRAD_PF
#include "instances.h"
#undef QAOA_INSTANCE
#define QAOA_INSTANCE template
QAOA_GRAD_PF_INSTANCES(12, 4, false)
