// grad_pf_w.cu -- the persistent prefetching forms of the compiled complex64 sweep programs for
// edge-weighted graphs (grad_pf_kernel<12, 4, true, grad_recipe(r)..., grad_masks(r, v)>), one
// translation unit.
#include "kernels.cuh"

#define QAOA_OWN_GRAD_PF_W
#include "instances.h"
#undef QAOA_INSTANCE
#define QAOA_INSTANCE template
QAOA_GRAD_PF_INSTANCES(12, 4, true)
