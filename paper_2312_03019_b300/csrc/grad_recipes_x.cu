// grad_recipes_x.cu -- the adjoint sweep's compiled first and last passes and the fused pass of
// 7-bit high groups (grad_kernel<float, ..., grad_recipe(r)..., grad_masks(r, v)>), complex64
// only, one translation unit.
#include "kernels.cuh"

#define QAOA_OWN_GRAD_RECIPES_X
#include "instances.h"
#undef QAOA_INSTANCE
#define QAOA_INSTANCE template
QAOA_GRAD_RECIPE_X_INSTANCES(float, 12, 4)
