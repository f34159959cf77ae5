// grad_recipes_m.cu -- the compiled sweep programs with their RXD masks compiled in
// (grad_kernel<float, ..., grad_recipe(r)..., grad_masks(r, v)>), complex64 only, one translation unit.
#include "kernels.cuh"

#define QAOA_OWN_GRAD_RECIPES_M
#include "instances.h"
#undef QAOA_INSTANCE
#define QAOA_INSTANCE template
QAOA_GRAD_RECIPE_M_INSTANCES(float, 12, 4)
