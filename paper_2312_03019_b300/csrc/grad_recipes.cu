// grad_recipes.cu -- adjoint-sweep pass kernels specialised to the compiled sweep programs
// (grad_kernel<float, ..., grad_recipe(r)...>), complex64 only, one translation unit.
#include "kernels.cuh"

#define QAOA_OWN_GRAD_RECIPES
#include "instances.h"
#undef QAOA_INSTANCE
#define QAOA_INSTANCE template
QAOA_GRAD_RECIPE_INSTANCES(float, 12, 4)
