// recipes_w_c64.cu -- complex64 pass kernels for edge-weighted graphs specialised to the compiled
// pass recipes, one translation unit.
#include "kernels.cuh"

#define QAOA_OWN_RECIPE_W_C64
#include "instances.h"
#undef QAOA_INSTANCE
#define QAOA_INSTANCE template
QAOA_RECIPE_W_INSTANCES(float, 13, 5)
