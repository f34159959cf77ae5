// recipes2_c64.cu -- complex64 pass kernels specialised to the programs of the two-group plans
// (recipes 8..12), one translation unit.
#include "kernels.cuh"

#define QAOA_OWN_RECIPE_2G_C64
#include "instances.h"
#undef QAOA_INSTANCE
#define QAOA_INSTANCE template
QAOA_RECIPE_2G_INSTANCES(float, 13, 5)
