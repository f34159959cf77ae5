// tile_c128.cu -- complex128 pass kernels (tile_kernel<double, 12, 4, ...>, recipes included), one
// translation unit.
#include "kernels.cuh"

#define QAOA_OWN_TILE_C128
#include "instances.h"
#undef QAOA_INSTANCE
#define QAOA_INSTANCE template
QAOA_TILE_INSTANCES(double, 12, 4)
QAOA_RECIPE_INSTANCES(double, 12, 4)
