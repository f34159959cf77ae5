// tile_c64.cu -- complex64 pass kernels (tile_kernel<float, 13, 5, ...>), one translation unit.
#include "kernels.cuh"

#define QAOA_OWN_TILE_C64
#include "instances.h"
#undef QAOA_INSTANCE
#define QAOA_INSTANCE template
QAOA_TILE_INSTANCES(float, 13, 5)
