// batch_c64.cu -- the packed (tile_batch_kernel) complex64 pass kernels of the request server's
// mid-size states, one translation unit.
#include "kernels.cuh"

#define QAOA_OWN_BATCH_C64
#include "instances.h"
#undef QAOA_INSTANCE
#define QAOA_INSTANCE template
QAOA_BATCH_INSTANCES(float, 13, 5)
