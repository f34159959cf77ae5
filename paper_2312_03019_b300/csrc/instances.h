// instances.h -- the heavy kernel template instantiations (the pass kernels, their packed forms and
// the adjoint-sweep kernels), each compiled in a translation unit of its own (tile_c64.cu,
// tile_c128.cu, batch_c64.cu, grad_kernels.cu, grad_recipes.cu, grad_recipes_m.cu, grad_recipes_x.cu, grad_pf.cu, grad_pf_w.cu, ...) so that the library builds
// in parallel.  capi.cu includes this file after
// kernels.cuh with QAOA_INSTANCE = "extern template" (declarations); each instance unit defines
// QAOA_OWN_* for the set it owns and instantiates that set with QAOA_INSTANCE = "template".
// Building this way needs -static-global-template-stub=false (external kernel stubs).
#pragma once

#ifndef QAOA_INSTANCE
#define QAOA_INSTANCE extern template
#endif

#define QAOA_TILE_INSTANCES(real, Q, R)                                                                  \
    namespace qaoa {                                                                                      \
    QAOA_INSTANCE __global__ void tile_kernel<real, Q, R, false, 0, 0>(const __grid_constant__ TileArgs<Q>);                \
    QAOA_INSTANCE __global__ void tile_kernel<real, Q, R, true, 0, 0>(const __grid_constant__ TileArgs<Q>);                 \
    }

#define QAOA_RECIPE_ONE(real, Q, R, r) QAOA_RECIPE_W(real, Q, R, r, false)
#define QAOA_RECIPE_W(real, Q, R, r, w)                                                                   \
    QAOA_INSTANCE __global__ void tile_kernel<real, Q, R, w, recipe_def(r).code, recipe_def(r).nops,         \
                                              recipe_masks<real>(r)>(const __grid_constant__ TileArgs<Q>);

// edge-weighted complex64 passes: the recipes with a phase or <C> op (first, fused, last, and
// the full-mask first and last); plain mixer passes of weighted graphs run the unit-weight ones
#define QAOA_RECIPE_W_INSTANCES(real, Q, R)                                                               \
    namespace qaoa {                                                                                       \
    QAOA_RECIPE_W(real, Q, R, 0, true)                                                                     \
    QAOA_RECIPE_W(real, Q, R, 2, true)                                                                     \
    QAOA_RECIPE_W(real, Q, R, 3, true)                                                                     \
    QAOA_RECIPE_W(real, Q, R, 5, true)                                                                     \
    QAOA_RECIPE_W(real, Q, R, 7, true)                                                                     \
    }

#define QAOA_RECIPE_INSTANCES(real, Q, R)                                                                 \
    namespace qaoa {                                                                                       \
    QAOA_RECIPE_ONE(real, Q, R, 0)                                                                         \
    QAOA_RECIPE_ONE(real, Q, R, 1)                                                                         \
    QAOA_RECIPE_ONE(real, Q, R, 2)                                                                         \
    QAOA_RECIPE_ONE(real, Q, R, 3)                                                                         \
    QAOA_RECIPE_ONE(real, Q, R, 4)                                                                         \
    QAOA_RECIPE_ONE(real, Q, R, 5)                                                                         \
    QAOA_RECIPE_ONE(real, Q, R, 6)                                                                         \
    QAOA_RECIPE_ONE(real, Q, R, 7)                                                                         \
    }

#define QAOA_GRAD_INSTANCES(real, Q, R)                                              \
    namespace qaoa {                                                                  \
    QAOA_INSTANCE __global__ void grad_kernel<real, Q, R, false>(const __grid_constant__ TileArgs<Q>);  \
    QAOA_INSTANCE __global__ void grad_kernel<real, Q, R, true>(const __grid_constant__ TileArgs<Q>);   \
    }

// complex64 passes of the two-group plans (recipes 8..12, runtime masks; recipe 9 has 13 ops and
// uses the second program word)
#define QAOA_RECIPE_2G(real, Q, R, r)                                                                 \
    QAOA_INSTANCE __global__ void tile_kernel<real, Q, R, false, recipe_def(r).code, recipe_def(r).nops, \
                                              recipe_masks<real>(r), recipe_def(r).hi>(                 \
        const __grid_constant__ TileArgs<Q>);
#define QAOA_RECIPE_2G_INSTANCES(real, Q, R)                                                          \
    namespace qaoa {                                                                                   \
    QAOA_RECIPE_2G(real, Q, R, 8)                                                                      \
    QAOA_RECIPE_2G(real, Q, R, 9)                                                                      \
    QAOA_RECIPE_2G(real, Q, R, 10)                                                                     \
    QAOA_RECIPE_2G(real, Q, R, 11)                                                                     \
    QAOA_RECIPE_2G(real, Q, R, 12)                                                                     \
    }

// complex64 adjoint-sweep passes specialised to the compiled sweep programs (unit and edge weights; the
// complex128 ones spill at 255 registers and stay on the interpreting instance)
#define QAOA_GRAD_RECIPE_V(real, Q, R, r, v)                                                             \
    QAOA_INSTANCE __global__ void grad_kernel<real, Q, R, false, grad_recipe(r).code, grad_recipe(r).nops,     \
                                              grad_masks(r, v)>(const __grid_constant__ TileArgs<Q>);          \
    QAOA_INSTANCE __global__ void grad_kernel<real, Q, R, true, grad_recipe(r).code, grad_recipe(r).nops,      \
                                              grad_masks(r, v)>(const __grid_constant__ TileArgs<Q>);
#define QAOA_GRAD_RECIPE(real, Q, R, r) QAOA_GRAD_RECIPE_V(real, Q, R, r, 0)
#define QAOA_GRAD_RECIPE_INSTANCES(real, Q, R)                                                        \
    namespace qaoa {                                                                                   \
    QAOA_GRAD_RECIPE(real, Q, R, 0)                                                                    \
    QAOA_GRAD_RECIPE(real, Q, R, 1)                                                                    \
    QAOA_GRAD_RECIPE(real, Q, R, 2)                                                                    \
    }

// the sweep programs with compiled-in RXD masks (grad_masks: variants 1 and 2)
#define QAOA_GRAD_RECIPE_M_INSTANCES(real, Q, R)                                                      \
    namespace qaoa {                                                                                   \
    QAOA_GRAD_RECIPE_V(real, Q, R, 0, 1)                                                               \
    QAOA_GRAD_RECIPE_V(real, Q, R, 1, 1)                                                               \
    QAOA_GRAD_RECIPE_V(real, Q, R, 1, 2)                                                               \
    }

// the sweep's first and last passes (runtime and full masks) and the fused pass of 7-bit high
// groups (grad_masks variant 3)
#define QAOA_GRAD_RECIPE_X_INSTANCES(real, Q, R)                                                      \
    namespace qaoa {                                                                                   \
    QAOA_GRAD_RECIPE_V(real, Q, R, 3, 0)                                                               \
    QAOA_GRAD_RECIPE_V(real, Q, R, 3, 1)                                                               \
    QAOA_GRAD_RECIPE_V(real, Q, R, 4, 0)                                                               \
    QAOA_GRAD_RECIPE_V(real, Q, R, 4, 1)                                                               \
    QAOA_GRAD_RECIPE_V(real, Q, R, 1, 3)                                                               \
    }

// the persistent prefetching sweep programs (grad_pf_kernel), complex64, unit weights (w =
// false, grad_pf.cu) and edge weights (w = true, grad_pf_w.cu)
#define QAOA_GRAD_PF_ONE(Q, R, w, r, v)                                                               \
    QAOA_INSTANCE __global__ void grad_pf_kernel<Q, R, w, grad_recipe(r).code, grad_recipe(r).nops,        \
                                                 grad_masks(r, v), grad_recipe(r).hi>(                         \
        const __grid_constant__ TileArgs<Q>, uint64_t);
#define QAOA_GRAD_PF_INSTANCES(Q, R, w)                                                               \
    namespace qaoa {                                                                                   \
    QAOA_GRAD_PF_ONE(Q, R, w, 0, 1)                                                                    \
    QAOA_GRAD_PF_ONE(Q, R, w, 1, 0)                                                                    \
    QAOA_GRAD_PF_ONE(Q, R, w, 1, 1)                                                                    \
    QAOA_GRAD_PF_ONE(Q, R, w, 1, 2)                                                                    \
    QAOA_GRAD_PF_ONE(Q, R, w, 1, 3)                                                                    \
    QAOA_GRAD_PF_ONE(Q, R, w, 3, 0)                                                                    \
    QAOA_GRAD_PF_ONE(Q, R, w, 3, 1)                                                                    \
    QAOA_GRAD_PF_ONE(Q, R, w, 4, 0)                                                                    \
    QAOA_GRAD_PF_ONE(Q, R, w, 4, 1)                                                                    \
    QAOA_GRAD_PF_ONE(Q, R, w, 5, 0)                                                                    \
    QAOA_GRAD_PF_ONE(Q, R, w, 6, 0)                                                                    \
    QAOA_GRAD_PF_ONE(Q, R, w, 7, 0)                                                                    \
    QAOA_GRAD_PF_ONE(Q, R, w, 8, 0)                                                                    \
    }

// packed mid-size requests of the server: the complex64 two-group programs (recipes 8..12) and the
// interpreting program, unit weights
#define QAOA_BATCH_ONE(real, Q, R, r)                                                                 \
    QAOA_INSTANCE __global__ void tile_batch_kernel<real, Q, R, false, recipe_def(r).code, recipe_def(r).nops, \
                                                    recipe_masks<real>(r), recipe_def(r).hi>(const TileArgs<Q>*);
#define QAOA_BATCH_INSTANCES(real, Q, R)                                                              \
    namespace qaoa {                                                                                   \
    QAOA_INSTANCE __global__ void tile_batch_kernel<real, Q, R, false, 0, 0, 0, 0>(const TileArgs<Q>*);   \
    QAOA_BATCH_ONE(real, Q, R, 8)                                                                      \
    QAOA_BATCH_ONE(real, Q, R, 9)                                                                      \
    QAOA_BATCH_ONE(real, Q, R, 10)                                                                     \
    QAOA_BATCH_ONE(real, Q, R, 11)                                                                     \
    QAOA_BATCH_ONE(real, Q, R, 12)                                                                     \
    }

#if !defined(QAOA_OWN_BATCH_C64)
QAOA_BATCH_INSTANCES(float, 13, 5)
#endif
#if !defined(QAOA_OWN_TILE_C64)
QAOA_TILE_INSTANCES(float, 13, 5)
#endif
#if !defined(QAOA_OWN_RECIPE_C64)
QAOA_RECIPE_INSTANCES(float, 13, 5)
#endif
#if !defined(QAOA_OWN_RECIPE_W_C64)
QAOA_RECIPE_W_INSTANCES(float, 13, 5)
#endif
#if !defined(QAOA_OWN_TILE_C128)
QAOA_TILE_INSTANCES(double, 12, 4)
QAOA_RECIPE_INSTANCES(double, 12, 4)
#endif
#if !defined(QAOA_OWN_GRAD)
QAOA_GRAD_INSTANCES(float, 12, 4)
QAOA_GRAD_INSTANCES(double, 12, 4)
#endif
#if !defined(QAOA_OWN_RECIPE_2G_C64)
QAOA_RECIPE_2G_INSTANCES(float, 13, 5)
#endif
#if !defined(QAOA_OWN_GRAD_RECIPES)
QAOA_GRAD_RECIPE_INSTANCES(float, 12, 4)
#endif
#if !defined(QAOA_OWN_GRAD_RECIPES_M)
QAOA_GRAD_RECIPE_M_INSTANCES(float, 12, 4)
#endif
#if !defined(QAOA_OWN_GRAD_RECIPES_X)
QAOA_GRAD_RECIPE_X_INSTANCES(float, 12, 4)
#endif
#if !defined(QAOA_OWN_GRAD_PF)
QAOA_GRAD_PF_INSTANCES(12, 4, false)
#endif
#if !defined(QAOA_OWN_GRAD_PF_W)
QAOA_GRAD_PF_INSTANCES(12, 4, true)
#endif
