// walk_diag_fp64.cu -- the FP64 product engine of the all-detected walk
// (Algorithm 1, Sec. 3.1.3) and its adjoint for one tile shape: FK_TPB
// pivots per tile, FK_CH output rows per register chunk.  The build compiles
// this file once per shape (128/8, 128/4, 64/8, 64/4, 256/8), so the shapes
// compile in parallel.
#include "walk_diag_impl.cuh"

#ifndef FK_TPB
#error "FK_TPB and FK_CH select the tile shape of this translation unit"
#endif

#define FK_CAT2(a, b, c) a##_##b##_##c
#define FK_CAT(a, b, c) FK_CAT2(a, b, c)

namespace fk {

namespace {

const WalkKernels kShape = {FK_TPB, FK_CH, 0, (const void *)diag_forward_kernel<FK_TPB, FK_CH, 0>,
                            (const void *)diag_vjp_kernel<FK_TPB, FK_CH, 0>, nullptr,
                            &Walk<FK_TPB, FK_CH>::smem_bytes};

}  // namespace

const WalkKernels *FK_CAT(fp64_walk_kernels, FK_TPB, FK_CH)() { return &kShape; }

}  // namespace fk
