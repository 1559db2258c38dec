// walk_diag_tc3.cu -- the tensor-core product engine of the all-detected
// walk (Algorithm 1, Sec. 3.1.3) and its adjoint for 9..12 kept modes
// (3 K steps of 16 real rows): forward, reverse walk and partial-sum pass.
#include "walk_diag_impl.cuh"

namespace fk {

namespace {

const WalkKernels kTc = {128, 4, 3, (const void *)diag_forward_kernel<128, 4, 3>,
                         (const void *)diag_vjp_kernel<128, 4, 3>,
                         (const void *)diag_vjp_partials_kernel<128, 4, 3>, &Walk<128, 4, 3>::smem_bytes};

}  // namespace

const WalkKernels *tc3_walk_kernels() { return &kTc; }

}  // namespace fk
