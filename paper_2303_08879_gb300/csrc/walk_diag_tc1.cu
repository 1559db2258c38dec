// walk_diag_tc1.cu -- the tensor-core product engine of the all-detected
// walk (Algorithm 1, Sec. 3.1.3) and its adjoint for 1..4 kept modes
// (1 K step of 16 real rows): forward, reverse walk and partial-sum pass.
#include "walk_diag_impl.cuh"

namespace fk {

namespace {

const WalkKernels kTc = {128, 4, 1, (const void *)diag_forward_kernel<128, 4, 1>,
                         (const void *)diag_vjp_kernel<128, 4, 1>,
                         (const void *)diag_vjp_partials_kernel<128, 4, 1>, &Walk<128, 4, 1>::smem_bytes};

}  // namespace

const WalkKernels *tc1_walk_kernels() { return &kTc; }

}  // namespace fk
