// walk_cond_k1.cu -- the conditional-state walk (Algorithm 2, Sec. 3.2)
// and its adjoint on the tensor-core engine with 1 K step of 16 real rows (up to 4 modes).
#include "walk_cond_impl.cuh"

namespace fk {

namespace {

const CondKernels kK = {(const void *)cond_forward_kernel<1>, (const void *)cond_vjp_kernel<1>};

}  // namespace

const CondKernels *cond_kernels_k1() { return &kK; }

}  // namespace fk
