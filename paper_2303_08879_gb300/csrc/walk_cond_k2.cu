// walk_cond_k2.cu -- the conditional-state walk (Algorithm 2, Sec. 3.2)
// and its adjoint on the tensor-core engine with 2 K steps of 16 real rows (up to 8 modes).
#include "walk_cond_impl.cuh"

namespace fk {

namespace {

const CondKernels kK = {(const void *)cond_forward_kernel<2>, (const void *)cond_vjp_kernel<2>};

}  // namespace

const CondKernels *cond_kernels_k2() { return &kK; }

}  // namespace fk
