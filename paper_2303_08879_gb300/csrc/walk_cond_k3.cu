// walk_cond_k3.cu -- the conditional-state walk (Algorithm 2, Sec. 3.2)
// and its adjoint on the tensor-core engine with 3 K steps of 16 real rows (up to 12 modes).
#include "walk_cond_impl.cuh"

namespace fk {

namespace {

const CondKernels kK = {(const void *)cond_forward_kernel<3>, (const void *)cond_vjp_kernel<3>};

}  // namespace

const CondKernels *cond_kernels_k3() { return &kK; }

}  // namespace fk
