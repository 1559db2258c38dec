// walk_cond_k0.cu -- the conditional-state walk (Algorithm 2, Sec. 3.2)
// and its adjoint on the FP64 engine (Gauss's three-multiplication products).
#include "walk_cond_impl.cuh"

namespace fk {

namespace {

const CondKernels kK = {(const void *)cond_forward_kernel<0>, (const void *)cond_vjp_kernel<0>};

}  // namespace

const CondKernels *cond_kernels_k0() { return &kK; }

}  // namespace fk
