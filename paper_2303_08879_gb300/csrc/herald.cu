// herald.cu -- scores of heralded conditional states: for circuit i, the
// unnormalised density matrix rho = rho_i(n*) of the undetected mode for the
// heralding pattern n* (a block of the fock_conditional_dm output),
//   P = Tr rho (success probability),  F = <t|rho|t> / P (fidelity to the
//   normalised target t),  J = F + lambda ln P,
// and, optionally, dJ/drho in PyTorch's convention for a real objective:
//   gbar_kl = (t_k conj(t_l) - F delta_kl + lambda delta_kl) / P.
#include <cuda_runtime.h>

#include "fk_internal.h"
#include "walk_common.cuh"
#include "../../include/fockdiag.h"

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) herald_kernel(const double2 *rho, const int64_t *offs,
                                                          int NU, const double2 *t, double lam,
                                                          double *P, double *F, double2 *grad)
{
    __shared__ double red_t[kThreads], red_n[kThreads];
    __shared__ double s_T, s_F;
    const int c = blockIdx.x;
    const double2 *R = rho + offs[c];
    double T = 0.0, N = 0.0;
    for (int e = threadIdx.x; e < NU * NU; e += blockDim.x) {
        const int k = e / NU, l = e % NU;
        const double2 r = R[e];
        if (k == l) T += r.x;
        // Re(conj(t_k) r t_l)
        const double2 tk = t[k], tl = t[l];
        const double2 rt = make_double2(r.x * tl.x - r.y * tl.y, r.x * tl.y + r.y * tl.x);
        N += tk.x * rt.x + tk.y * rt.y;
    }
    red_t[threadIdx.x] = T;
    red_n[threadIdx.x] = N;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red_t[threadIdx.x] += red_t[threadIdx.x + s];
            red_n[threadIdx.x] += red_n[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        s_T = red_t[0];
        s_F = red_n[0] / red_t[0];
        P[c] = s_T;
        F[c] = s_F;
    }
    __syncthreads();
    if (!grad) return;
    const double iT = 1.0 / s_T, Fv = s_F;
    double2 *G = grad + offs[c];
    for (int e = threadIdx.x; e < NU * NU; e += blockDim.x) {
        const int k = e / NU, l = e % NU;
        const double2 tk = t[k], tl = t[l];
        // t_k conj(t_l)
        double gx = tk.x * tl.x + tk.y * tl.y, gy = tk.y * tl.x - tk.x * tl.y;
        if (k == l) gx += lam - Fv;
        G[e] = make_double2(gx * iT, gy * iT);
    }
}

}  // namespace

extern "C" int fk_herald_scores(int batch, const fk_c128 *rho, const int64_t *offsets, int NU,
                                const fk_c128 *target, double lam, double *P, double *F,
                                fk_c128 *grad_rho, void *stream)
{
    if (batch < 1 || NU < 1 || !rho || !offsets || !target || !P || !F) return FK_EINVAL;
    herald_kernel<<<batch, kThreads, 0, (cudaStream_t)stream>>>(
        (const double2 *)rho, offsets, NU, (const double2 *)target, lam, P, F, (double2 *)grad_rho);
    return cudaGetLastError() == cudaSuccess ? FK_OK : FK_ECUDA;
}
