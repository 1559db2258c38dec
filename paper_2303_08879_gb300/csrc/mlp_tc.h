// mlp_tc.h -- the tcgen05 GEMM of the proposal MLP (mlp_tc.cu), shared with
// mlp.cu.  Not part of the public ABI.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace fk {

enum TcEpiKind { TC_EPI_HIDDEN = 0, TC_EPI_BACK_HIDDEN = 1, TC_EPI_PARTIAL = 2, TC_EPI_OUT = 3 };

// What the GEMM does with C[m][n] (row m of A, row n of B):
//   HIDDEN:       z = C + bias[n] -> z (fp32), act = SiLU(z) (bf16), actT (bf16, transposed)
//   OUT:          z = C + bias[n] (fp32)
//   BACK_HIDDEN:  act = C * SiLU'(zprev) (bf16), actT (transposed)
//   PARTIAL:      fp32 C of K slice blockIdx.z at out[z][m][n]; summed into sum_to when set
// Outputs [M][ldo]; actT [N][ldT] (null: not written).
struct TcEpilogue {
    int kind;
    int ldo;
    int64_t ldT;
    const float *bias;
    float *z;
    __nv_bfloat16 *act, *actT;
    const float *zprev;
    float *out, *sum_to;
    int *status;           // FK_ETIMEOUT on a wait that ran out (device word), or null
};

// C = A B^T: A [M][K] (leading dimension lda), B [N][K] (ldb), bf16, K-major;
// N <= 256 or a multiple of 256 (columns n >= N are neither computed from
// memory nor written); leading dimensions multiples of 8 and 16-byte aligned
// bases (TMA).  ksplit > 1 splits K over CTAs (PARTIAL only).
int tc_gemm(int M, int N, int K, const void *A, int64_t lda, const void *B, int64_t ldb, int ksplit,
            const TcEpilogue &e, void *stream);
// Number of K slices tc_gemm uses for (K, ksplit).
int tc_gemm_slices(int K, int ksplit);

}  // namespace fk
