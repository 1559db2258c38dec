// mlp.cu -- the learned proposal model: a 15 -> 256 -> 256 -> 256 -> 2
// multilayer perceptron with BF16 weights and activations, FP32 accumulation
// on the tensor cores, SiLU hidden activations, an MSE loss and Adam on FP32
// master weights.  Every GEMM of the forward and backward passes (outputs,
// input gradients, weight gradients) runs on the tcgen05 GEMM of mlp_tc.cu,
// with K-major operands: the weights and their transposes are kept in bf16,
// and the epilogues write the transposed activations and gradients that the
// weight-gradient GEMMs (K = the batch) take.  It predicts, from 15 circuit
// parameters, two scores of the state the circuit heralds; the exact
// recurrence checks every proposal it makes.
//
// State buffer (device, FP32 unless noted), offsets in fk_mlp_layout():
//   master[P]  packed W1 b1 W2 b2 W3 b3 W4 b4 (W row-major [out][in])
//   adam_m[P], adam_v[P]
//   W1h [256][16] bf16 (input padded 15 -> 16), W2h, W3h [256][256] bf16,
//   W4h [16][256] bf16 (output padded 2 -> 16), W2t, W3t [256][256], W4t
//   [256][16]: W2h, W3h, W4h transposed (the B operands, K-major, of the
//   input-gradient GEMMs)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <stdint.h>

#include "mlp_tc.h"
#include "../../include/fockdiag.h"
#include "../../include/fockdiag_mlp.h"

namespace {

constexpr int IN = FK_MLP_IN, INP = 16, H = FK_MLP_HIDDEN, OUT = FK_MLP_OUT, OUTP = 16;
constexpr int64_t NW1 = (int64_t)H * IN, NW2 = (int64_t)H * H, NW3 = (int64_t)H * H,
                  NW4 = (int64_t)OUT * H;
constexpr int64_t OW1 = 0, OB1 = OW1 + NW1, OW2 = OB1 + H, OB2 = OW2 + NW2, OW3 = OB2 + H,
                  OB3 = OW3 + NW3, OW4 = OB3 + H, OB4 = OW4 + NW4, NPARAM = OB4 + OUT;

struct StateLayout {
    size_t master, m, v, w1h, w2h, w3h, w4h, w2t, w3t, w4t, total;
};

size_t al(size_t x) { return (x + 255) / 256 * 256; }

StateLayout state_layout()
{
    StateLayout s;
    size_t o = 0;
    s.master = o; o = al(o + NPARAM * 4);
    s.m = o; o = al(o + NPARAM * 4);
    s.v = o; o = al(o + NPARAM * 4);
    s.w1h = o; o = al(o + (size_t)H * INP * 2);
    s.w2h = o; o = al(o + (size_t)H * H * 2);
    s.w3h = o; o = al(o + (size_t)H * H * 2);
    s.w4h = o; o = al(o + (size_t)OUTP * H * 2);
    s.w2t = o; o = al(o + (size_t)H * H * 2);
    s.w3t = o; o = al(o + (size_t)H * H * 2);
    s.w4t = o; o = al(o + (size_t)H * OUTP * 2);
    s.total = o;
    return s;
}

// Workspace per batch: activations (bf16) and pre-activations (fp32) of the
// three hidden layers, the padded input, the output, and backward buffers.
struct WsLayout {
    size_t x, z1, a1, z2, a2, z3, a3, y, g3, g2, g1, gy, gp, loss, wpart, bpart;
    size_t a1t, a2t, a3t, g1t, g2t, g3t, xt, gyt, status, total;   // transposed [H or 16][ldT] copies
                                                                   // (weight-gradient operands)
    int64_t ldT;
};

// The weight gradients contract over the batch (K): their K range is split
// over CTAs (about 1024 samples each, at most 128 slices) into a scratch
// array summed in a fixed order, since the output tiles alone give 1-2 CTAs.
int tc_ksplit(int B) { return B >= 2048 ? (B / 1024 < 128 ? B / 1024 : 128) : 1; }

WsLayout ws_layout(int B)
{
    WsLayout w;
    size_t o = 0;
    const size_t b = (size_t)B;
    w.x = o; o = al(o + b * INP * 2);
    w.z1 = o; o = al(o + b * H * 4);
    w.a1 = o; o = al(o + b * H * 2);
    w.z2 = o; o = al(o + b * H * 4);
    w.a2 = o; o = al(o + b * H * 2);
    w.z3 = o; o = al(o + b * H * 4);
    w.a3 = o; o = al(o + b * H * 2);
    w.y = o; o = al(o + b * OUTP * 4);
    w.gy = o; o = al(o + b * OUTP * 2);
    w.g3 = o; o = al(o + b * H * 2);
    w.g2 = o; o = al(o + b * H * 2);
    w.g1 = o; o = al(o + b * H * 2);
    w.gp = o; o = al(o + NPARAM * 4);
    w.loss = o; o = al(o + 64);
    const int slices = fk::tc_gemm_slices(B, tc_ksplit(B));
    w.wpart = o; o = al(o + (size_t)slices * H * H * 4);
    w.bpart = o; o = al(o + (size_t)((B + 8191) / 8192) * H * 4);
    w.ldT = (b + 7) / 8 * 8;
    w.a1t = o; o = al(o + (size_t)H * w.ldT * 2);
    w.a2t = o; o = al(o + (size_t)H * w.ldT * 2);
    w.a3t = o; o = al(o + (size_t)H * w.ldT * 2);
    w.g1t = o; o = al(o + (size_t)H * w.ldT * 2);
    w.g2t = o; o = al(o + (size_t)H * w.ldT * 2);
    w.xt = o; o = al(o + (size_t)INP * w.ldT * 2);
    w.gyt = o; o = al(o + (size_t)OUTP * w.ldT * 2);
    w.g3t = o; o = al(o + (size_t)H * w.ldT * 2);
    w.status = o; o = al(o + 64);
    w.total = o;
    return w;
}

__global__ void sum_slices(const float *part, int slices, int64_t n, float *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int z = 0; z < slices; ++z) s += part[(int64_t)z * n + i];
    out[i] = s;
}

// ------------------------------------------------------------ small kernels
// x [B][15] fp32 -> bf16 [B][16] (zero padded) and its transpose [16][ldT]
__global__ void pack_input(const float *x, __nv_bfloat16 *xp, __nv_bfloat16 *xt, int64_t ldT, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * INP) return;
    const int b = i / INP, k = i % INP;
    const __nv_bfloat16 v = __float2bfloat16(k < IN ? x[(int64_t)b * IN + k] : 0.f);
    xp[i] = v;
    if (xt) xt[(int64_t)k * ldT + b] = v;
}

// bf16 working copies of the master weights (padded shapes), and the
// transposes of W2, W3 and W4
__global__ void refresh_bf16(const float *master, __nv_bfloat16 *w1, __nv_bfloat16 *w2,
                             __nv_bfloat16 *w3, __nv_bfloat16 *w4, __nv_bfloat16 *w2t, __nv_bfloat16 *w3t,
                             __nv_bfloat16 *w4t)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (int64_t)H * INP) {
        const int r = (int)(i / INP), k = (int)(i % INP);
        w1[i] = __float2bfloat16(k < IN ? master[OW1 + (int64_t)r * IN + k] : 0.f);
    }
    if (i < NW2) {
        const __nv_bfloat16 v2 = __float2bfloat16(master[OW2 + i]);
        const __nv_bfloat16 v3 = __float2bfloat16(master[OW3 + i]);
        w2[i] = v2;
        w3[i] = v3;
        const int64_t t = (i % H) * H + i / H;
        w2t[t] = v2;
        w3t[t] = v3;
    }
    if (i < (int64_t)OUTP * H) {
        const int r = (int)(i / H), c = (int)(i % H);
        const __nv_bfloat16 v = __float2bfloat16(r < OUT ? master[OW4 + i] : 0.f);
        w4[i] = v;
        w4t[(int64_t)c * OUTP + r] = v;
    }
}

// dL/dy for L = mean_b sum_j (y_bj - t_bj)^2 / OUT, as bf16 (padded) and
// transposed ([16][ldT]), and the loss itself (block partial sums, then one
// atomic per block).
__global__ void loss_grad(const float *y, const float *t, __nv_bfloat16 *gy, __nv_bfloat16 *gyt, int64_t ldT,
                          float *loss, int B)
{
    __shared__ float red[256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < B * OUTP) {
        const int b = i / OUTP, j = i % OUTP;
        float g = 0.f;
        if (j < OUT) {
            const float d = y[(int64_t)b * OUTP + j] - t[(int64_t)b * OUT + j];
            l = d * d / (float)(B * OUT);
            g = 2.f * d / (float)(B * OUT);
        }
        gy[i] = __float2bfloat16(g);
        gyt[(int64_t)j * ldT + b] = __float2bfloat16(g);
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// upstream gradient [B][OUT] fp32 -> padded bf16 [B][OUTP] and its transpose
__global__ void pack_grad(const float *gy, __nv_bfloat16 *out, __nv_bfloat16 *outt, int64_t ldT, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * OUTP) return;
    const int b = i / OUTP, j = i % OUTP;
    const __nv_bfloat16 v = __float2bfloat16(j < OUT ? gy[(int64_t)b * OUT + j] : 0.f);
    out[i] = v;
    outt[(int64_t)j * ldT + b] = v;
}

// bias gradients: row sums of a transposed bf16 gradient gT [rows][ldT]
// (the first B entries of each row).  Block (r, s) sums the 8192-entry
// slice s of row r with 16-byte loads and a fixed-order tree; a second pass
// adds the slices in order.
constexpr int kBiasSlice = 8192;

__global__ void bias_grad_part(const __nv_bfloat16 *gT, int B, int64_t ldT, float *part, int rows)
{
    __shared__ float red[256];
    const int r = blockIdx.x, s = blockIdx.y;
    const int64_t b0 = (int64_t)s * kBiasSlice;
    const __nv_bfloat16 *row = gT + (int64_t)r * ldT;
    float acc = 0.f;
    // 32 entries per thread: four runs of 8
    for (int k = 0; k < 4; ++k) {
        const int64_t b = b0 + (int64_t)(k * 256 + threadIdx.x) * 8;
        if (b + 8 <= B && ((ldT & 7) == 0)) {
            const uint4 w = *(const uint4 *)(row + b);
            const __nv_bfloat16 *h = (const __nv_bfloat16 *)&w;
#pragma unroll
            for (int i = 0; i < 8; ++i) acc += __bfloat162float(h[i]);
        } else {
            for (int i = 0; i < 8; ++i)
                if (b + i < B) acc += __bfloat162float(row[b + i]);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)s * rows + r] = red[0];
}

void bias_grad(const __nv_bfloat16 *gT, int B, int64_t ldT, int rows, float *part, float *out, cudaStream_t st)
{
    const int slices = (B + kBiasSlice - 1) / kBiasSlice;
    bias_grad_part<<<dim3(rows, slices), 256, 0, st>>>(gT, B, ldT, part, rows);
    sum_slices<<<(rows + 255) / 256, 256, 0, st>>>(part, slices, rows, out);
}

__global__ void adam_kernel(float *w, float *m, float *v, const float *g, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

struct Ptrs {
    float *master, *m, *v;
    __nv_bfloat16 *w1, *w2, *w3, *w4, *w2t, *w3t, *w4t;
    __nv_bfloat16 *x, *a1, *a2, *a3, *gy, *g3, *g2, *g1;
    __nv_bfloat16 *a1t, *a2t, *a3t, *g1t, *g2t, *g3t, *xt, *gyt;
    float *z1, *z2, *z3, *y, *gp, *loss, *wpart, *bpart;
    int *status;
    int64_t ldT;
};

Ptrs ptrs(void *state, void *ws, int B)
{
    const StateLayout s = state_layout();
    const WsLayout w = ws_layout(B);
    char *S = (char *)state, *W = (char *)ws;
    Ptrs p;
    p.master = (float *)(S + s.master);
    p.m = (float *)(S + s.m);
    p.v = (float *)(S + s.v);
    p.w1 = (__nv_bfloat16 *)(S + s.w1h);
    p.w2 = (__nv_bfloat16 *)(S + s.w2h);
    p.w3 = (__nv_bfloat16 *)(S + s.w3h);
    p.w4 = (__nv_bfloat16 *)(S + s.w4h);
    p.w2t = (__nv_bfloat16 *)(S + s.w2t);
    p.w3t = (__nv_bfloat16 *)(S + s.w3t);
    p.w4t = (__nv_bfloat16 *)(S + s.w4t);
    p.a1t = (__nv_bfloat16 *)(W + w.a1t);
    p.a2t = (__nv_bfloat16 *)(W + w.a2t);
    p.a3t = (__nv_bfloat16 *)(W + w.a3t);
    p.g1t = (__nv_bfloat16 *)(W + w.g1t);
    p.xt = (__nv_bfloat16 *)(W + w.xt);
    p.gyt = (__nv_bfloat16 *)(W + w.gyt);
    p.g2t = (__nv_bfloat16 *)(W + w.g2t);
    p.g3t = (__nv_bfloat16 *)(W + w.g3t);
    p.status = (int *)(W + w.status);
    p.ldT = w.ldT;
    p.x = (__nv_bfloat16 *)(W + w.x);
    p.z1 = (float *)(W + w.z1);
    p.a1 = (__nv_bfloat16 *)(W + w.a1);
    p.z2 = (float *)(W + w.z2);
    p.a2 = (__nv_bfloat16 *)(W + w.a2);
    p.z3 = (float *)(W + w.z3);
    p.a3 = (__nv_bfloat16 *)(W + w.a3);
    p.y = (float *)(W + w.y);
    p.gy = (__nv_bfloat16 *)(W + w.gy);
    p.g3 = (__nv_bfloat16 *)(W + w.g3);
    p.g2 = (__nv_bfloat16 *)(W + w.g2);
    p.g1 = (__nv_bfloat16 *)(W + w.g1);
    p.gp = (float *)(W + w.gp);
    p.loss = (float *)(W + w.loss);
    p.wpart = (float *)(W + w.wpart);
    p.bpart = (float *)(W + w.bpart);
    return p;
}

fk::TcEpilogue epilogue(const Ptrs &p, int kind)
{
    fk::TcEpilogue e{};
    e.kind = kind;
    e.ldo = H;
    e.ldT = p.ldT;
    e.status = p.status;
    return e;
}

// Hidden layer: z = a_in W^T + b (K = Kin), act = SiLU(z) and, when training,
// the transposed activations for the weight gradients.
int hidden(const Ptrs &p, int B, const __nv_bfloat16 *ain, int Kin, const __nv_bfloat16 *W, const float *bias,
           float *z, __nv_bfloat16 *act, __nv_bfloat16 *actT, cudaStream_t st)
{
    fk::TcEpilogue e = epilogue(p, fk::TC_EPI_HIDDEN);
    e.bias = bias;
    e.z = z;
    e.act = act;
    e.actT = actT;
    return fk::tc_gemm(B, H, Kin, ain, Kin, W, Kin, 1, e, st);
}

// train: also the transposed activations the weight gradients need
int forward(const Ptrs &p, int B, const float *x, cudaStream_t st, bool train = false)
{
    if (cudaMemsetAsync(p.status, 0, sizeof(int), st) != cudaSuccess) return FK_ECUDA;
    pack_input<<<(B * INP + 255) / 256, 256, 0, st>>>(x, p.x, train ? p.xt : nullptr, p.ldT, B);
    int rc;
    if ((rc = hidden(p, B, p.x, INP, p.w1, p.master + OB1, p.z1, p.a1, train ? p.a1t : nullptr, st))) return rc;
    if ((rc = hidden(p, B, p.a1, H, p.w2, p.master + OB2, p.z2, p.a2, train ? p.a2t : nullptr, st))) return rc;
    if ((rc = hidden(p, B, p.a2, H, p.w3, p.master + OB3, p.z3, p.a3, train ? p.a3t : nullptr, st))) return rc;
    // output layer: y = a3 W4^T + b4, the 2 real outputs of [B][16]
    fk::TcEpilogue e = epilogue(p, fk::TC_EPI_OUT);
    e.bias = p.master + OB4;
    e.z = p.y;
    e.ldo = OUTP;
    return fk::tc_gemm(B, OUT, H, p.a3, H, p.w4, H, 1, e, st);
}

// dL/dW = g^T a_in over the batch (K split over CTAs, fixed-order sum) into
// the packed gradient at `dst` ([M][N], leading dimension N).
int wgrad(const Ptrs &p, int B, const __nv_bfloat16 *gT, int M, const __nv_bfloat16 *aT, int N, float *dst,
          cudaStream_t st)
{
    fk::TcEpilogue e = epilogue(p, fk::TC_EPI_PARTIAL);
    e.ldo = N;
    e.out = p.wpart;
    e.sum_to = dst;
    return fk::tc_gemm(M, N, B, gT, p.ldT, aT, p.ldT, tc_ksplit(B), e, st);
}

// dL/dz_in = (g W) * silu'(z_in): A = g [B][Kg], B = W^T [H][Kg].
int back_hidden(const Ptrs &p, int B, const __nv_bfloat16 *g, int Kg, const __nv_bfloat16 *Wt, const float *zin,
                __nv_bfloat16 *gout, __nv_bfloat16 *goutT, cudaStream_t st)
{
    fk::TcEpilogue e = epilogue(p, fk::TC_EPI_BACK_HIDDEN);
    e.act = gout;
    e.actT = goutT;
    e.zprev = zin;
    return fk::tc_gemm(B, H, Kg, g, Kg, Wt, Kg, 1, e, st);
}

// Back-propagate gy (bf16 [B][OUTP], and its transpose) into the parameter
// gradients p.gp (packed like master).
int backward(const Ptrs &p, int B, cudaStream_t st)
{
    int rc;
    // layer 4: dL/dW4 = gy^T a3 ([2][H]), dL/db4, dL/dz3 = (gy W4) * silu'(z3)
    if ((rc = wgrad(p, B, p.gyt, OUT, p.a3t, H, p.gp + OW4, st))) return rc;
    bias_grad(p.gyt, B, p.ldT, OUT, p.bpart, p.gp + OB4, st);
    if ((rc = back_hidden(p, B, p.gy, OUTP, p.w4t, p.z3, p.g3, p.g3t, st))) return rc;
    // layer 3
    if ((rc = wgrad(p, B, p.g3t, H, p.a2t, H, p.gp + OW3, st))) return rc;
    bias_grad(p.g3t, B, p.ldT, H, p.bpart, p.gp + OB3, st);
    if ((rc = back_hidden(p, B, p.g3, H, p.w3t, p.z2, p.g2, p.g2t, st))) return rc;
    // layer 2
    if ((rc = wgrad(p, B, p.g2t, H, p.a1t, H, p.gp + OW2, st))) return rc;
    bias_grad(p.g2t, B, p.ldT, H, p.bpart, p.gp + OB2, st);
    if ((rc = back_hidden(p, B, p.g2, H, p.w2t, p.z1, p.g1, p.g1t, st))) return rc;
    // layer 1: the 15 real inputs of W1
    if ((rc = wgrad(p, B, p.g1t, H, p.xt, IN, p.gp + OW1, st))) return rc;
    bias_grad(p.g1t, B, p.ldT, H, p.bpart, p.gp + OB1, st);
    return FK_OK;
}

bool aligned256(const void *p) { return ((uintptr_t)p & 255u) == 0; }

}  // namespace

extern "C" {

int fk_mlp_sizes(int batch, size_t *state_bytes, size_t *ws_bytes, int64_t *n_params)
{
    if (batch < 1 || batch > (1 << 24)) return FK_EINVAL;
    if (state_bytes) *state_bytes = state_layout().total;
    if (ws_bytes) *ws_bytes = ws_layout(batch).total;
    if (n_params) *n_params = NPARAM;
    return FK_OK;
}

int fk_mlp_load(void *state, const float *master, void *stream)
{
    if (!state || !master || !aligned256(state)) return FK_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const StateLayout s = state_layout();
    char *S = (char *)state;
    if (cudaMemcpyAsync(S + s.master, master, NPARAM * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return FK_ECUDA;
    if (cudaMemsetAsync(S + s.m, 0, s.w1h - s.m, st) != cudaSuccess) return FK_ECUDA;
    const int64_t n = NW2;
    refresh_bf16<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        (const float *)(S + s.master), (__nv_bfloat16 *)(S + s.w1h), (__nv_bfloat16 *)(S + s.w2h),
        (__nv_bfloat16 *)(S + s.w3h), (__nv_bfloat16 *)(S + s.w4h), (__nv_bfloat16 *)(S + s.w2t),
        (__nv_bfloat16 *)(S + s.w3t), (__nv_bfloat16 *)(S + s.w4t));
    return cudaGetLastError() == cudaSuccess ? FK_OK : FK_ECUDA;
}

int fk_mlp_forward(const void *state, int batch, const float *x, float *y, void *ws, size_t ws_bytes,
                   void *stream)
{
    if (!state || !x || !y || !ws || batch < 1 || !aligned256(ws)) return FK_EINVAL;
    if (ws_bytes < ws_layout(batch).total) return FK_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    Ptrs p = ptrs((void *)state, ws, batch);
    int rc = forward(p, batch, x, st);
    if (rc) return rc;
    // compact [B][OUTP] -> [B][OUT]
    if (cudaMemcpy2DAsync(y, OUT * 4, p.y, OUTP * 4, OUT * 4, batch, cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
        return FK_ECUDA;
    return FK_OK;
}

int fk_mlp_backward(const void *state, int batch, const float *x, const float *gy, float *gparams,
                    void *ws, size_t ws_bytes, void *stream)
{
    if (!state || !x || !gy || !gparams || !ws || batch < 1 || !aligned256(ws)) return FK_EINVAL;
    if (ws_bytes < ws_layout(batch).total) return FK_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    Ptrs p = ptrs((void *)state, ws, batch);
    int rc = forward(p, batch, x, st, true);
    if (rc) return rc;
    // upstream gradient [B][OUT] fp32 -> padded bf16 and its transpose
    pack_grad<<<(unsigned)((batch * OUTP + 255) / 256), 256, 0, st>>>(gy, p.gy, p.gyt, p.ldT, batch);
    if ((rc = backward(p, batch, st))) return rc;
    if (cudaMemcpyAsync(gparams, p.gp, NPARAM * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return FK_ECUDA;
    return FK_OK;
}

int fk_mlp_train_step(void *state, int batch, const float *x, const float *target, float lr,
                      float beta1, float beta2, float eps, int step, float *loss, void *ws,
                      size_t ws_bytes, void *stream)
{
    if (!state || !x || !target || !ws || batch < 1 || step < 1 || !aligned256(ws)) return FK_EINVAL;
    if (ws_bytes < ws_layout(batch).total) return FK_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    Ptrs p = ptrs(state, ws, batch);
    int rc = forward(p, batch, x, st, true);
    if (rc) return rc;
    if (cudaMemsetAsync(p.loss, 0, 4, st) != cudaSuccess) return FK_ECUDA;
    loss_grad<<<(batch * OUTP + 255) / 256, 256, 0, st>>>(p.y, target, p.gy, p.gyt, p.ldT, p.loss, batch);
    if ((rc = backward(p, batch, st))) return rc;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<(unsigned)((NPARAM + 255) / 256), 256, 0, st>>>(p.master, p.m, p.v, p.gp, NPARAM,
                                                                  lr, beta1, beta2, eps, c1, c2);
    refresh_bf16<<<(unsigned)((NW2 + 255) / 256), 256, 0, st>>>(p.master, p.w1, p.w2, p.w3, p.w4, p.w2t,
                                                                p.w3t, p.w4t);
    if (loss && cudaMemcpyAsync(loss, p.loss, 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return FK_ECUDA;
    return cudaGetLastError() == cudaSuccess ? FK_OK : FK_ECUDA;
}

}  // extern "C"
