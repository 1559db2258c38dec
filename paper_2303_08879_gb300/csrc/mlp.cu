// mlp.cu -- the learned proposal model: a 15 -> 256 -> 256 -> 256 -> 2
// multilayer perceptron with BF16 weights and activations, FP32 accumulation
// on the tensor cores, SiLU hidden activations, an MSE loss and Adam on FP32
// master weights.  The 256 x 256 layers (forward, input gradients and weight
// gradients) run on the tcgen05 GEMM of mlp_tc.cu; the 16-wide first and
// last layers on a small mma.sync GEMM.  It predicts, from 15 circuit
// parameters, two scores of the state the circuit heralds; the exact
// recurrence checks every proposal it makes.
//
// State buffer (device, FP32 unless noted), offsets in fk_mlp_layout():
//   master[P]  packed W1 b1 W2 b2 W3 b3 W4 b4 (W row-major [out][in])
//   adam_m[P], adam_v[P]
//   W1h [256][16] bf16 (input padded 15 -> 16), W2h, W3h [256][256] bf16,
//   W4h [16][256] bf16 (output padded 2 -> 16), W2t, W3t: W2h, W3h transposed
//   (the B operands, K-major, of the input-gradient GEMMs)
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
    size_t master, m, v, w1h, w2h, w3h, w4h, w2t, w3t, total;
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
    s.total = o;
    return s;
}

// Workspace per batch: activations (bf16) and pre-activations (fp32) of the
// three hidden layers, the padded input, the output, and backward buffers.
struct WsLayout {
    size_t x, z1, a1, z2, a2, z3, a3, y, g3, g2, g1, gy, gp, loss, wpart, bpart;
    size_t a1t, a2t, g2t, g3t, status, total;   // transposed [H][ldT] copies (weight-gradient operands)
    int64_t ldT;
};

// The weight gradients contract over the batch: from 1024 samples on their
// K range is split over ksplit(B) slices written to a scratch array and summed
// in a fixed order (the output tiles alone give 4-16 CTAs).
constexpr int kBiasRows = 4096;   // batch rows per block of the bias-gradient sums
int ksplit(int B) { return B >= 1024 ? (B / 512 < 32 ? B / 512 : 32) : 1; }
// K slices of the tcgen05 weight-gradient GEMMs (K = batch): about 1024
// samples per CTA, at most 128 slices.
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
    w.wpart = o; o = al(o + (size_t)(ksplit(B) > slices ? ksplit(B) : slices) * H * H * 4);
    w.bpart = o; o = al(o + (size_t)((B + kBiasRows - 1) / kBiasRows) * H * 4);
    w.ldT = (b + 7) / 8 * 8;
    w.a1t = o; o = al(o + (size_t)H * w.ldT * 2);
    w.a2t = o; o = al(o + (size_t)H * w.ldT * 2);
    w.g2t = o; o = al(o + (size_t)H * w.ldT * 2);
    w.g3t = o; o = al(o + (size_t)H * w.ldT * 2);
    w.status = o; o = al(o + 64);
    w.total = o;
    return w;
}

// ----------------------------------------------------------------- GEMM
// C[m][n] = sum_k A(m, k) B(n, k), A(m,k) = A[m*sam + k*sak], B(n,k) =
// B[n*sbn + k*sbk], bf16 operands, fp32 accumulation on mma.sync
// m16n8k16.  64 x 64 CTA tile, 4 warps of 32 x 32, K step 32.
constexpr int BM = 64, BN = 64, BK = 32, PADK = BK + 8;

enum Epi { EPI_HIDDEN = 0, EPI_OUT = 1, EPI_BACK_HIDDEN = 2, EPI_WGRAD = 3, EPI_BACK_IN = 4 };

struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16 *A, *B;
    int64_t sam, sak, sbn, sbk;
    int epi;
    const float *bias;          // EPI_HIDDEN / EPI_OUT
    float *z;                   // EPI_HIDDEN: pre-activation out; EPI_OUT: output
    __nv_bfloat16 *act;         // EPI_HIDDEN: SiLU(z); EPI_BACK_HIDDEN: g * SiLU'(zprev)
    const float *zprev;         // EPI_BACK_HIDDEN
    float *wgrad;               // EPI_WGRAD destination [M][ldw]
    int ldo;                    // leading dimension of the outputs
    int nvalid;                 // columns actually stored (<= N)
    int ksplit;                 // EPI_WGRAD: K slices (blockIdx.z), partials to wpart
    float *wpart;               // [ksplit][M][ldo]
};

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }

__device__ __forceinline__ float dsilu(float z)
{
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ void mma16816(float *c, const uint32_t *a, const uint32_t *b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) gemm_kernel(GemmArgs g)
{
    __shared__ __align__(16) __nv_bfloat16 As[BM][PADK];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][PADK];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int grp = lane >> 2, tig = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    // K slice of this block (split-K for the weight gradients)
    const int kper = ((g.K + g.ksplit - 1) / g.ksplit + BK - 1) / BK * BK;
    const int kbeg = blockIdx.z * kper, kend = min(g.K, kbeg + kper);
    // operands stored k-major (transposed) are filled with m (n) fastest so a
    // warp reads consecutive addresses
    const bool at = g.sak > g.sam, bt = g.sbk > g.sbn;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        for (int e = tid; e < BM * BK; e += blockDim.x) {
            const int r = at ? e % BM : e / BK, kk = at ? e / BM : e % BK;
            const int m = m0 + r, k = k0 + kk;
            As[r][kk] = (m < g.M && k < kend) ? g.A[(int64_t)m * g.sam + (int64_t)k * g.sak] : zero;
        }
        for (int e = tid; e < BN * BK; e += blockDim.x) {
            const int r = bt ? e % BN : e / BK, kk = bt ? e / BN : e % BK;
            const int n = n0 + r, k = k0 + kk;
            Bs[r][kk] = (n < g.N && k < kend) ? g.B[(int64_t)n * g.sbn + (int64_t)k * g.sbk] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm * 32 + i * 16 + grp;
                af[i][0] = *(const uint32_t *)&As[r][ks + tig * 2];
                af[i][1] = *(const uint32_t *)&As[r + 8][ks + tig * 2];
                af[i][2] = *(const uint32_t *)&As[r][ks + 8 + tig * 2];
                af[i][3] = *(const uint32_t *)&As[r + 8][ks + 8 + tig * 2];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn * 32 + j * 8 + grp;
                bf[j][0] = *(const uint32_t *)&Bs[c][ks + tig * 2];
                bf[j][1] = *(const uint32_t *)&Bs[c][ks + 8 + tig * 2];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }
    // epilogue: c0,c1 -> (row grp, cols 2tig, 2tig+1); c2,c3 -> row grp + 8
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm * 32 + i * 16 + grp + (r >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + j * 8 + tig * 2 + (r & 1);
                if (m >= g.M || n >= g.nvalid) continue;
                const float v = acc[i][j][r];
                const int64_t o = (int64_t)m * g.ldo + n;
                switch (g.epi) {
                case EPI_HIDDEN: {
                    const float z = v + g.bias[n];
                    g.z[o] = z;
                    g.act[o] = __float2bfloat16(silu(z));
                    break;
                }
                case EPI_OUT: g.z[o] = v + g.bias[n]; break;
                case EPI_BACK_HIDDEN: g.act[o] = __float2bfloat16(v * dsilu(g.zprev[o])); break;
                case EPI_WGRAD:
                    if (g.ksplit > 1) g.wpart[(int64_t)blockIdx.z * g.M * g.ldo + o] = v;
                    else g.wgrad[o] = v;
                    break;
                default: break;
                }
            }
}

__global__ void sum_slices(const float *part, int slices, int64_t n, float *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int z = 0; z < slices; ++z) s += part[(int64_t)z * n + i];
    out[i] = s;
}

int gemm(GemmArgs g, cudaStream_t st)
{
    if (g.ksplit < 1 || g.epi != EPI_WGRAD) g.ksplit = 1;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.ksplit);
    gemm_kernel<<<grid, 128, 0, st>>>(g);
    if (g.ksplit > 1) {
        const int64_t n = (int64_t)g.M * g.ldo;
        sum_slices<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g.wpart, g.ksplit, n, g.wgrad);
    }
    return cudaGetLastError() == cudaSuccess ? FK_OK : FK_ECUDA;
}

// ------------------------------------------------------------ small kernels
__global__ void pack_input(const float *x, __nv_bfloat16 *xp, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * INP) return;
    const int b = i / INP, k = i % INP;
    xp[i] = __float2bfloat16(k < IN ? x[(int64_t)b * IN + k] : 0.f);
}

// bf16 working copies of the master weights (padded shapes), and the
// transposes of W2 and W3
__global__ void refresh_bf16(const float *master, __nv_bfloat16 *w1, __nv_bfloat16 *w2,
                             __nv_bfloat16 *w3, __nv_bfloat16 *w4, __nv_bfloat16 *w2t, __nv_bfloat16 *w3t)
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
        const int r = (int)(i / H);
        w4[i] = __float2bfloat16(r < OUT ? master[OW4 + i] : 0.f);
    }
}

// out[c][r] = in[r][c] for a [rows][H] bf16 matrix (out leading dimension
// ldo), through a 32 x 33 shared tile.
__global__ void transpose_bf16(const __nv_bfloat16 *in, int rows, __nv_bfloat16 *out, int64_t ldo)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        t[y][threadIdx.x] = r < rows ? in[(int64_t)r * H + c] : __float2bfloat16(0.f);
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (r < rows) out[(int64_t)c * ldo + r] = t[threadIdx.x][y];
    }
}

void transpose(const __nv_bfloat16 *in, int rows, __nv_bfloat16 *out, int64_t ldo, cudaStream_t st)
{
    transpose_bf16<<<dim3((rows + 31) / 32, H / 32), dim3(32, 8), 0, st>>>(in, rows, out, ldo);
}

// dL/dy for L = mean_b sum_j (y_bj - t_bj)^2 / OUT, as bf16 (padded), and
// the loss itself (block partial sums, then one atomic per block).
__global__ void loss_grad(const float *y, const float *t, __nv_bfloat16 *gy, float *loss, int B)
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
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// upstream gradient [B][OUT] fp32 -> padded bf16 [B][OUTP]
__global__ void pack_grad(const float *gy, __nv_bfloat16 *out, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * OUT) return;
    const int b = i / OUT, j = i % OUT;
    out[(int64_t)b * OUTP + j] = __float2bfloat16(gy[i]);
}

// bias gradients: column sums of a [B][ld] bf16 gradient (first n columns).
// Block (x: 32 columns, y: kBiasRows rows), 32 x 8 threads; the 8 row
// strands are summed in a fixed order, then the row blocks (second kernel).
__global__ void bias_grad_part(const __nv_bfloat16 *g, int B, int ld, int n, float *part)
{
    __shared__ float red[8][33];
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int b0 = blockIdx.y * kBiasRows, b1 = min(B, b0 + kBiasRows);
    float s = 0.f;
    if (j < n)
        for (int b = b0 + threadIdx.y; b < b1; b += 8) s += __bfloat162float(g[(int64_t)b * ld + j]);
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && j < n) {
        float t = 0.f;
        for (int y = 0; y < 8; ++y) t += red[y][threadIdx.x];
        part[(int64_t)blockIdx.y * n + j] = t;
    }
}

void bias_grad(const __nv_bfloat16 *g, int B, int ld, int n, float *part, float *out, cudaStream_t st)
{
    const int rb = (B + kBiasRows - 1) / kBiasRows;
    bias_grad_part<<<dim3((n + 31) / 32, rb), dim3(32, 8), 0, st>>>(g, B, ld, n, part);
    sum_slices<<<(n + 255) / 256, 256, 0, st>>>(part, rb, n, out);
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
    __nv_bfloat16 *w1, *w2, *w3, *w4, *w2t, *w3t;
    __nv_bfloat16 *x, *a1, *a2, *a3, *gy, *g3, *g2, *g1;
    __nv_bfloat16 *a1t, *a2t, *g2t, *g3t;
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
    p.a1t = (__nv_bfloat16 *)(W + w.a1t);
    p.a2t = (__nv_bfloat16 *)(W + w.a2t);
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

GemmArgs fwd_layer(int B, const __nv_bfloat16 *X, int K, const __nv_bfloat16 *W, int N,
                   const float *bias, float *z, __nv_bfloat16 *act, int epi, int nvalid)
{
    GemmArgs g{};
    g.M = B; g.N = N; g.K = K;
    g.A = X; g.sam = K; g.sak = 1;
    g.B = W; g.sbn = K; g.sbk = 1;
    g.epi = epi; g.bias = bias; g.z = z; g.act = act; g.ldo = N; g.nvalid = nvalid;
    return g;
}

// Layer l = 2, 3 on the tcgen05 GEMM: z = a_in W^T + b, act = SiLU(z), and
// with actT the transposed activations for the weight gradients.
int hidden_tc(const Ptrs &p, int B, const __nv_bfloat16 *ain, const __nv_bfloat16 *W, const float *bias,
              float *z, __nv_bfloat16 *act, __nv_bfloat16 *actT, cudaStream_t st)
{
    fk::TcEpilogue e{};
    e.kind = fk::TC_EPI_HIDDEN;
    e.ldo = H;
    e.ldT = p.ldT;
    e.bias = bias;
    e.z = z;
    e.act = act;
    e.actT = actT;
    e.status = p.status;
    return fk::tc_gemm(B, H, H, ain, H, W, H, 1, e, st);
}

// train: also the transposed activations the weight gradients need
int forward(const Ptrs &p, int B, const float *x, cudaStream_t st, bool train = false)
{
    if (cudaMemsetAsync(p.status, 0, sizeof(int), st) != cudaSuccess) return FK_ECUDA;
    pack_input<<<(B * INP + 255) / 256, 256, 0, st>>>(x, p.x, B);
    int rc;
    if ((rc = gemm(fwd_layer(B, p.x, INP, p.w1, H, p.master + OB1, p.z1, p.a1, EPI_HIDDEN, H), st))) return rc;
    if (train) transpose(p.a1, B, p.a1t, p.ldT, st);
    if ((rc = hidden_tc(p, B, p.a1, p.w2, p.master + OB2, p.z2, p.a2, train ? p.a2t : nullptr, st))) return rc;
    if ((rc = hidden_tc(p, B, p.a2, p.w3, p.master + OB3, p.z3, p.a3, nullptr, st))) return rc;
    GemmArgs g = fwd_layer(B, p.a3, H, p.w4, OUTP, p.master + OB4, p.y, nullptr, EPI_OUT, OUT);
    g.ldo = OUTP;
    return gemm(g, st);
}

// Back-propagate gy (bf16 [B][OUTP]) into parameter gradients p.gp (packed
// like master); writes g1 = dL/dz1 (bf16).
int backward(const Ptrs &p, int B, cudaStream_t st)
{
    int rc;
    // dL/dW4 = gy^T a3  ([OUT][H]); dL/db4
    GemmArgs g{};
    g.M = OUT; g.N = H; g.K = B;
    g.A = p.gy; g.sam = 1; g.sak = OUTP;          // A(m=j, k=b) = gy[b][j]
    g.B = p.a3; g.sbn = 1; g.sbk = H;             // B(n, k=b) = a3[b][n]
    g.epi = EPI_WGRAD; g.wgrad = p.gp + OW4; g.ldo = H; g.nvalid = H;
    g.ksplit = ksplit(B); g.wpart = p.wpart;
    if ((rc = gemm(g, st))) return rc;
    bias_grad(p.gy, B, OUTP, OUT, p.bpart, p.gp + OB4, st);
    // dL/dz3 = (gy W4) * silu'(z3)
    g = GemmArgs{};
    g.M = B; g.N = H; g.K = OUTP;
    g.A = p.gy; g.sam = OUTP; g.sak = 1;
    g.B = p.w4; g.sbn = 1; g.sbk = H;             // B(n=h, k=j) = W4[j][h]
    g.epi = EPI_BACK_HIDDEN; g.act = p.g3; g.zprev = p.z3; g.ldo = H; g.nvalid = H;
    if ((rc = gemm(g, st))) return rc;
    transpose(p.g3, B, p.g3t, p.ldT, st);
    // layers 3 and 2 on the tcgen05 GEMM: dL/dW = g^T a_in (K = batch, split
    // over CTAs, fixed-order sum), then dL/dz_in = (g W) * silu'(z_in)
    const __nv_bfloat16 *gT[2] = {p.g3t, p.g2t}, *aT[2] = {p.a2t, p.a1t}, *gl[2] = {p.g3, p.g2};
    const __nv_bfloat16 *Wt[2] = {p.w3t, p.w2t};
    const float *zp[2] = {p.z2, p.z1};
    __nv_bfloat16 *gout[2] = {p.g2, p.g1}, *goutT[2] = {p.g2t, nullptr};
    const int64_t ow[2] = {OW3, OW2}, ob[2] = {OB3, OB2};
    for (int l = 0; l < 2; ++l) {
        fk::TcEpilogue e{};
        e.kind = fk::TC_EPI_PARTIAL;
        e.ldo = H;
        e.out = p.wpart;
        e.sum_to = p.gp + ow[l];
        e.status = p.status;
        if ((rc = fk::tc_gemm(H, H, B, gT[l], p.ldT, aT[l], p.ldT, tc_ksplit(B), e, st))) return rc;
        bias_grad(gl[l], B, H, H, p.bpart, p.gp + ob[l], st);
        fk::TcEpilogue b{};
        b.kind = fk::TC_EPI_BACK_HIDDEN;
        b.ldo = H;
        b.ldT = p.ldT;
        b.act = gout[l];
        b.actT = goutT[l];
        b.zprev = zp[l];
        b.status = p.status;
        if ((rc = fk::tc_gemm(B, H, H, gl[l], H, Wt[l], H, 1, b, st))) return rc;
    }
    // layer 1: dL/dW1 = g1^T x (the 15 real inputs), dL/db1
    g = GemmArgs{};
    g.M = H; g.N = INP; g.K = B;
    g.A = p.g1; g.sam = 1; g.sak = H;
    g.B = p.x; g.sbn = 1; g.sbk = INP;
    g.epi = EPI_WGRAD; g.wgrad = p.gp + OW1; g.ldo = IN; g.nvalid = IN;
    g.ksplit = ksplit(B); g.wpart = p.wpart;
    if ((rc = gemm(g, st))) return rc;
    bias_grad(p.g1, B, H, H, p.bpart, p.gp + OB1, st);
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
        (__nv_bfloat16 *)(S + s.w3t));
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
    // upstream gradient [B][OUT] fp32 -> padded bf16
    if (cudaMemsetAsync(p.gy, 0, (size_t)batch * OUTP * 2, st) != cudaSuccess) return FK_ECUDA;
    pack_grad<<<(unsigned)((batch * OUT + 255) / 256), 256, 0, st>>>(gy, p.gy, batch);
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
    loss_grad<<<(batch * OUTP + 255) / 256, 256, 0, st>>>(p.y, target, p.gy, p.loss, batch);
    if ((rc = backward(p, batch, st))) return rc;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<(unsigned)((NPARAM + 255) / 256), 256, 0, st>>>(p.master, p.m, p.v, p.gp, NPARAM,
                                                                  lr, beta1, beta2, eps, c1, c2);
    refresh_bf16<<<(unsigned)((NW2 + 255) / 256), 256, 0, st>>>(p.master, p.w1, p.w2, p.w3, p.w4, p.w2t,
                                                                p.w3t);
    if (loss && cudaMemcpyAsync(loss, p.loss, 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return FK_ECUDA;
    return cudaGetLastError() == cudaSuccess ? FK_OK : FK_ECUDA;
}

}  // extern "C"
