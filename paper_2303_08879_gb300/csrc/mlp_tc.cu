// mlp_tc.cu -- the 256-wide GEMMs of the proposal MLP on the fifth-generation
// tensor cores: C = A B^T with A [M][K] and B [N][K] bf16 (both K-major, rows
// of K contiguous), fp32 accumulation in tensor memory.
//
// One CTA of 8 warps computes a 128 x 256 tile of C (the 128 TMEM lanes are
// the rows, 256 fp32 TMEM columns the columns).  The K loop runs in steps of 64 bf16
// (one 128-byte row per tile row): warp 0 (one lane) loads the A and B tiles
// of a step with TMA (cp.async.bulk.tensor, 128-byte swizzle) into a 2-stage
// ring of shared memory (about 97 KB, so two CTAs share an SM and one's
// epilogue overlaps the other's loads), warp 1 (one lane) issues four tcgen05.mma of K = 16
// per step and frees the stage with tcgen05.commit; when the last MMA has
// landed every warp reads 32 TMEM lanes of half the columns (tcgen05.ld) and
// applies the layer's epilogue.  A K range split over blockIdx.z (the weight gradients,
// whose K is the batch) writes fp32 partials that a second kernel sums in a
// fixed order.
//
// Every wait on an mbarrier is bounded; on expiry the CTA records FK_ETIMEOUT
// in the caller's status word, skips the rest of its work, still frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <stdint.h>

#include "mlp_tc.h"
#include "../../include/fockdiag.h"

namespace fk {

namespace {

constexpr int TBM = 128, TBN = 256, TBK = 64, STAGES = 2, TPB_TC = 256;
constexpr uint32_t A_BYTES = TBM * TBK * 2, B_BYTES = TBN * TBK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = 256;
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 /* alignment */ + 256 /* barriers */;
constexpr unsigned kSpinLimit = 1u << 26;   // about a second of polling per wait

struct TcArgs {
    int M, N, K, kper;         // k range of a CTA: [z kper, (z + 1) kper)
    TcEpilogue e;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the phase of parity `parity` to complete; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile stored as rows of 128
// bytes with the 128-byte swizzle (what TMA writes for a 64-wide bf16 box):
// start address >> 4, leading byte offset 16 (unused for this layout), stride
// byte offset 1024 (8 rows x 128 bytes), descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N = TBN, M = TBM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                            ((uint32_t)(TBM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t accum)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
        ::"r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }

__device__ __forceinline__ float dsilu(float z)
{
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

__global__ void __launch_bounds__(TPB_TC, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb,
                   const __grid_constant__ TcArgs g)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;   // 128-byte swizzle atoms: 1 KB aligned
    const uint32_t bars = base + STAGES * STAGE_BYTES;               // full[S], empty[S], done
    const uint32_t full0 = bars, empty0 = bars + 8 * STAGES, done = bars + 16 * STAGES;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    const int kbeg = blockIdx.z * g.kper, kend = min(g.K, kbeg + g.kper);
    const int nk = kend > kbeg ? (kend - kbeg + TBK - 1) / TBK : 0;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(full0 + 8 * i, 1);
            mbar_init(empty0 + 8 * i, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {   // tensor memory for the 128 x 256 fp32 accumulator
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&s_tmem)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (warp == 0 && lane == 0 && nk > 0) {
        // producer: TMA loads of the A and B tiles of each K step
        for (int kt = 0; kt < nk; ++kt) {
            const int st = kt % STAGES;
            if (kt >= STAGES && !mbar_wait(empty0 + 8 * st, ((kt / STAGES) & 1) ^ 1)) {
                atomicExch(&s_abort, 1);
                break;
            }
            if (*(volatile int *)&s_abort) break;
            const uint32_t sa = base + st * STAGE_BYTES, sb = sa + A_BYTES;
            mbar_expect_tx(full0 + 8 * st, STAGE_BYTES);
            tma_load_2d(sa, &ma, kbeg + kt * TBK, m0, full0 + 8 * st);
            tma_load_2d(sb, &mb, kbeg + kt * TBK, n0, full0 + 8 * st);
        }
    } else if (warp == 1 && lane == 0 && nk > 0) {
        // MMA issuer: four K = 16 MMAs per stage, then free the stage
        for (int kt = 0; kt < nk; ++kt) {
            const int st = kt % STAGES;
            if (!mbar_wait(full0 + 8 * st, (kt / STAGES) & 1)) {
                atomicExch(&s_abort, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = base + st * STAGE_BYTES, sb = sa + A_BYTES;
            const uint64_t ad = smem_desc(sa), bd = smem_desc(sb);
#pragma unroll
            for (int kk = 0; kk < TBK / 16; ++kk)   // 32 bytes of K per MMA: start address + 2 (16-byte units)
                mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, (kt > 0 || kk > 0) ? 1u : 0u);
            mma_commit(empty0 + 8 * st);
        }
        mma_commit(done);   // arrives once every MMA issued above has completed
    }
    __syncwarp();
    // every warp: wait for the accumulator, then its 32 rows of the epilogue
    bool ok = true;
    if (nk > 0) ok = mbar_wait(done, 0);
    if (!ok) atomicExch(&s_abort, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    const bool aborted = *(volatile int *)&s_abort != 0;
    if (aborted && threadIdx.x == 0 && g.e.status) atomicCAS(g.e.status, 0, (int)FK_ETIMEOUT);
    if (!aborted) {
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 (the lanes its quarter may
        // access); warps w and w + 4 take the two halves of the columns.  A lane
        // holds one row of a 32-column chunk; row-major outputs go through the
        // warp's 32 x 33 staging tile in the (now idle) operand ring, so that each
        // store instruction writes one contiguous row; the transposed outputs are
        // written straight from the lane-per-row layout, which is already coalesced.
        const int q = warp & 3, half = warp >> 2;
        const int mrow0 = m0 + q * 32, m = mrow0 + lane;
        const TcEpilogue &e = g.e;
        float *fst = (float *)(smem_raw + (base - smem_u32(smem_raw))) + warp * (32 * 33 * 3 / 2 + 16);
        unsigned short *hst = (unsigned short *)(fst + 32 * 33);
        const int mrows = min(32, g.M - mrow0);
        for (int c0 = half * (TBN / 2); c0 < (half + 1) * (TBN / 2); c0 += 32) {
            float v[32];
            if (nk > 0) {
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.f;
            }
            const int n = n0 + c0;
            if (mrows <= 0 || n >= g.N) continue;
            const int nv = min(32, g.N - n);
            const bool in = m < g.M;
            __syncwarp();
            switch (e.kind) {
            case TC_EPI_HIDDEN:
            case TC_EPI_OUT: {
                const bool hid = e.kind == TC_EPI_HIDDEN;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float z = i < nv ? v[i] + e.bias[n + i] : 0.f;
                    const __nv_bfloat16 a = __float2bfloat16(silu(z));
                    fst[lane * 33 + i] = z;
                    hst[lane * 33 + i] = __bfloat16_as_ushort(a);
                    if (hid && e.actT && in && i < nv) e.actT[(int64_t)(n + i) * e.ldT + m] = a;
                }
                __syncwarp();
                if (lane < nv)
                    for (int r = 0; r < mrows; ++r) {
                        const int64_t o = (int64_t)(mrow0 + r) * e.ldo + n + lane;
                        e.z[o] = fst[r * 33 + lane];
                        if (hid) e.act[o] = __ushort_as_bfloat16(hst[r * 33 + lane]);
                    }
                break;
            }
            case TC_EPI_BACK_HIDDEN: {
                // z_prev rows in, coalesced, through the staging tile
                if (lane < nv)
                    for (int r = 0; r < mrows; ++r)
                        fst[r * 33 + lane] = e.zprev[(int64_t)(mrow0 + r) * e.ldo + n + lane];
                __syncwarp();
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const __nv_bfloat16 a = __float2bfloat16(v[i] * dsilu(fst[lane * 33 + i]));
                    hst[lane * 33 + i] = __bfloat16_as_ushort(a);
                    if (e.actT && in && i < nv) e.actT[(int64_t)(n + i) * e.ldT + m] = a;
                }
                __syncwarp();
                if (lane < nv)
                    for (int r = 0; r < mrows; ++r)
                        e.act[(int64_t)(mrow0 + r) * e.ldo + n + lane] = __ushort_as_bfloat16(hst[r * 33 + lane]);
                break;
            }
            case TC_EPI_PARTIAL: {
#pragma unroll
                for (int i = 0; i < 32; ++i) fst[lane * 33 + i] = v[i];
                __syncwarp();
                float *dst = e.out + (int64_t)blockIdx.z * g.M * e.ldo;
                if (lane < nv)
                    for (int r = 0; r < mrows; ++r)
                        dst[(int64_t)(mrow0 + r) * e.ldo + n + lane] = fst[r * 33 + lane];
                break;
            }
            default: break;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
}

__global__ void sum_partials(const float *part, int slices, int64_t n, float *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int z = 0; z < slices; ++z) s += part[(int64_t)z * n + i];
    out[i] = s;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// 2-D tensor map of a row-major bf16 matrix [rows][cols] with leading
// dimension ld (elements), box [box_rows][64] with the 128-byte swizzle.
int make_map(CUtensorMap *map, const void *ptr, int rows, int cols, int64_t ld, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return FK_ECUDA;
    if (((uintptr_t)ptr & 15u) || ((ld * 2) & 15)) return FK_EINVAL;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {(cuuint32_t)TBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? FK_OK : FK_ECUDA;
}

}  // namespace

int tc_gemm(int M, int N, int K, const void *A, int64_t lda, const void *B, int64_t ldb, int ksplit,
            const TcEpilogue &e, void *stream)
{
    if (M < 1 || N < 1 || K < 1 || (N > TBN && (N % TBN) != 0) || ksplit < 1) return FK_EINVAL;
    CUtensorMap ma, mb;
    int rc = make_map(&ma, A, M, K, lda, TBM);
    if (rc) return rc;
    if ((rc = make_map(&mb, B, N, K, ldb, TBN)) != 0) return rc;
    static std::once_flag attr;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr, [] {
        attr_err = cudaFuncSetAttribute((const void *)tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)SMEM_BYTES);
    });
    if (attr_err != cudaSuccess) return FK_ECUDA;
    TcArgs g;
    g.M = M;
    g.N = N;
    g.K = K;
    g.kper = ((K + ksplit - 1) / ksplit + TBK - 1) / TBK * TBK;
    g.e = e;
    const int zs = (K + g.kper - 1) / g.kper;
    const dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM, zs);
    cudaStream_t st = (cudaStream_t)stream;
    tc_gemm_kernel<<<grid, TPB_TC, SMEM_BYTES, st>>>(ma, mb, g);
    if (cudaGetLastError() != cudaSuccess) return FK_ECUDA;
    if (e.kind == TC_EPI_PARTIAL && e.sum_to) {
        const int64_t n = (int64_t)M * e.ldo;
        sum_partials<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(e.out, zs, n, e.sum_to);
        if (cudaGetLastError() != cudaSuccess) return FK_ECUDA;
    }
    return FK_OK;
}

int tc_gemm_slices(int K, int ksplit)
{
    const int kper = ((K + ksplit - 1) / ksplit + TBK - 1) / TBK * TBK;
    return (K + kper - 1) / kper;
}

}  // namespace fk

extern "C" int fk_tc_gemm_bf16(int M, int N, int K, const void *d_A, const void *d_B, float *d_C,
                               float *d_partials, int ksplit, int *d_status, void *stream)
{
    using namespace fk;
    if (!d_A || !d_B || !d_C) return FK_EINVAL;
    TcEpilogue e{};
    e.kind = TC_EPI_PARTIAL;
    e.ldo = N;
    e.status = d_status;
    if (ksplit > 1) {
        if (!d_partials) return FK_EINVAL;
        e.out = d_partials;
        e.sum_to = d_C;
    } else {
        e.out = d_C;
        e.sum_to = nullptr;
    }
    return tc_gemm(M, N, K, d_A, K, d_B, K, ksplit, e, stream);
}
