// walk_common.cuh -- device helpers shared by the persistent walk kernels:
// complex FP64 multiply-accumulate, the bounded grid-wide barrier, packed
// digit vectors and the level-count tables used to enumerate the pivots of
// one level (digit sum) of a mixed-radix box.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fk_internal.h"
#include "../../include/fockdiag.h"

namespace fk {

constexpr int kTabN = FK_MAX_CUTOFF + 2;

__device__ __forceinline__ double2 cfma(double2 a, double2 x, double2 acc)
{   // acc + a * x  (four DFMA)
    acc.x = fma(a.x, x.x, acc.x);
    acc.x = fma(-a.y, x.y, acc.x);
    acc.y = fma(a.x, x.y, acc.y);
    acc.y = fma(a.y, x.x, acc.y);
    return acc;
}

__device__ __forceinline__ double2 cfma_conj(double2 a, double2 x, double2 acc)
{   // acc + conj(a) * x
    acc.x = fma(a.x, x.x, acc.x);
    acc.x = fma(a.y, x.y, acc.x);
    acc.y = fma(a.x, x.y, acc.y);
    acc.y = fma(-a.y, x.x, acc.y);
    return acc;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 x)
{
    return make_double2(a.x * x.x - a.y * x.y, a.x * x.y + a.y * x.x);
}

__device__ __forceinline__ double2 rscale(double2 a, double s)
{
    return make_double2(a.x * s, a.y * s);
}

__device__ __forceinline__ double2 cadd(double2 a, double2 b)
{
    return make_double2(a.x + b.x, a.y + b.y);
}

__device__ __forceinline__ double2 czero() { return make_double2(0.0, 0.0); }

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Polling read of a word another block writes: strong, but without the
// acquire's invalidation of the SM's L1, which would take the cached lines of
// every other block resident on the SM (a waiting block polls every ~0.1 us);
// the waiter orders its later reads with one fence after the wait instead.
__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_status(const Control *ctl)
{
    return *(volatile const int *)&ctl->status;
}

// Set before the launch by the input scan of FK_FLAG_CHECK_FINITE and never
// written by a walk kernel, so every block of a launch reads the same value.
__device__ __forceinline__ bool skip_walk(const Control *ctl)
{
    return *(volatile const int *)&ctl->skip != 0;
}

// Grid-wide barrier of a cooperative launch.  Every wait is bounded by
// `timeout_ns`; on expiry the status word becomes FK_ETIMEOUT and all blocks
// leave.  Returns false once any error is recorded.
__device__ __forceinline__ bool grid_sync(Control *ctl, unsigned nblocks,
                                          unsigned long long timeout_ns)
{
    __shared__ int s_ok;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned gen = ld_acquire(&ctl->bar_gen);
        __threadfence();
        const unsigned prev = atomicAdd(&ctl->bar_count, 1u);
        if (prev == nblocks - 1) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            const unsigned long long t0 = gtimer();
            while (ld_relaxed(&ctl->bar_gen) == gen) {
                if (ld_status(ctl) != 0) break;
                if (gtimer() - t0 > timeout_ns) {
                    atomicCAS(&ctl->status, 0, (int)FK_ETIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = (ld_status(ctl) == 0);
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------------ debug checks
// Built with -DFK_DEBUG_CHECKS (a separate library, libfockdiag_debug.so),
// every index of an amplitude, adjoint, scratch, output or geometry access is
// checked against the storage box it must lie in.  A violation is counted in
// the launch's control block (the first one with its source line, index and
// box) and the access is redirected to the first entry of the same box, so
// the check itself never reads or writes outside the buffers.  The normal
// build compiles the checks away.
#ifdef FK_DEBUG_CHECKS
__device__ __forceinline__ Control *&dbg_ctl()
{
    __shared__ Control *p;
    return p;
}

// Called by every thread at kernel entry, before the first checked access.
__device__ __forceinline__ void dbg_begin(Control *ctl)
{
    if (threadIdx.x == 0) dbg_ctl() = ctl;
    __syncthreads();
}

static __device__ __noinline__ void dbg_record(long long i, long long lo, long long hi, int site)
{
    Control *ctl = dbg_ctl();
    if (atomicAdd(&ctl->dbg_count, 1) == 0) {
        ctl->dbg_site = site;
        ctl->dbg_index = i;
        ctl->dbg_lo = lo;
        ctl->dbg_hi = hi;
    }
}
#define FK_DBG_BEGIN(ctl) ::fk::dbg_begin(ctl)
#else
#define FK_DBG_BEGIN(ctl) ((void)0)
#endif

// Index i of an access that must lie in [lo, hi) (see above).
__device__ __forceinline__ int64_t in_box(int64_t i, int64_t lo, int64_t hi, int site)
{
#ifdef FK_DEBUG_CHECKS
    if (i < lo || i >= hi) {
        dbg_record(i, lo, hi, site);
        return lo;
    }
#else
    (void)lo;
    (void)hi;
    (void)site;
#endif
    return i;
}
#define FK_BOX(i, lo, hi) ::fk::in_box((int64_t)(i), (int64_t)(lo), (int64_t)(hi), __LINE__)

// Per-level device timestamps of the debug-checks build: after each grid
// barrier of a walk, thread 0 of block 0 appends (tag, %globaltimer) to a
// caller-registered buffer (word 0: the number of records).
__device__ __forceinline__ void trace_mark(unsigned long long *buf, int cap, unsigned tag)
{
#ifdef FK_DEBUG_CHECKS
    if (buf != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long n = atomicAdd(buf, 1ull);
        if ((long long)n < (long long)cap) {
            buf[1 + 2 * n] = tag;
            buf[2 + 2 * n] = gtimer();
        }
    }
#else
    (void)buf;
    (void)cap;
    (void)tag;
#endif
}

// Up to 16 digits of at most 8 bits, packed in two registers.
struct Dig {
    uint64_t lo = 0, hi = 0;
    __device__ __forceinline__ int operator()(int i) const
    {
        const uint64_t w = i < 8 ? lo : hi;
        return (int)((w >> (8 * (i & 7))) & 0xffu);
    }
    __device__ __forceinline__ void set(int i, int v)
    {
        if (i < 8) lo |= (uint64_t)v << (8 * i);
        else hi |= (uint64_t)v << (8 * (i - 8));
    }
};

// Level-count table: W[i][t] = number of digit vectors over modes i..M-1
// (extents C_i) with digit sum t; row M is [t == 0].
struct LevelTab {
    const unsigned *W;
    int Wn;   // row length (max digit sum + 2)
    __device__ __forceinline__ unsigned at(int i, int t) const
    {
        return (t < 0 || t >= Wn) ? 0u : W[i * Wn + t];
    }
};

// The same counts kept as prefix sums over t: S[i][t] = sum_{u <= t} W[i][u]
// (one table serves counts, level offsets and lexicographic ranks).
struct PrefixTab {
    const unsigned *S;
    int Wn;
    __device__ __forceinline__ unsigned pre(int i, int t) const
    {
        return t < 0 ? 0u : S[i * Wn + (t < Wn ? t : Wn - 1)];
    }
    __device__ __forceinline__ unsigned at(int i, int t) const
    {
        return (t < 0 || t >= Wn) ? 0u : pre(i, t) - pre(i, t - 1);
    }
};

// Block-cooperative construction of the table for cutoffs C[0..M-1].
__device__ __forceinline__ void build_level_table(unsigned *W, int Wn, const int *C, int M)
{
    for (int t = threadIdx.x; t < Wn; t += blockDim.x) W[M * Wn + t] = (t == 0) ? 1u : 0u;
    __syncthreads();
    for (int i = M - 1; i >= 0; --i) {
        for (int t = threadIdx.x; t < Wn; t += blockDim.x) {
            unsigned acc = 0;
            for (int v = 0; v < C[i] && v <= t; ++v) acc += W[(i + 1) * Wn + t - v];
            W[i * Wn + t] = acc;
        }
        __syncthreads();
    }
}

// Block-cooperative prefix form: W, then each row summed in place.
__device__ __forceinline__ void build_prefix_table(unsigned *S, int Wn, const int *C, int M)
{
    build_level_table(S, Wn, C, M);
    for (int i = threadIdx.x; i <= M; i += blockDim.x) {
        unsigned acc = 0;
        for (int t = 0; t < Wn; ++t) {
            acc += S[i * Wn + t];
            S[i * Wn + t] = acc;
        }
    }
    __syncthreads();
}

// Number of digit vectors over modes k0..M-1 with digit k0 in [0, C_k0 - dk0)
// and the others in [0, C_i), summing to s.
template <class Tab>
__device__ __forceinline__ unsigned level_count(const int *C, const Tab &W, int k0, int dk0, int s)
{
    unsigned n = 0;
    for (int v = 0; v < C[k0] - dk0; ++v) n += W.at(k0 + 1, s - v);
    return n;
}

// The rank-th such vector in lexicographic order (mode k0 slowest).
template <class Tab>
__device__ __forceinline__ Dig unrank(const int *C, int M, const Tab &W, int k0, int dk0, int s,
                                      unsigned rank)
{
    Dig d;
    int rem = s;
    for (int i = k0; i < M; ++i) {
        const int ext = C[i] - (i == k0 ? dk0 : 0);
        int v = 0;
        for (; v < ext - 1; ++v) {
            const unsigned c = W.at(i + 1, rem - v);
            if (rank < c) break;
            rank -= c;
        }
        d.set(i, v);
        rem -= v;
    }
    return d;
}

// Reciprocals 1/v and factorials v! for v < kTabN (block-cooperative).
__device__ __forceinline__ void build_scalar_tables(double *inv, double *fact)
{
    for (int v = threadIdx.x; v < kTabN; v += blockDim.x) {
        inv[v] = v > 0 ? 1.0 / (double)v : 0.0;
        double f = 1.0;
        for (int u = 2; u <= v; ++u) f *= (double)u;
        fact[v] = f;
    }
}

}  // namespace fk
