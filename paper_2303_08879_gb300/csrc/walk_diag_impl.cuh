// walk_diag_impl.cuh -- persistent sm_103a kernels for the all-detected walk
// (Algorithm 1 of arXiv 2303.08879, Sec. 3.1) and its reverse-mode adjoint
// (the chain rule of Sec. 2.5 run backwards through the same walk).
//
// Arithmetic.  The kernels carry F_k = G_k / sqrt(k!) instead of G_k.  Eq.
// (recrel) then reads
//     F_{P+1_w} = (b_w F_P + sum_l A_wl F_{P-1_l}) / (P_w + 1),
// the rescaled matrix-vector form the paper mentions in Sec. 4: every term
// of a sum carries the same factor sqrt(P!) relative to the original form,
// so no read needs its own sqrt weight and each write is one complex
// matrix-vector row times a reciprocal from a table.  Probabilities are
// G_d = F_d * prod_j d_j!.  Values are IEEE complex128.  Two product engines:
// FP64 (Gauss's three-multiplication complex product, 3 DFMA per term) and
// the tensor-core engine (exact base-256 digit products on fp16 MMAs,
// recombined in int64: the same sums with an error near 2^-53 of the
// largest term).
//
// Parallel structure.  One cooperative persistent launch walks every level
// s = 0..L-1 (pivot digit sum, Sec. 2.2: pivots of equal weight are
// independent) for all circuits of the batch; a grid-wide barrier with a
// time limit separates the phases.  A level is split into tiles of 128
// pivots of one (anchor K, circuit) segment, handed to blocks through a
// counter; a thread owns one pivot: it takes the pivot's geometry (from a
// table shared by the circuits when M <= 8), gathers its reads into shared
// memory, runs the 2(M-K) x 2(M-K) complex matrix-vector product against A
// held in shared memory, and scatters the writes.  The VJP runs the levels
// backwards; with the tensor engine its partial dL/dA and dL/db sums are a
// second launch over all pivots once the walk is done.
//
// This header holds the kernels as templates over the tile shape and engine;
// walk_diag_fp64.cu and walk_diag_tc.cu instantiate them (in parallel
// translation units) and hand their addresses to the host code of
// walk_diag.cu.
#pragma once

#include <cuda_runtime.h>

#include "fk_internal.h"
#include "walk_common.cuh"
#include "walk_digits.cuh"
#include "../../include/fockdiag.h"

namespace fk {

namespace {

constexpr int TABN = kTabN;

struct DiagArgs {
    DiagShape sh;
    int B;
    int grid;
    int slots;                    // partial-sum slots per circuit (grid x slots per block)
    unsigned flags;
    const double2 *A, *b, *c;     // caller layout, D_orig
    double2 *probs;
    Control *ctl;
    double2 *As, *bs, *F;
    unsigned char *dig;           // tensor engine: per-circuit digit fragments of A (kDigBytes each)
    int *geo;                     // AP pivot geometry shared by the circuits (M <= 8), or null
    int *ctr;                     // [4 (L + 1)] next-tile counters: DP phase of level l at 2l, AP at
                                  // 2l + 1; the tensor engine's partial pass at 2 (L + 1) + the same
    const double2 *gprobs;
    double2 *Fbar, *scratch, *partA, *partb;
    double2 *gA, *gb, *gc;
    unsigned long long timeout_ns;
    // early stop on the probability sum (Sec. 2.3): lvl[c][n] = fixed-point
    // (2^56) sum of the probabilities with n photons written so far
    int early;
    unsigned long long thr;       // (1 - eps) 2^56
    unsigned long long *lvl;      // [B][L + 2]
    int *levels;                  // [B] photon numbers completed (device, optional)
    // several shapes in one launch (G > 0): sh is then the envelope (largest
    // kept M and L, has_b) that sizes shared memory, and each group's own
    // arguments are views written by the kernel's prologue
    int G;
    const DiagGroup *grp;         // [G]
    DiagArgs *gargs;              // [G] views: the group's shape, circuits and workspace regions
    const int *gtiles;            // [L][2][G + 1] tile prefix sums per phase
    const int *cidx;              // caller's circuit index of each local circuit (null: identity)
    const int64_t *oidx;          // output offset of each local circuit (null: circ * n_diag)
    char *wsbase;
    // debug-checks build: per-level timestamps (see trace_mark), or null
    unsigned long long *trace;
    int trace_cap;
    // circuit-per-block mode (batches of at least twice as many circuits as
    // blocks): each block walks whole circuits taken from a counter, with block
    // barriers between its phases instead of grid barriers
    int pc;
    // key of the pivot geometry table for this shape and workspace (0: none);
    // geo_reuse: the table may be taken as built when the workspace's control
    // block holds the same key (the reverse walk after its forward)
    unsigned long long geo_key;
    int geo_reuse;
    int pad_geo;
};

// ------------------------------------------------------------ shared memory
struct Smem {
    unsigned *S;      // [(M+1)][L+2]: S[i][t] = number of digit vectors over modes
                      // i..M-1 (extents C) with digit sum <= t
    int64_t *cum0;    // [M] offset of the current phase's level in family K
    int64_t *cum1;    // [M] offset of the level below
    int64_t *cum2;    // [M] offset of the level above
    int Wn;           // row length
    double *inv;      // 1/v
    double *fact;     // v!
    double *A3;       // [3][D][D]: Re A, Re A + Im A, Im A - Re A of the tile's circuit
    double2 *bs;      // D
    double *R3;       // [3][D][RS] reads per pivot (three planes, see store_read)
    double *Y3;       // [3][D][RS] scaled output adjoints per pivot (VJP)
    double2 *FP;      // [RS] pivot values (VJP, b != 0)
    uint4 *Af;        // tensor-core engine: [KS][KS][7][32] fp16 digit fragments of the real
                      // form of A (m16n8k16 A-operand order, one 16-byte word per lane)
    int *fA;          // tensor-core engine: [2D] row exponent fields e_r
    double *wb;       // tensor-core engine: per-warp [16 KS][WBS] reads in, products out
    double *wy;       // tensor-core VJP: per-warp [16 KS][WBS] scaled output adjoints
    int *wf;          // tensor-core VJP: [TPB] exponent field of each pivot's largest read
    int *wg;          // tensor-core VJP: per-warp [32] row exponents of the partial dL/dA
    int *idx;         // [M][TPB] box indices per pivot
    int *tiles;       // [M + 2] tile prefix sums of the current phase, then [M + 2] the
                      // pivots of each segment
    int loaded_circ;
    int multi_key;    // several shapes: (group, level, kind) the tables hold, or -1
};

// ---------------------------------------------------------------- geometry
struct TileId {
    int seg, circ;
    unsigned rank0, count;
};

// AP(K) pivot with base e: read column j / write row i addresses and masks.
// (level-major addresses inside the circuit's amplitude array, see fk_shape.h)
struct ApGeom {
    int64_t r;        // rank of the pivot e in family K at its level s
    int64_t rd;       // DIAG[e]            (level s)
    int64_t rt2;      // T2(K)[e - 1_K]     (level s - 1; valid if e_K >= 1)
    int64_t wt2;      // T2(K)[e]
    int64_t wdiag;    // DIAG[e + 1_K]      (level s + 1)
    int64_t pout;     // caller's probability index of e + 1_K (row-major over modes)
    int64_t lk0, lkm; // family-K offsets of levels s and s - 1
    int64_t fp;       // T1K(K)[e] (pivot value, b != 0)
    unsigned vmask;   // valid reads
    unsigned nmask;   // needed writes
};

// DP pivot d (b != 0): read column j = 2q -> T1B(q)[d-1_q], 2q+1 -> T1K(q)[d-1_q];
// write row i = 2q -> T1K(q)[d], 2q+1 -> T1B(q)[d].
struct DpGeom {
    int64_t r;        // rank of d in family 0 at its level s
    int64_t rdiag;    // DIAG[d] (the pivot value)
    int64_t l00, l0m; // family-0 offsets of levels s and s - 1
    unsigned vmask, nmask;
};

// Trace tags (debug-checks build): kernel in bits 24.., level in bits 8..23,
// phase (0 = AP, 1 = DP) in bit 0.
constexpr unsigned kTraceFwd = 1u << 24, kTraceVjp = 2u << 24, kTraceFinish = 3u << 24;

// Shared-memory layouts of the walk kernels (see Walk::smem_plan).
constexpr int kFwd = 0, kVjp = 1, kPart = 2;

// The walk for one tile shape: TPB pivots per tile (= threads per block) and
// either CH output rows per FP64 register chunk (KS = 0) or, for KS > 0, the
// tensor-core digit engine with up to 16 KS real rows (M <= 4 KS); the
// autotuner picks the instantiation.
template <int TPB, int CH, int KS = 0>
struct Walk {
    static constexpr int RS = TPB + 1;   // padded row stride of per-thread smem columns
    static constexpr bool TC = KS > 0;   // forward products on the tensor cores
    static constexpr int XS = 16 * (KS > 0 ? KS : 1);   // rows of a per-warp buffer
    static constexpr int WBS = 34;       // column stride (doubles) of a per-warp buffer
    static constexpr int NDIG = kNDig;   // base-256 digits per value (Sec. 2.1 accuracy)

    // Shared-memory plan, one for sizing (host) and carving (device) so the two
    // cannot disagree.  Modes: kFwd the forward walk; kVjp the reverse walk
    // (FP64 engine: with the partial dL/dA; tensor engine: products only, in
    // place in the adjoint buffer); kPart the tensor engine's partial dL/dA
    // pass.  Absent regions have offset kNone.
    static constexpr size_t kNone = ~(size_t)0;
    struct SmemPlan {
        size_t S, cum, inv, bs, fA, wb, wy, FP, wf, wg, Af, A3, R3, Y3, idx, tiles, bytes;
    };

    static __host__ __device__ SmemPlan smem_plan(int M, int L, int mode, bool has_b)
    {
        SmemPlan q;
        q.bs = q.fA = q.wb = q.wy = q.FP = q.wf = q.wg = q.Af = q.A3 = q.R3 = q.Y3 = q.idx = kNone;
        const int D = 2 * M, D2 = 2 * D;
        size_t n = 0;
        const auto al = [&n]() { n = (n + 15) & ~(size_t)15; };
        q.S = n; n += (size_t)(M + 1) * (L + 2) * sizeof(unsigned); al();
        q.cum = n; n += 3 * (size_t)M * sizeof(int64_t); al();
        q.inv = n; n += 2 * TABN * sizeof(double); al();
        if (TC) {
            const size_t buf = (size_t)(TPB / 32) * XS * WBS * sizeof(double);
            if (mode != kPart) {
                q.bs = n; n += (size_t)D * sizeof(double2);
                q.fA = n; n += (size_t)D2 * sizeof(int); al();
                q.Af = n; n += (size_t)KS * KS * NDIG * 32 * sizeof(uint4); al();
            }
            if (mode != kVjp) { q.wb = n; n += buf; al(); }
            if (mode != kFwd) { q.wy = n; n += buf; al(); }
            if (mode == kPart) {
                if (has_b) { q.FP = n; n += (size_t)TPB * sizeof(double2); }
                q.wf = n; n += (size_t)TPB * sizeof(int);
                q.wg = n; n += (size_t)TPB * sizeof(int); al();
            }
            // the forward and the partial pass keep AP read ranks in registers
            if (mode == kVjp || has_b) { q.idx = n; n += (size_t)M * TPB * sizeof(int); al(); }
        } else {
            q.A3 = n; n += 3 * (size_t)D * D * sizeof(double); al();
            q.bs = n; n += (size_t)D * sizeof(double2); al();
            q.R3 = n; n += 3 * (size_t)D * RS * sizeof(double); al();
            if (mode == kVjp) {
                q.Y3 = n; n += 3 * (size_t)D * RS * sizeof(double); al();
                q.FP = n; n += RS * sizeof(double2); al();
            }
            q.idx = n; n += (size_t)M * TPB * sizeof(int); al();
        }
        q.tiles = n; n += 2 * (M + 2) * sizeof(int);
        q.bytes = n + 64;
        return q;
    }

    static __host__ __device__ size_t smem_bytes(int M, int L, int mode, bool has_b)
    {
        return smem_plan(M, L, mode, has_b).bytes;
    }

    static __device__ Smem carve_smem(const DiagShape &sh, int mode)
    {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        const SmemPlan q = smem_plan(sh.M, sh.L, mode, sh.has_b != 0);
        const auto at = [&](size_t o) { return o == kNone ? nullptr : (void *)(smem_raw + o); };
        const int M = sh.M;
        Smem s;
        s.S = (unsigned *)at(q.S);
        s.Wn = sh.L + 2;
        s.cum0 = (int64_t *)at(q.cum);
        s.cum1 = s.cum0 + M;
        s.cum2 = s.cum0 + 2 * M;
        s.inv = (double *)at(q.inv);
        s.fact = s.inv + TABN;
        s.bs = (double2 *)at(q.bs);
        s.fA = (int *)at(q.fA);
        s.Af = (uint4 *)at(q.Af);
        s.wb = (double *)at(q.wb);
        s.wy = (double *)at(q.wy);
        s.FP = (double2 *)at(q.FP);
        s.wf = (int *)at(q.wf);
        s.wg = (int *)at(q.wg);
        s.A3 = (double *)at(q.A3);
        s.R3 = (double *)at(q.R3);
        s.Y3 = (double *)at(q.Y3);
        s.idx = (int *)at(q.idx);
        s.tiles = (int *)at(q.tiles);
        s.loaded_circ = -1;
        s.multi_key = -1;
        return s;
    }

    // Level-count, reciprocal and factorial tables (every block builds its own
    // copy; they depend on the cutoffs only).
    static __device__ void build_tables(const DiagShape &sh, Smem &s)
    {
        build_scalar_tables(s.inv, s.fact);
        build_prefix_table(s.S, s.Wn, sh.C, sh.M);
    }

    // Level-major ranks.  For a family over modes k0..M-1 (suffix extents C),
    // the rank of x among the vectors of its digit sum in lexicographic order
    // is sum_i Pf(i, t_i, x_i) with t_i the digit sum of x_i..x_{M-1} and
    //   Pf(i, t, x) = sum_{v < x} W[i+1][t - v] = S[i+1][t] - S[i+1][t - x].
    // A restriction x_k0 <= C_k0 - 2 never changes the rank of an admitted x.
    static __device__ __forceinline__ unsigned Sv(const Smem &s, int i, int t)
    {
        return t < 0 ? 0u : s.S[i * s.Wn + (t < s.Wn ? t : s.Wn - 1)];
    }

    static __device__ __forceinline__ int64_t Pf(const Smem &s, int i, int t, int x)
    {
        return (int64_t)(Sv(s, i + 1, t) - Sv(s, i + 1, t - x));
    }

    // Offset of level `lev` in the DIAG family (all modes, all digits).
    static __device__ __forceinline__ int64_t cum_full(const Smem &s, int lev)
    {
        return (int64_t)Sv(s, 0, lev - 1);
    }

    // Offset of level `lev` in family K: sum over the levels below of the
    // family's counts Pf(K, l, C_K - 1).  Warp 0 fills s.cum0 / s.cum1 /
    // s.cum2 for the level of each phase, the one below and the one above:
    // its lanes take the levels l = lane (mod 32) and a butterfly adds them,
    // instead of one thread walking M x lev table entries in a row while the
    // block waits.
    static __device__ void phase_offsets(const DiagShape &sh, Smem &s, int lev)
    {
        const int lane = threadIdx.x & 31;
        for (int K = 0; K < sh.M; ++K) {
            long long c0 = 0, c1 = 0;
            for (int l = lane; l < lev; l += 32) {
                const long long n = Pf(s, K, l, sh.C[K] - 1);
                c0 += n;
                if (l + 1 < lev) c1 += n;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                c0 += __shfl_xor_sync(0xffffffffu, c0, o);
                c1 += __shfl_xor_sync(0xffffffffu, c1, o);
            }
            if (lane == 0) {
                s.cum0[K] = c0;
                s.cum1[K] = c1;
                s.cum2[K] = c0 + Pf(s, K, lev, sh.C[K] - 1);
            }
        }
    }

    static __device__ __forceinline__ PrefixTab ltab(const Smem &s) { return PrefixTab{s.S, s.Wn}; }

    static __device__ __forceinline__ unsigned level_count(const DiagShape &sh, const Smem &sm, int k0,
                                                    int dk0, int s)
    {
        return fk::level_count(sh.C, ltab(sm), k0, dk0, s);
    }

    static __device__ __forceinline__ Dig unrank(const DiagShape &sh, const Smem &sm, int k0, int dk0, int s,
                                          unsigned rank)
    {
        return fk::unrank(sh.C, sh.M, ltab(sm), k0, dk0, s, rank);
    }

    // Load A_s (symmetric part, kept modes) and b of one circuit into smem.
    // A is kept as three real planes for Gauss's three-multiplication complex
    // product: Re A, Re A + Im A and Im A - Re A.
    static __device__ void load_circuit(const DiagArgs &a, Smem &s, int circ)
    {
        if (s.loaded_circ == circ) return;
        __syncthreads();
        const int D = 2 * a.sh.M, DD = D * D;
        const double2 *As = a.As + (size_t)circ * DD;
        if (TC && s.Af != nullptr) {
            // digit fragments prepared once per launch by build_digits
            const unsigned char *src = a.dig + (size_t)circ * kDigBytes;
            const uint4 *gf = (const uint4 *)(src + 256);
            for (int e = threadIdx.x; e < KS * KS * NDIG * 32; e += blockDim.x) s.Af[e] = __ldcg(gf + e);
            for (int r = threadIdx.x; r < 2 * D; r += blockDim.x) s.fA[r] = __ldcg((const int *)src + r);
            for (int e = threadIdx.x; e < D; e += blockDim.x) s.bs[e] = a.bs[(size_t)circ * D + e];
            __syncthreads();
            s.loaded_circ = circ;
            return;
        }
        for (int e = threadIdx.x; e < DD; e += blockDim.x) {
            const double2 v = As[e];
            s.A3[e] = v.x;
            s.A3[DD + e] = v.x + v.y;
            s.A3[2 * DD + e] = v.y - v.x;
        }
        for (int e = threadIdx.x; e < D; e += blockDim.x) s.bs[e] = a.bs[(size_t)circ * D + e];
        __syncthreads();
        s.loaded_circ = circ;
    }

    // Per-pivot gather of N values: load(j) gives value j, put(j, v) stores
    // it.  With the tensor engine the loop is unrolled to its largest length
    // so that every load is in flight before the first store (one memory
    // latency per gather instead of one per value).
    template <class Load, class Put>
    static __device__ __forceinline__ void gather(int N, Load load, Put put)
    {
        if constexpr (TC) {
            constexpr int NM = 8 * (KS > 0 ? KS : 1);
            double2 v[NM];
#pragma unroll
            for (int j = 0; j < NM; ++j) v[j] = j < N ? load(j) : make_double2(0, 0);
#pragma unroll
            for (int j = 0; j < NM; ++j)
                if (j < N) put(j, v[j]);
        } else {
            for (int j = 0; j < N; ++j) put(j, load(j));
        }
    }

    // Three planes of a read x: forward (Re x, Im x, Re x + Im x); reverse
    // (Re x, Re x - Im x, Re x + Im x).
    static __device__ __forceinline__ void store_read(Smem &s, int D, int j, int t, double2 x,
                                                      bool reverse)
    {
        if (TC) {
            double *w = s.wb + (size_t)(t >> 5) * XS * WBS + (t & 31);
            w[(2 * j) * WBS] = x.x;
            w[(2 * j + 1) * WBS] = x.y;
            return;
        }
        s.R3[(size_t)j * RS + t] = x.x;
        s.R3[(size_t)(D + j) * RS + t] = reverse ? x.x - x.y : x.y;
        s.R3[(size_t)(2 * D + j) * RS + t] = x.x + x.y;
    }

    // Three planes of a scaled output adjoint y: (Re y, Im y, Re y + Im y).
    static __device__ __forceinline__ void store_adj(Smem &s, int D, int i, int t, double2 y)
    {
        if (TC) {
            double *w = s.wy + (size_t)(t >> 5) * XS * WBS + (t & 31);
            w[(2 * i) * WBS] = y.x;
            w[(2 * i + 1) * WBS] = y.y;
            return;
        }
        s.Y3[(size_t)i * RS + t] = y.x;
        s.Y3[(size_t)(D + i) * RS + t] = y.y;
        s.Y3[(size_t)(2 * D + i) * RS + t] = y.x + y.y;
    }

    static __device__ __forceinline__ double2 load_adj(const Smem &s, int D, int i, int t)
    {
        if (TC) {
            const double *w = s.wy + (size_t)(t >> 5) * XS * WBS + (t & 31);
            return make_double2(w[(2 * i) * WBS], w[(2 * i + 1) * WBS]);
        }
        return make_double2(s.Y3[(size_t)i * RS + t], s.Y3[(size_t)(D + i) * RS + t]);
    }

    // Rows row0 + i (i in [0, N)) of A x for this thread's reads, CH rows at a
    // time: with x = xr + i xi and s = xr + xi,
    //   Re = sum Ar s - sum (Ar + Ai) xi,  Im = sum Ar s + sum (Ai - Ar) xr,
    // three DFMA per complex term.  `emit(i, value)` receives each row.
    template <bool HASB, class Emit>
    static __device__ __forceinline__ void matvec(const Smem &s, int D, int row0, int N,
                                                  unsigned vm, unsigned nm, double2 pv, Emit emit)
    {
        const int t = threadIdx.x, DD = D * D;
        const double *Ar = s.A3 + (size_t)row0 * D + row0;
        const double *Ap = Ar + DD, *Am = Ar + 2 * DD;
        for (int i0 = 0; i0 < N; i0 += CH) {
            if (((nm >> i0) & ((1u << CH) - 1u)) == 0) continue;
            double p1[CH], p2[CH], p3[CH];
#pragma unroll
            for (int ii = 0; ii < CH; ++ii) p1[ii] = p2[ii] = p3[ii] = 0.0;
            for (int j = 0; j < N; ++j) {
                if (!((vm >> j) & 1u)) continue;
                const double xr = s.R3[(size_t)j * RS + t];
                const double xi = s.R3[(size_t)(D + j) * RS + t];
                const double xs = s.R3[(size_t)(2 * D + j) * RS + t];
#pragma unroll
                for (int ii = 0; ii < CH; ++ii)
                    if (i0 + ii < N && ((nm >> (i0 + ii)) & 1u)) {
                        const size_t o = (size_t)(i0 + ii) * D + j;
                        p1[ii] = fma(Ar[o], xs, p1[ii]);
                        p2[ii] = fma(Ap[o], xi, p2[ii]);
                        p3[ii] = fma(Am[o], xr, p3[ii]);
                    }
            }
#pragma unroll
            for (int ii = 0; ii < CH; ++ii) {
                const int i = i0 + ii;
                if (i < N && ((nm >> i) & 1u)) {
                    double2 v = make_double2(p1[ii] - p2[ii], p1[ii] + p3[ii]);
                    if (HASB) v = cadd(v, cmul(s.bs[row0 + i], pv));
                    emit(i, v);
                }
            }
        }
    }

    // Caller's circuit index of local circuit c (its A, b, c and gradients)
    // and the offset of its outputs (probabilities, upstream gradients): a
    // launch of one shape uses the identity and c * n_diag; a group of a
    // launch of several shapes maps through its tables.
    static __device__ __forceinline__ size_t cix(const DiagArgs &a, int c)
    {
        return a.cidx ? (size_t)a.cidx[c] : (size_t)c;
    }
    static __device__ __forceinline__ size_t oix(const DiagArgs &a, int c)
    {
        return a.oidx ? (size_t)a.oidx[c] : (size_t)c * (size_t)a.sh.n_diag;
    }

    // Entry (w, l) of A_s = (A + A^T)/2 restricted to the kept modes, from the
    // caller's A (the same arithmetic as the prologue's copy).
    static __device__ __forceinline__ double2 as_entry(const DiagArgs &a, int c, int w, int l)
    {
        const DiagShape &sh = a.sh;
        const int Do = sh.D_orig;
        const int ow = 2 * sh.mode_map[w / 2] + (w & 1), ol = 2 * sh.mode_map[l / 2] + (l & 1);
        const double2 x = a.A[cix(a, c) * Do * Do + (size_t)ow * Do + ol];
        const double2 y = a.A[cix(a, c) * Do * Do + (size_t)ol * Do + ow];
        return make_double2(0.5 * (x.x + y.x), 0.5 * (x.y + y.y));
    }

    // Digit fragments of the real form R of every circuit's A_s (row 2i: Re
    // A_ij at column 2j, -Im A_ij at 2j+1; row 2i+1: Im A_ij, Re A_ij), padded
    // with zeros to 16 KS x 16 KS, in the register order of the A operand of
    // mma m16n8k16: tile (mt, ks), digit s, lane (grp, tig) holds rows
    // 16 mt + grp (+8) and columns 16 ks + 2 tig (+1, +8, +9).  Row r is fixed
    // point relative to the largest exponent field of its row of A.  One block
    // per circuit writes them to the workspace (row exponent fields first).
    static __device__ void build_digits(const DiagArgs &a, Smem &s)
    {
        const int D = 2 * a.sh.M, D2 = 2 * D;
        constexpr int P = 16 * (KS > 0 ? KS : 1);
        for (int circ = blockIdx.x; circ < a.B; circ += gridDim.x) {
            int *gA = (int *)(a.dig + (size_t)circ * kDigBytes);
            uint32_t *Af = (uint32_t *)(a.dig + (size_t)circ * kDigBytes + 256);
            __syncthreads();
            for (int r = threadIdx.x; r < D2; r += blockDim.x) s.fA[r] = 0;
            __syncthreads();
            for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
                const double2 v = as_entry(a, circ, e / D, e % D);
                const int f = max(fexp(v.x), fexp(v.y));
                if (f != 0) atomicMax(&s.fA[2 * (e / D)], f);
            }
            __syncthreads();
            for (int i = threadIdx.x; i < D; i += blockDim.x) s.fA[2 * i + 1] = s.fA[2 * i];
            __syncthreads();
            for (int r = threadIdx.x; r < D2; r += blockDim.x) gA[r] = s.fA[r];
            for (int e = threadIdx.x; e < P * P / 2; e += blockDim.x) {
                const int r = e / (P / 2), c = 2 * (e % (P / 2));
                uint32_t wd[NDIG];
                if (r < D2 && c < D2) {
                    const double2 v = as_entry(a, circ, r >> 1, c >> 1);
                    const double x0 = (r & 1) ? v.y : v.x, x1 = (r & 1) ? v.x : -v.y;
                    digit_words(to_fixed(x0, s.fA[r]), to_fixed(x1, s.fA[r]), wd);
                } else {
#pragma unroll
                    for (int sl = 0; sl < NDIG; ++sl) wd[sl] = 0u;
                }
                const int rr = r & 15, cc = c & 15;
                const int lane = (rr & 7) * 4 + ((cc & 7) >> 1), k = (rr >> 3) | ((cc >> 3) << 1);
                const int tile = (r >> 4) * KS + (c >> 4);
#pragma unroll
                for (int sl = 0; sl < NDIG; ++sl) Af[(((tile * NDIG + sl) * 32 + lane) << 2) + k] = wd[sl];
            }
        }
        __syncthreads();
    }

    // Products of the 32 pivots of this warp with the real form of A (CONJ:
    // of conj(A)) restricted to rows and columns from row0 (complex index):
    // out[r][p] = sum_c R[2 row0 + r][2 row0 + c] in[c][p] for r, c < 2N, in
    // and out per-warp buffers (row = real index 2j + {re, im} relative to
    // row0, column = lane).  The MMA tiles are the aligned 16 x 16 tiles of R
    // that the rows [2 row0, 2 row0 + 2N) meet; inputs outside that range
    // enter as zeros.  MMA tile m16n8k16: M = output real rows, N = 8 pivots,
    // K = input real rows.  out may alias in: an N tile is read before its
    // products land.
    template <bool CONJ>
    static __device__ __forceinline__ void tc_products(const Smem &s, int D, int row0, int N, double *in,
                                                       double *out)
    {
        const int lane = threadIdx.x & 31, grp = lane >> 2, tig = lane & 3;
        const int r0 = 2 * row0, n2 = 2 * N, t0 = r0 >> 4, t1 = (r0 + n2 + 15) >> 4;
        // conj(A) in real form: the Im A entries change sign (high half of a
        // fragment word in even rows, low half in odd rows; digits negate exactly)
        const uint32_t cflip = CONJ ? ((grp & 1) ? 0x00008000u : 0x80000000u) : 0u;
        const uint4 *Af = s.Af + lane;
#pragma unroll 1
        for (int nt = 0; nt < 4; ++nt) {
            const int p = nt * 8 + grp;
            double xv[KS][2][2];
            int fm = 0;
#pragma unroll
            for (int ks = 0; ks < KS; ++ks)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = 16 * ks + 8 * h + 2 * tig - r0;
                    const bool ok = ks >= t0 && ks < t1 && c >= 0 && c < n2;
                    xv[ks][h][0] = ok ? in[c * WBS + p] : 0.0;
                    xv[ks][h][1] = ok ? in[(c + 1) * WBS + p] : 0.0;
                    fm = max(fm, max(fexp(xv[ks][h][0]), fexp(xv[ks][h][1])));
                }
            fm = max(fm, __shfl_xor_sync(0xffffffffu, fm, 1));
            fm = max(fm, __shfl_xor_sync(0xffffffffu, fm, 2));
            // an N tile whose inputs all count as zero (inactive pivots at a
            // tile's end) has zero products: write them without the MMAs
            if (!__any_sync(0xffffffffu, fm >= 26)) {
                for (int r = tig; r < n2; r += 4) out[r * WBS + p] = 0.0;
                continue;
            }
            uint32_t bq[NDIG][KS][2];
#pragma unroll
            for (int ks = 0; ks < KS; ++ks)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t wd[NDIG];
                    digit_words(to_fixed(xv[ks][h][0], fm), to_fixed(xv[ks][h][1], fm), wd);
#pragma unroll
                    for (int sl = 0; sl < NDIG; ++sl) bq[sl][ks][h] = wd[sl];
                }
            __syncwarp();   // every lane has read this N tile's inputs
            // exponent fields of the two pivots whose products this lane combines
            const int fx0 = __shfl_sync(0xffffffffu, fm, 8 * tig) - 2096;
            const int fx1 = __shfl_sync(0xffffffffu, fm, 8 * tig + 4) - 2096;
#pragma unroll 1
            for (int mt = t0; mt < t1; ++mt) {
                float acc[NDIG][4];
#pragma unroll
                for (int d = 0; d < NDIG; ++d)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[d][q] = 0.f;
                // consecutive MMAs go to different digit diagonals
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) {
                    if (ks < t0 || ks >= t1) continue;
#pragma unroll
                    for (int sa = 0; sa < NDIG; ++sa) {
                        const uint4 f = Af[((mt * KS + ks) * NDIG + sa) * 32];
                        const uint32_t af[4] = {f.x ^ cflip, f.y ^ cflip, f.z ^ cflip, f.w ^ cflip};
#pragma unroll
                        for (int u = 0; u + sa < NDIG; ++u) mma_f16(acc[sa + u], af, bq[u][ks]);
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int ra = 16 * mt + grp + 8 * (q >> 1), r = ra - r0;
                    const int pc = nt * 8 + 2 * tig + (q & 1);
                    if (r >= 0 && r < n2) {
                        // up to 7 x 16 KS x 2^14 per diagonal: below 2^22 for KS <= 2
                        const long long Y = KS > 2 ? combine_digits_wide(acc, q) : combine_digits(acc, q);
                        out[r * WBS + pc] = scale2(__ll2double_rn(Y), s.fA[ra] + ((q & 1) ? fx1 : fx0));
                    }
                }
            }
        }
        __syncwarp();
    }

    // Forward rows row0 + i (i < N) of A x for this warp's pivots (reads in
    // the warp's buffer); each lane then emits its own pivot's rows.
    template <bool HASB, class Emit>
    static __device__ __forceinline__ void matvec_tc(const Smem &s, int D, int row0, int N, unsigned nm,
                                                     double2 pv, Emit emit)
    {
        const int lane = threadIdx.x & 31;
        double *wb = s.wb + (size_t)(threadIdx.x >> 5) * XS * WBS;
        tc_products<false>(s, D, row0, N, wb, wb);
        for (int i = 0; i < N; ++i) {
            if (!((nm >> i) & 1u)) continue;
            double2 v = make_double2(wb[(2 * i) * WBS + lane], wb[(2 * i + 1) * WBS + lane]);
            if (HASB) v = cadd(v, cmul(s.bs[row0 + i], pv));
            emit(i, v);
        }
    }

    // Partial dL/dA of this warp's 32 pivots on the tensor cores:
    //   P[w][j] = sum_t Y_w(t) conj(X_j(t)),  w, j < N (from row0),
    // Y = scaled output adjoints (warp buffer wy), X = reads (warp buffer wb).
    // Each pivot's reads are scaled by 2^(1022 - e_t) (e_t: largest exponent
    // field of its reads) and its adjoints by the inverse, which leaves every
    // product unchanged; the adjoints then share a power of two per row w
    // over the 32 pivots, so each term is exact relative to the largest
    // product of its row.  Real form with K = (pivot t, re/im) = 64 and two
    // accumulators per output:
    //   A[w][(t,0)] = Yr, A[w][(t,1)] = Yi;
    //   Re P = A [Xr; Xi],  Im P = A [-Xi; Xr]  (column j of each B).
    // Each read is converted once; the digits of (-Xi, Xr) are those of
    // (Xr, Xi) with the halves swapped and the low half negated (a balanced
    // digit negates exactly in fp16).  The result is added to the warp's own
    // slot (single writer).
    //
    // These sums feed no recurrence, so they take NDP = 6 digits (21 digit
    // pairs): a term's error is below 2^-45 of the largest product of its row
    // in the tile, under the rounding of the FP64 additions that follow (about
    // 60 tiles per slot, then the slots), so the gradient is as accurate as
    // an FP64 sum of the same terms.
    static constexpr int NDP = 6;

    static __device__ void tc_partials(const DiagArgs &a, const Smem &s, int circ, int row0, int N)
    {
        constexpr int NT = KS;   // N tiles of 8 columns j (N <= 8 KS)
        const int lane = threadIdx.x & 31, grp = lane >> 2, tig = lane & 3, warp = threadIdx.x >> 5;
        const int D = 2 * a.sh.M, nnt = (N + 7) >> 3, nmt = KS > 2 ? (N + 15) >> 4 : 1;
        const double *wx = s.wb + (size_t)warp * XS * WBS;
        const double *wy = s.wy + (size_t)warp * XS * WBS;
        const int *ef = s.wf + warp * 32;
        const int *gy = s.wg + warp * 32;
        const size_t slot = (size_t)blockIdx.x * (TPB / 32) + warp;
        double *pA = (double *)(a.partA + ((size_t)circ * a.slots + slot) * D * D);
        // rows w of the m16 tile mt (one tile up to 16 rows, two beyond)
#pragma unroll 1
        for (int mt = 0; mt < nmt; ++mt) {
            float ar[NDP][NT][4], ai[NDP][NT][4];
#pragma unroll
            for (int d = 0; d < NDP; ++d)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int q = 0; q < 4; ++q) ar[d][nt][q] = ai[d][nt][q] = 0.f;
            // A rows of this lane: w0 = 16 mt + grp, w1 = w0 + 8
            const int w0 = 16 * mt + grp, w1 = w0 + 8;
            const int g0 = w0 < N ? gy[w0] : 0, g1 = w1 < N ? gy[w1] : 0;
#pragma unroll 1
            for (int ks = 0; ks < 4; ++ks) {
                const int t0 = 8 * ks + tig, t1 = t0 + 4;
                const int e0 = ef[t0], e1 = ef[t1];
                if (!__any_sync(0xffffffffu, e0 != 0 || e1 != 0)) continue;   // 8 pivots without reads
                uint32_t aq[NDP][4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int w = (k & 1) ? w1 : w0, t = (k & 2) ? t1 : t0, e = (k & 2) ? e1 : e0;
                    const int g = (k & 1) ? g1 : g0;
                    double yr = 0.0, yi = 0.0;
                    if (w < N && g != 0 && e != 0) {
                        yr = wy[(2 * w) * WBS + t];
                        yi = wy[(2 * w + 1) * WBS + t];
                    }
                    const int fm = g - e + 1022;
                    uint32_t wd[NDP];
                    digit_words<NDP>(to_fixed_rel<NDP>(yr, fm), to_fixed_rel<NDP>(yi, fm), wd);
#pragma unroll
                    for (int sl = 0; sl < NDP; ++sl) aq[sl][k] = wd[sl];
                }
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    if (nt >= nnt) continue;
                    const int j = 8 * nt + grp;
                    uint32_t bq[NDP][2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int t = h ? t1 : t0, e = h ? e1 : e0;
                        double xr = 0.0, xi = 0.0;
                        if (j < N) {
                            xr = wx[(2 * j) * WBS + t];
                            xi = wx[(2 * j + 1) * WBS + t];
                        }
                        uint32_t wd[NDP];
                        digit_words<NDP>(to_fixed<NDP>(xr, e), to_fixed<NDP>(xi, e), wd);
#pragma unroll
                        for (int sl = 0; sl < NDP; ++sl) bq[sl][h] = wd[sl];
                    }
#pragma unroll
                    for (int u = 0; u < NDP; ++u) {
                        const uint32_t bi[2] = {__byte_perm(bq[u][0], 0u, 0x1032) ^ 0x8000u,
                                                __byte_perm(bq[u][1], 0u, 0x1032) ^ 0x8000u};
#pragma unroll
                        for (int sa = 0; sa + u < NDP; ++sa) {
                            mma_f16(ar[sa + u][nt], aq[sa], bq[u]);
                            mma_f16(ai[sa + u][nt], aq[sa], bi);
                        }
                    }
                }
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                if (nt >= nnt) continue;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int w = (q >> 1) ? w1 : w0, j = 8 * nt + 2 * tig + (q & 1);
                    const int g = (q >> 1) ? g1 : g0;
                    if (w < N && j < N && g >= 26) {
                        float a6[NDP][4];
#pragma unroll
                        for (int d = 0; d < NDP; ++d) a6[d][0] = ar[d][nt][q];
                        const long long Yr = combine_digits_wide<NDP>(a6, 0);
#pragma unroll
                        for (int d = 0; d < NDP; ++d) a6[d][0] = ai[d][nt][q];
                        const long long Yi = combine_digits_wide<NDP>(a6, 0);
                        double *dst = pA + 2 * ((size_t)(row0 + w) * D + row0 + j);
                        // reductions without return: the warp does not wait for
                        // the old values.  The slot has one warp as its only
                        // writer and its updates are ordered by the warp's
                        // barriers between tiles, so the sum order is fixed.
                        // Scale: Y carries the product of the two fixed points
                        // over 2^(8 NDP), i.e. 2^(1074 - 8 (7 - NDP) - g).
                        atomicAdd(dst, scale2(__ll2double_rn(Yr), g - 1074 + 8 * (NDIG - NDP)));
                        atomicAdd(dst + 1, scale2(__ll2double_rn(Yi), g - 1074 + 8 * (NDIG - NDP)));
                    }
                }
            }
        }
    }

    template <bool HASB, class Emit>
    static __device__ __forceinline__ void matvec_any(const Smem &s, int D, int row0, int N, unsigned vm,
                                                      unsigned nm, double2 pv, Emit emit)
    {
        if constexpr (TC) matvec_tc<HASB>(s, D, row0, N, nm, pv, emit);
        else matvec<HASB>(s, D, row0, N, vm, nm, pv, emit);
    }

    // Columns row0 + j of A^H y for this thread's scaled output adjoints:
    //   Re = sum Ar ys + sum (Ai - Ar) yi,  Im = sum Ar ys - sum (Ar + Ai) yr.
    template <class Emit>
    static __device__ __forceinline__ void matvec_adj(const Smem &s, int D, int row0, int N,
                                                      unsigned vm, unsigned nm, Emit emit)
    {
        const int t = threadIdx.x, DD = D * D;
        const double *Ar = s.A3 + (size_t)row0 * D + row0;
        const double *Ap = Ar + DD, *Am = Ar + 2 * DD;
        for (int j0 = 0; j0 < N; j0 += CH) {
            if (((vm >> j0) & ((1u << CH) - 1u)) == 0) continue;
            double p1[CH], q2[CH], q3[CH];
#pragma unroll
            for (int jj = 0; jj < CH; ++jj) p1[jj] = q2[jj] = q3[jj] = 0.0;
            for (int i = 0; i < N; ++i) {
                if (!((nm >> i) & 1u)) continue;
                const double yr = s.Y3[(size_t)i * RS + t];
                const double yi = s.Y3[(size_t)(D + i) * RS + t];
                const double ys = s.Y3[(size_t)(2 * D + i) * RS + t];
#pragma unroll
                for (int jj = 0; jj < CH; ++jj)
                    if (j0 + jj < N && ((vm >> (j0 + jj)) & 1u)) {
                        const size_t o = (size_t)i * D + j0 + jj;
                        p1[jj] = fma(Ar[o], ys, p1[jj]);
                        q2[jj] = fma(Am[o], yi, q2[jj]);
                        q3[jj] = fma(Ap[o], yr, q3[jj]);
                    }
            }
#pragma unroll
            for (int jj = 0; jj < CH; ++jj) {
                const int j = j0 + jj;
                if (j < N && ((vm >> j) & 1u)) emit(j, make_double2(p1[jj] + q2[jj], p1[jj] - q3[jj]));
            }
        }
    }

    // ------------------------------------------------------------ early stop
    // A pivot tile of level `lev` runs while the probabilities with at most
    // `lev` photons sum to less than 1 - eps.  The per-photon-number sums are
    // final once the level below has passed its barrier, and fixed point
    // keeps them independent of the order of the additions, so every block
    // takes the same decision.
    static __device__ __forceinline__ unsigned long long fixed_prob(double p)
    {
        return p > 0.0 ? (unsigned long long)(p * 0x1p56) : 0ull;
    }

    static __device__ __forceinline__ bool pivots_run(const DiagArgs &a, int circ, int lev)
    {
        if (!a.early) return lev < a.sh.L;
        if (lev >= a.sh.L) return false;
        const unsigned long long *l = a.lvl + (size_t)circ * (a.sh.L + 2);
        unsigned long long cum = 0;
        for (int n = 0; n <= lev; ++n) cum += __ldcg(l + n);
        return cum < a.thr;
    }

    // The same, the sum split over the 32 lanes of a warp whose lanes all ask
    // for the same (circ, lev) (integer sums: the same decision, in two loads
    // per lane instead of lev + 1).
    static __device__ __forceinline__ bool pivots_run_w(const DiagArgs &a, int circ, int lev)
    {
        if (!a.early) return lev < a.sh.L;
        if (lev >= a.sh.L) return false;
        const unsigned long long *l = a.lvl + (size_t)circ * (a.sh.L + 2);
        unsigned long long cum = 0;
        for (int n = threadIdx.x & 31; n <= lev; n += 32) cum += __ldcg(l + n);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cum += __shfl_xor_sync(0xffffffffu, cum, o);
        return cum < a.thr;
    }

    // Block-wide sum of v added to lvl[circ][n] (thread 0).
    static __device__ void add_level_prob(const DiagArgs &a, int circ, int n, double v)
    {
        __shared__ double s_part[32];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
            atomicAdd(a.lvl + (size_t)circ * (a.sh.L + 2) + n, fixed_prob(t));
        }
        __syncthreads();
    }

    // fn(tile) over the tiles [0, nt) of a phase: block b first takes tile b,
    // then the next free tile of the phase's counter (requested while the
    // current tile runs), so blocks that drew light tiles take more of them
    // and a phase ends at most about one tile after its mean.
    template <class Fn>
    static __device__ void run_tiles(int *ctr, int nt, Fn fn)
    {
        __shared__ int s_next[2];
        int tile = blockIdx.x, k = 0;
        while (tile < nt) {
            int nxt = 0;
            if (threadIdx.x == 0) nxt = atomicAdd(ctr, 1);
            fn(tile);
            if (threadIdx.x == 0) s_next[k & 1] = (int)gridDim.x + nxt;
            __syncthreads();
            tile = s_next[k & 1];
            ++k;
        }
    }

    // Circuit-per-block mode: the next circuit for this block (all threads
    // get the same value), from the counter ctr, or a.B when none is left.
    static __device__ int next_circuit(int *ctr)
    {
        __shared__ int s_c;
        __syncthreads();
        if (threadIdx.x == 0) s_c = atomicAdd(ctr, 1);
        __syncthreads();
        return s_c;
    }

    // The tiles of circuit c in a phase of nt tiles (circuit-major numbering),
    // one after the other in this block.
    template <class Fn>
    static __device__ void circuit_tiles(const DiagArgs &a, int c, int nt, Fn fn)
    {
        const int per = nt / a.B;
        for (int j = 0; j < per; ++j) {
            fn(c * per + j);
            __syncthreads();
        }
    }

    // Tiles of a phase are numbered circuit-major: circuit c, then segment k
    // (anchor K for AP; one segment for DP), then ceil(count / TPB) tiles;
    // tiles[k] = prefix over k within one circuit, tiles[nseg] = tiles per
    // circuit.  Blocks take them in counter order, so at any moment the grid
    // works on one or two circuits and the reads that pivots of different
    // anchors share stay in L2.  kind: 0 = AP, 1 = DP.
    static __device__ int phase_tiles(const DiagArgs &a, Smem &s, int kind, int lev)
    {
        const DiagShape &sh = a.sh;
        __syncthreads();
        if (threadIdx.x < 32) phase_offsets(sh, s, lev);
        if (threadIdx.x == 0) {
            int acc = 0;
            const int nseg = (kind == 0) ? sh.M : 1;
            for (int k = 0; k < nseg; ++k) {
                const unsigned cnt = level_count(sh, s, kind == 0 ? k : 0, 1, lev);
                s.tiles[k] = acc;
                s.tiles[sh.M + 2 + k] = (int)cnt;
                acc += (int)((cnt + TPB - 1) / TPB);
            }
            s.tiles[nseg] = acc;
        }
        __syncthreads();
        return a.B * s.tiles[(kind == 0) ? sh.M : 1];
    }

    static __device__ TileId decode_tile(const DiagArgs &a, const Smem &s, int kind, int lev, int tile)
    {
        const DiagShape &sh = a.sh;
        TileId t;
        const int nseg = (kind == 0) ? sh.M : 1;
        const int Tc = s.tiles[nseg];
        t.circ = tile / Tc;
        const int r = tile - t.circ * Tc;
        int k = 0;
        while (k + 1 < nseg && r >= s.tiles[k + 1]) ++k;
        t.seg = k;
        t.rank0 = (unsigned)(r - s.tiles[k]) * TPB;
        t.count = (unsigned)s.tiles[sh.M + 2 + k];   // the segment's pivots, from phase_tiles
        return t;
    }

    // ------------------------------------------------------- per-pivot geometry

    // The circuit-independent part of an AP(K) pivot's geometry (pivot e of
    // level `lev`, rank r in family K): the ranks of e - 1_m (m > K) within
    // their level, the offset of T2(K)[e - 1_K] within level lev - 1 of family
    // K and of DIAG[e + 1_K] within level lev + 1 of the DIAG family.
    static constexpr int kRel = KS > 2 ? FK_MAXM - 1 : 7;   // modes after K an AP pivot reads
    struct ApRel {
        int idx[kRel];    // idx[m - K - 1] for m = K+1..M-1
        int rt2, wdiag;
    };

    static __device__ __forceinline__ ApRel ap_rel(const DiagShape &sh, const Dig &e, int K, const Smem &s,
                                                   int lev, int64_t r)
    {
        ApRel q;
        const int eK = e(K);
        int t = lev;
        int64_t cum = Pf(s, K, t, eK);
        q.rt2 = eK >= 1 ? (int)(Pf(s, K, t - 1, eK - 1) + (r - cum)) : 0;
        q.wdiag = (int)(Pf(s, K, lev + 1, eK + 1) + (r - cum));
        int64_t pre = Pf(s, K, t - 1, eK);
        t -= eK;
#pragma unroll
        for (int i = 0; i < kRel; ++i) {
            const int m = K + 1 + i;
            q.idx[i] = 0;
            if (m >= sh.M) continue;
            const int em = e(m);
            cum += Pf(s, m, t, em);
            q.idx[i] = em >= 1 ? (int)(pre + Pf(s, m, t - 1, em - 1) + (r - cum)) : 0;
            pre += Pf(s, m, t - 1, em);
            t -= em;
        }
        return q;
    }

    // AP(K) pivot e of level `lev` with rank r in family K (M <= 4 KS):
    // addresses of its reads and writes from its relative geometry; the ranks
    // of e - 1_m (m > K) go to s.idx[m][thread].  ap_geom below is the same
    // computation for any M.
    template <bool STORE_IDX = true>
    static __device__ __forceinline__ ApGeom ap_assemble(const DiagShape &sh, const Dig &e, int K, Smem &s,
                                                         int lev, int64_t r, const ApRel &q)
    {
        ApGeom g;
        const int eK = e(K);
        g.r = r;
        g.rd = cum_full(s, lev) + r;
        g.lk0 = s.cum0[K];
        g.lkm = s.cum1[K];
        g.wt2 = sh.lm_t2[K] + g.lk0 + r;
        g.fp = sh.has_b ? box_t1(sh, K, sh.lm_t1[K] + 2 * (s.cum0[0] + r) + 1) : 0;
        int64_t pout = sh.stride[K];
        for (int i = K; i < sh.M; ++i) pout += (int64_t)e(i) * sh.stride[i];
        g.pout = pout;
        g.rt2 = eK >= 1 ? sh.lm_t2[K] + g.lkm + q.rt2 : 0;
        g.wdiag = cum_full(s, lev + 1) + q.wdiag;
        g.vmask = 1u | (eK >= 1 ? 2u : 0u);
        g.nmask = 2u | (eK <= sh.C[K] - 3 ? 1u : 0u);
#pragma unroll
        for (int i = 0; i < kRel; ++i) {
            const int m = K + 1 + i;
            if (m >= sh.M) continue;
            const int em = e(m);
            if (STORE_IDX) s.idx[m * TPB + threadIdx.x] = q.idx[i];
            if (em >= 1) g.vmask |= 3u << (2 * (m - K));
            if (em <= sh.C[m] - 2) g.nmask |= 3u << (2 * (m - K));
        }
        return g;
    }

    // AP(K) pivot e of level `lev` with rank r in family K: addresses of its
    // reads and writes; the ranks of e - 1_m (m > K) go to s.idx[m][thread].
    static __device__ __forceinline__ ApGeom ap_geom(const DiagShape &sh, const Dig &e, int K, Smem &s,
                                                     int lev, int64_t r)
    {
        ApGeom g;
        const int eK = e(K);
        g.r = r;
        g.rd = cum_full(s, lev) + r;
        g.lk0 = s.cum0[K];
        g.lkm = s.cum1[K];
        g.wt2 = sh.lm_t2[K] + g.lk0 + r;
        g.fp = sh.has_b ? box_t1(sh, K, sh.lm_t1[K] + 2 * (s.cum0[0] + r) + 1) : 0;
        int64_t pout = sh.stride[K];
        for (int i = K; i < sh.M; ++i) pout += (int64_t)e(i) * sh.stride[i];
        g.pout = pout;
        int t = lev;
        int64_t cum = Pf(s, K, t, eK);
        g.rt2 = eK >= 1 ? sh.lm_t2[K] + g.lkm + Pf(s, K, t - 1, eK - 1) + (r - cum) : 0;
        g.wdiag = cum_full(s, lev + 1) + Pf(s, K, lev + 1, eK + 1) + (r - cum);
        int64_t pre = Pf(s, K, t - 1, eK);
        t -= eK;
        g.vmask = 1u | (eK >= 1 ? 2u : 0u);
        g.nmask = 2u | (eK <= sh.C[K] - 3 ? 1u : 0u);
        for (int m = K + 1; m < sh.M; ++m) {
            const int em = e(m);
            cum += Pf(s, m, t, em);
            s.idx[m * TPB + threadIdx.x] = em >= 1 ? (int)(pre + Pf(s, m, t - 1, em - 1) + (r - cum)) : 0;
            pre += Pf(s, m, t - 1, em);
            t -= em;
            if (em >= 1) g.vmask |= 3u << (2 * (m - K));
            if (em <= sh.C[m] - 2) g.nmask |= 3u << (2 * (m - K));
        }
        return g;
    }

    // Pivot e and its geometry: from the launch's shared table when there is
    // one (same values as computing them), else computed.
    static __device__ __forceinline__ ApGeom ap_pivot(const DiagArgs &a, Smem &s, int K, int lev, unsigned r,
                                                      Dig &e)
    {
        const DiagShape &sh = a.sh;
        if (a.geo == nullptr) {
            e = unrank(sh, s, K, 1, lev, r);
            return ap_geom(sh, e, K, s, lev, (int64_t)r);
        }
        const int4 *rec = (const int4 *)(a.geo + (size_t)box_ap(sh, K, sh.off_ap[K] + s.cum0[K] + r) * kGeoInts);
        const int4 w0 = __ldcg(rec), w1 = __ldcg(rec + 1), w2 = __ldcg(rec + 2);
        e.lo = (uint64_t)(unsigned)w0.x | ((uint64_t)(unsigned)w0.y << 32);
        e.hi = 0;
        ApRel q;
        q.idx[0] = w0.z; q.idx[1] = w0.w;
        q.idx[2] = w1.x; q.idx[3] = w1.y; q.idx[4] = w1.z; q.idx[5] = w1.w;
        q.idx[6] = w2.x;
        q.rt2 = w2.y;
        q.wdiag = w2.z;
        return ap_assemble(sh, e, K, s, lev, (int64_t)r, q);
    }

    // The same from the table (M <= 8), the ranks of the reads left in q.
    static __device__ __forceinline__ ApGeom ap_pivot_regs(const DiagArgs &a, Smem &s, int K, int lev,
                                                           unsigned r, Dig &e, ApRel &q)
    {
        const DiagShape &sh = a.sh;
        if (a.geo == nullptr) {
            e = unrank(sh, s, K, 1, lev, r);
            q = ap_rel(sh, e, K, s, lev, (int64_t)r);
            return ap_assemble<false>(sh, e, K, s, lev, (int64_t)r, q);
        }
        const int4 *rec = (const int4 *)(a.geo + (size_t)box_ap(sh, K, sh.off_ap[K] + s.cum0[K] + r) * kGeoInts);
        const int4 w0 = __ldcg(rec), w1 = __ldcg(rec + 1), w2 = __ldcg(rec + 2);
        e.lo = (uint64_t)(unsigned)w0.x | ((uint64_t)(unsigned)w0.y << 32);
        e.hi = 0;
        q.idx[0] = w0.z; q.idx[1] = w0.w;
        q.idx[2] = w1.x; q.idx[3] = w1.y; q.idx[4] = w1.z; q.idx[5] = w1.w;
        q.idx[6] = w2.x;
        q.rt2 = w2.y;
        q.wdiag = w2.z;
        return ap_assemble<false>(sh, e, K, s, lev, (int64_t)r, q);
    }

    // The table: every AP pivot of the pivot levels.  The pivots (K, level, r)
    // in that order are numbered densely and handed out grid-stride, so every
    // thread gets the same share whatever the level sizes; a thread's numbers
    // only grow, so it advances its (K, level) position instead of searching.
    static __device__ void build_geometry(const DiagArgs &a, const Smem &s)
    {
        const DiagShape &sh = a.sh;
        const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
        int K = 0, lev = 0;
        int64_t kbase = 0, lbase = 0;   // dense numbers of the first pivot of family K, of (K, lev)
        int64_t cnt = Pf(s, 0, 0, sh.C[0] - 1);
        for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;; t += gsz) {
            while (t >= lbase + cnt) {
                lbase += cnt;
                if (++lev >= sh.L) {
                    if (++K >= sh.M) return;
                    lev = 0;
                    kbase = lbase;
                }
                cnt = Pf(s, K, lev, sh.C[K] - 1);
            }
            const int64_t r = t - lbase;
            const Dig e = unrank(sh, s, K, 1, lev, (unsigned)r);
            const ApRel q = ap_rel(sh, e, K, s, lev, r);
            int4 *rec = (int4 *)(a.geo + (size_t)box_ap(sh, K, sh.off_ap[K] + (lbase - kbase) + r) * kGeoInts);
            rec[0] = make_int4((int)(unsigned)e.lo, (int)(unsigned)(e.lo >> 32), q.idx[0], q.idx[1]);
            rec[1] = make_int4(q.idx[2], q.idx[3], q.idx[4], q.idx[5]);
            rec[2] = make_int4(q.idx[6], q.rt2, q.wdiag, 0);
        }
    }

    // P1010/P1001(K,m) pair base (interleaved: P1010 even, P1001 odd).
    static __device__ __forceinline__ int64_t pair_base(const DiagShape &sh, int K, int m)
    {
        return sh.lm_p[K] + 2 * (int64_t)(m - K - 1) * sh.fam[K];
    }

    // Storage boxes of one circuit's amplitude array for the debug checks:
    // DIAG [0, n_diag); T2(K) and the P pairs (K, m) in family K; the T1
    // pair of mode q in family 0.
    static __device__ __forceinline__ int64_t box_diag(const DiagShape &sh, int64_t i)
    {
        return FK_BOX(i, 0, sh.n_diag);
    }
    static __device__ __forceinline__ int64_t box_t2(const DiagShape &sh, int K, int64_t i)
    {
        return FK_BOX(i, sh.lm_t2[K], sh.lm_t2[K] + sh.fam[K]);
    }
    static __device__ __forceinline__ int64_t box_pair(const DiagShape &sh, int K, int m, int64_t i)
    {
        return FK_BOX(i, pair_base(sh, K, m), pair_base(sh, K, m) + 2 * sh.fam[K]);
    }
    static __device__ __forceinline__ int64_t box_t1(const DiagShape &sh, int q, int64_t i)
    {
        return FK_BOX(i, sh.lm_t1[q], sh.lm_t1[q] + 2 * sh.fam[0]);
    }
    // AP(K) pivots: VJP scratch entries and geometry records
    static __device__ __forceinline__ int64_t box_ap(const DiagShape &sh, int K, int64_t i)
    {
        return FK_BOX(i, sh.off_ap[K], sh.off_ap[K] + sh.fam[K]);
    }

    // Address (within the circuit's amplitude array) of AP read column j.
    static __device__ __forceinline__ int64_t ap_read_addr(const DiagShape &sh, const ApGeom &g, int K,
                                                    int j, const Smem &s)
    {
        if (j == 0) return box_diag(sh, g.rd);
        if (j == 1) return box_t2(sh, K, g.rt2);
        const int m = K + j / 2;
        const int64_t rk = s.idx[m * TPB + threadIdx.x];
        return box_pair(sh, K, m, pair_base(sh, K, m) + 2 * (g.lkm + rk) + ((j & 1) ? 0 : 1));
    }

    // The same with the ranks of e - 1_m in registers (q.idx[m - K - 1]); j is
    // a compile-time index in the unrolled gather.
    static __device__ __forceinline__ int64_t ap_read_addr_q(const DiagShape &sh, const ApGeom &g, int K,
                                                             int j, const ApRel &q)
    {
        if (j == 0) return box_diag(sh, g.rd);
        if (j == 1) return box_t2(sh, K, g.rt2);
        const int m = K + j / 2;
        return box_pair(sh, K, m, pair_base(sh, K, m) + 2 * (g.lkm + q.idx[j / 2 - 1]) + ((j & 1) ? 0 : 1));
    }

    // Address of AP write row i and its scale index P_w + 1.
    static __device__ __forceinline__ int64_t ap_write_addr(const DiagShape &sh, const ApGeom &g,
                                                     const Dig &e, int K, int i, const Smem &s,
                                                     int *den)
    {
        if (i == 0) { *den = e(K) + 2; return box_t2(sh, K, g.wt2); }
        if (i == 1) { *den = e(K) + 1; return box_diag(sh, g.wdiag); }
        const int m = K + i / 2;
        *den = e(m) + 1;
        return box_pair(sh, K, m, pair_base(sh, K, m) + 2 * (g.lk0 + g.r) + (i & 1));
    }

    // DP pivot d of level `lev` with rank r in family 0; ranks of d - 1_q go
    // to s.idx[q][thread].
    static __device__ __forceinline__ DpGeom dp_geom(const DiagShape &sh, const Dig &d, Smem &s, int lev,
                                                     int64_t r)
    {
        DpGeom g;
        g.r = r;
        g.rdiag = box_diag(sh, cum_full(s, lev) + r);
        g.l00 = s.cum0[0];
        g.l0m = s.cum1[0];
        g.vmask = 0;
        g.nmask = 0;
        int t = lev;
        int64_t cum = 0, pre = 0;
        for (int q = 0; q < sh.M; ++q) {
            const int dq = d(q);
            cum += Pf(s, q, t, dq);
            s.idx[q * TPB + threadIdx.x] = dq >= 1 ? (int)(pre + Pf(s, q, t - 1, dq - 1) + (r - cum)) : 0;
            pre += Pf(s, q, t - 1, dq);
            t -= dq;
            if (dq >= 1) g.vmask |= 3u << (2 * q);
            if (q == 0) {
                g.nmask |= 1u;
                if (dq <= sh.C[0] - 3) g.nmask |= 2u;
            } else if (dq <= sh.C[q] - 2) {
                g.nmask |= 3u << (2 * q);
            }
        }
        return g;
    }

    // T1 pair of mode q (interleaved: T1B even, T1K odd).
    static __device__ __forceinline__ int64_t dp_read_addr(const DiagShape &sh, const DpGeom &g, int j,
                                                    const Smem &s)
    {
        const int q = j / 2;
        return box_t1(sh, q, sh.lm_t1[q] + 2 * (g.l0m + s.idx[q * TPB + threadIdx.x]) + (j & 1));
    }

    static __device__ __forceinline__ int64_t dp_write_addr(const DiagShape &sh, const DpGeom &g,
                                                     const Dig &d, int i, const Smem &s, int *den)
    {
        const int q = i / 2;
        *den = d(q) + 1;
        return box_t1(sh, q, sh.lm_t1[q] + 2 * (g.l00 + g.r) + ((i & 1) ? 0 : 1));
    }

    // ---------------------------------------------------------------- prologue
    // A_s = (A + A^T)/2 restricted to kept modes, b restricted, vacuum seeds.
    static __device__ void prologue(const DiagArgs &a, Smem &s, bool seed, bool clear_ctr = true)
    {
        const DiagShape &sh = a.sh;
        const int D = 2 * sh.M, Do = sh.D_orig;
        const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
        int nz = 0;
        for (int64_t e = gtid; e < (int64_t)a.B * D * D; e += gsz) {
            const int c = (int)(e / (D * D));
            const int w = (int)((e / D) % D), l = (int)(e % D);
            const int ow = 2 * sh.mode_map[w / 2] + (w & 1), ol = 2 * sh.mode_map[l / 2] + (l & 1);
            const double2 x = a.A[cix(a, c) * Do * Do + (size_t)ow * Do + ol];
            const double2 y = a.A[cix(a, c) * Do * Do + (size_t)ol * Do + ow];
            a.As[e] = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y + y.y));
        }
        for (int64_t e = gtid; e < (int64_t)a.B * D; e += gsz) {
            const int c = (int)(e / D), w = (int)(e % D);
            const int ow = 2 * sh.mode_map[w / 2] + (w & 1);
            const double2 v = a.b[cix(a, c) * Do + ow];
            a.bs[e] = v;
            if (v.x != 0.0 || v.y != 0.0) nz = 1;
        }
        if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(&a.ctl->has_b, 1);
        if (clear_ctr)
            for (int64_t e = gtid; e < 4 * (int64_t)(sh.L + 1); e += gsz) a.ctr[e] = 0;
        if constexpr (TC) build_digits(a, s);
        if (a.geo != nullptr &&
            !(a.geo_reuse && *(volatile const unsigned long long *)&a.ctl->geo_key == a.geo_key))
            build_geometry(a, s);
        if (seed) {
            for (int64_t c = gtid; c < a.B; c += gsz) {
                const double2 v = a.c[cix(a, (int)c)];
                if (a.early) a.lvl[(size_t)c * (sh.L + 2)] = fixed_prob(v.x);
                a.F[(size_t)c * sh.circ_alloc] = v;
                a.probs[oix(a, (int)c)] = v;
            }
        }
    }

    // ------------------------------------------------------------- forward AP
    template <bool HASB, bool EARLY>
    static __device__ void ap_forward_tile(const DiagArgs &a, Smem &s, const TileId &tl, int K, int lev)
    {
        const DiagShape &sh = a.sh;
        const int t = threadIdx.x, D = 2 * sh.M, N = 2 * (sh.M - K);
        load_circuit(a, s, tl.circ);
        double2 *F = a.F + (size_t)tl.circ * sh.circ_alloc;
        const unsigned r = tl.rank0 + t;
        const bool act = r < tl.count;
        Dig e;
        ApGeom g{};
        double2 FP = make_double2(0, 0);
        double fe = 1.0, psum = 0.0;
        if (act) {
            if constexpr (TC) {
                ApRel q;
                g = ap_pivot_regs(a, s, K, lev, r, e, q);
                gather(
                    N,
                    [&](int j) {
                        return ((g.vmask >> j) & 1u) ? __ldcg(F + ap_read_addr_q(sh, g, K, j, q))
                                                     : make_double2(0, 0);
                    },
                    [&](int j, double2 v) { store_read(s, D, j, t, v, false); });
            } else {
                g = ap_pivot(a, s, K, lev, r, e);
                gather(
                    N,
                    [&](int j) {
                        return ((g.vmask >> j) & 1u) ? __ldcg(F + ap_read_addr(sh, g, K, j, s))
                                                     : make_double2(0, 0);
                    },
                    [&](int j, double2 v) { store_read(s, D, j, t, v, false); });
            }
            if (HASB) FP = __ldcg(F + g.fp);
            for (int i = K; i < sh.M; ++i) fe *= s.fact[e(i)];
        } else {
            for (int j = 0; j < N; ++j) store_read(s, D, j, t, make_double2(0, 0), false);
        }
        const unsigned vm = __reduce_or_sync(0xffffffffu, g.vmask);
        const unsigned nm = __reduce_or_sync(0xffffffffu, g.nmask);
        matvec_any<HASB>(s, D, 2 * K, N, vm, nm, FP, [&](int i, double2 acc) {
            if (!act || !((g.nmask >> i) & 1u)) return;
            int den;
            const int64_t addr = ap_write_addr(sh, g, e, K, i, s, &den);
            const double2 v = rscale(acc, s.inv[den]);
            F[addr] = v;
            if (i == 1) {
                const double2 p = rscale(v, fe * (double)(e(K) + 1));
                a.probs[oix(a, tl.circ) + box_diag(sh, sh.global ? g.wdiag : g.pout)] = p;
                if (EARLY) psum += p.x;
            }
        });
        if (EARLY) add_level_prob(a, tl.circ, lev + 1, psum);
    }

    // ------------------------------------------------------------- forward DP
    static __device__ void dp_forward_tile(const DiagArgs &a, Smem &s, const TileId &tl, int lev)
    {
        const DiagShape &sh = a.sh;
        const int t = threadIdx.x, D = 2 * sh.M, N = D;
        load_circuit(a, s, tl.circ);
        double2 *F = a.F + (size_t)tl.circ * sh.circ_alloc;
        const unsigned r = tl.rank0 + t;
        const bool act = r < tl.count;
        Dig d;
        DpGeom g{};
        double2 FP = make_double2(0, 0);
        if (act) {
            d = unrank(sh, s, 0, 1, lev, r);
            g = dp_geom(sh, d, s, lev, (int64_t)r);
            gather(
                N,
                [&](int j) {
                    return ((g.vmask >> j) & 1u) ? __ldcg(F + dp_read_addr(sh, g, j, s)) : make_double2(0, 0);
                },
                [&](int j, double2 v) { store_read(s, D, j, t, v, false); });
            FP = __ldcg(F + g.rdiag);
        } else {
            for (int j = 0; j < N; ++j) store_read(s, D, j, t, make_double2(0, 0), false);
        }
        const unsigned vm = __reduce_or_sync(0xffffffffu, g.vmask);
        const unsigned nm = __reduce_or_sync(0xffffffffu, g.nmask);
        matvec_any<true>(s, D, 0, N, vm, nm, FP, [&](int i, double2 acc) {
            if (!act || !((g.nmask >> i) & 1u)) return;
            int den;
            const int64_t addr = dp_write_addr(sh, g, d, i, s, &den);
            F[addr] = rscale(acc, s.inv[den]);
        });
    }

    // ------------------------------------------------- reverse-walk reductions
    // Accumulate sum_t Y[w][t] conj(R[j][t]) into the block's partial dL/dA and
    // sum_t Y[w][t] conj(FP[t]) into its partial dL/db (rows/cols from 2*k0).
    // With planes y = (yr, yi, yr + yi) and R = (Rr, Rr - Ri, Rr + Ri):
    //   Re = sum (yr + yi) Rr - sum yi (Rr - Ri),
    //   Im = sum (yr + yi) Rr - sum yr (Rr + Ri)   (three DFMA per term).
    static __device__ void reduce_partials(const DiagArgs &a, Smem &s, int circ, int k0, int N,
                                           bool hasb, unsigned wm, unsigned jm)
    {
        __shared__ unsigned s_m[2];
        if (threadIdx.x == 0) s_m[0] = s_m[1] = 0u;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) {   // wm, jm arrive OR-reduced over each warp
            atomicOr(&s_m[0], wm);
            atomicOr(&s_m[1], jm);
        }
        __syncthreads();
        wm = s_m[0];
        jm = s_m[1];
        const int D = 2 * a.sh.M;
        double2 *pA = a.partA + ((size_t)circ * a.slots + blockIdx.x) * D * D;
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
            const int w = e / N, j = e % N;
            if (!((wm >> w) & 1u) || !((jm >> j) & 1u)) continue;
            const double *ys = s.Y3 + (size_t)(2 * D + w) * RS, *yi = s.Y3 + (size_t)(D + w) * RS;
            const double *yr = s.Y3 + (size_t)w * RS;
            const double *rr = s.R3 + (size_t)j * RS, *rd = s.R3 + (size_t)(D + j) * RS;
            const double *rp = s.R3 + (size_t)(2 * D + j) * RS;
            double P = 0.0, Q = 0.0, T = 0.0;
            for (int tt = 0; tt < TPB; ++tt) {
                P = fma(ys[tt], rr[tt], P);
                Q = fma(yi[tt], rd[tt], Q);
                T = fma(yr[tt], rp[tt], T);
            }
            double2 &dst = pA[(size_t)(2 * k0 + w) * D + 2 * k0 + j];
            dst = cadd(dst, make_double2(P - Q, P - T));
        }
        if (hasb) {
            double2 *pb = a.partb + ((size_t)circ * a.slots + blockIdx.x) * D;
            for (int w = threadIdx.x; w < N; w += blockDim.x) {
                if (!((wm >> w) & 1u)) continue;
                double2 acc = make_double2(0, 0);
                for (int tt = 0; tt < TPB; ++tt) acc = cfma_conj(s.FP[tt], load_adj(s, D, w, tt), acc);
                pb[2 * k0 + w] = cadd(pb[2 * k0 + w], acc);
            }
        }
        __syncthreads();
    }

    // Adjoint of the DIAG value x = e + 1_K (level lev + 1) written by the
    // AP(K) pivot e of level lev: the upstream seed of p_x (times the
    // factorials f_x = prod_i x_i!), the read adjoints that the AP(k) pivots
    // with base x (k <= K, the first nonzero mode of x) left in scratch when
    // level lev + 1 ran, and, with b != 0, what the DP pivots of level lev + 1
    // added in Fbar.  x has this pivot as its only writer, so its adjoint is
    // complete here and is formed by its one reader instead of in a pass over
    // the DIAG values.
    template <bool HASB>
    static __device__ __forceinline__ double2 diag_adjoint(const DiagArgs &a, const Smem &s, int circ, int K,
                                                           int lev, const ApGeom &g, const Dig &e, bool up)
    {
        const DiagShape &sh = a.sh;
        double fe = 1.0;
        for (int i = K; i < sh.M; ++i) fe *= s.fact[e(i)];
        const int xK = e(K) + 1;
        double2 acc = rscale(a.gprobs[oix(a, circ) + box_diag(sh, sh.global ? g.wdiag : g.pout)],
                             fe * (double)xK);
        if (up) {   // level lev + 1 ran: its AP pivots left the scratch slots
            const double2 *sc = a.scratch + (size_t)circ * sh.n_ap;
            const int64_t rx = g.wdiag - cum_full(s, lev + 1);
            for (int k = 0; k <= K; ++k)
                if (k < K || xK <= sh.C[K] - 2) acc = cadd(acc, __ldcg(sc + box_ap(sh, k, sh.off_ap[k] + s.cum2[k] + rx)));
        }
        if (HASB) acc = cadd(acc, __ldcg(a.Fbar + (size_t)circ * sh.circ_alloc + g.wdiag));
        return acc;
    }

    // Adjoint of the vacuum (dL/dc): its seed, the read adjoints of the AP(k)
    // pivots of level 0 and, with b != 0, the DP contribution in Fbar.
    static __device__ double2 vacuum_adjoint(const DiagArgs &a, int circ, bool hb)
    {
        const DiagShape &sh = a.sh;
        double2 acc = a.gprobs[oix(a, circ)];
        if (pivots_run(a, circ, 0))
            for (int k = 0; k < sh.M; ++k) acc = cadd(acc, __ldcg(a.scratch + (size_t)circ * sh.n_ap + sh.off_ap[k]));
        if (hb) acc = cadd(acc, __ldcg(a.Fbar + (size_t)circ * sh.circ_alloc));
        return acc;
    }

    // --------------------------------------------------------- reverse AP
    template <bool HASB>
    static __device__ void ap_reverse_tile(const DiagArgs &a, Smem &s, const TileId &tl, int K, int lev)
    {
        const DiagShape &sh = a.sh;
        const int t = threadIdx.x, D = 2 * sh.M, N = 2 * (sh.M - K);
        load_circuit(a, s, tl.circ);
        const double2 *F = a.F + (size_t)tl.circ * sh.circ_alloc;
        double2 *Fb = a.Fbar + (size_t)tl.circ * sh.circ_alloc;
        const unsigned r = tl.rank0 + t;
        const bool act = r < tl.count;
        const bool up = pivots_run_w(a, tl.circ, lev + 1);   // level lev + 1 ran in reverse
        Dig e;
        ApGeom g{};
        if (act) {
            g = ap_pivot(a, s, K, lev, r, e);
            for (int j = 0; j < N; ++j) {
                double2 v = make_double2(0, 0);
                if ((g.vmask >> j) & 1u) v = __ldcg(F + ap_read_addr(sh, g, K, j, s));
                store_read(s, D, j, t, v, true);
            }
            for (int i = 0; i < N; ++i) {
                double2 v = make_double2(0, 0);
                if ((g.nmask >> i) & 1u) {
                    int den;
                    const int64_t addr = ap_write_addr(sh, g, e, K, i, s, &den);
                    // T2 and P values of a level whose pivots did not run have no
                    // reader: their adjoint is zero (Fbar is not cleared for b = 0)
                    const double2 y = i == 1 ? diag_adjoint<HASB>(a, s, tl.circ, K, lev, g, e, up)
                                      : up ? __ldcg(Fb + addr) : make_double2(0, 0);
                    v = rscale(y, s.inv[den]);
                }
                store_adj(s, D, i, t, v);
            }
            s.FP[t] = HASB ? __ldcg(F + g.fp) : make_double2(0, 0);
        } else {
            for (int j = 0; j < N; ++j) {
                store_read(s, D, j, t, make_double2(0, 0), true);
                store_adj(s, D, j, t, make_double2(0, 0));
            }
            s.FP[t] = make_double2(0, 0);
        }
        const unsigned vm = __reduce_or_sync(0xffffffffu, g.vmask);
        const unsigned nm = __reduce_or_sync(0xffffffffu, g.nmask);
        // adjoint of the reads: Rbar_j = sum_i conj(A_{w_i l_j}) Y_i
        matvec_adj(s, D, 2 * K, N, vm, nm, [&](int j, double2 acc) {
            if (!act || !((g.vmask >> j) & 1u)) return;
            if (j == 0) {
                const int64_t ia = g.lk0 + g.r;
                a.scratch[(size_t)tl.circ * sh.n_ap + box_ap(sh, K, sh.off_ap[K] + ia)] = acc;
            } else {
                // T2 and P1010/P1001 values have this pivot as their only
                // reader, so their adjoint is this one term
                Fb[ap_read_addr(sh, g, K, j, s)] = acc;
            }
        });
        if (HASB && act) {
            double2 fpb = make_double2(0, 0);
            for (int i = 0; i < N; ++i)
                if ((g.nmask >> i) & 1u) fpb = cfma_conj(s.bs[2 * K + i], load_adj(s, D, i, t), fpb);
            const int64_t addr = g.fp;
            Fb[addr] = cadd(__ldcg(Fb + addr), fpb);
        }
        reduce_partials(a, s, tl.circ, K, N, HASB, nm, vm);
    }

    // --------------------------------------------------------- reverse DP
    static __device__ void dp_reverse_tile(const DiagArgs &a, Smem &s, const TileId &tl, int lev)
    {
        const DiagShape &sh = a.sh;
        const int t = threadIdx.x, D = 2 * sh.M, N = D;
        load_circuit(a, s, tl.circ);
        const double2 *F = a.F + (size_t)tl.circ * sh.circ_alloc;
        double2 *Fb = a.Fbar + (size_t)tl.circ * sh.circ_alloc;
        const unsigned r = tl.rank0 + t;
        const bool act = r < tl.count;
        Dig d;
        DpGeom g{};
        if (act) {
            d = unrank(sh, s, 0, 1, lev, r);
            g = dp_geom(sh, d, s, lev, (int64_t)r);
            for (int j = 0; j < N; ++j) {
                double2 v = make_double2(0, 0);
                if ((g.vmask >> j) & 1u) v = __ldcg(F + dp_read_addr(sh, g, j, s));
                store_read(s, D, j, t, v, true);
            }
            for (int i = 0; i < N; ++i) {
                double2 v = make_double2(0, 0);
                if ((g.nmask >> i) & 1u) {
                    int den;
                    const int64_t addr = dp_write_addr(sh, g, d, i, s, &den);
                    v = rscale(__ldcg(Fb + addr), s.inv[den]);
                }
                store_adj(s, D, i, t, v);
            }
            s.FP[t] = __ldcg(F + g.rdiag);
        } else {
            for (int j = 0; j < N; ++j) {
                store_read(s, D, j, t, make_double2(0, 0), true);
                store_adj(s, D, j, t, make_double2(0, 0));
            }
            s.FP[t] = make_double2(0, 0);
        }
        const unsigned vm = __reduce_or_sync(0xffffffffu, g.vmask);
        const unsigned nm = __reduce_or_sync(0xffffffffu, g.nmask);
        matvec_adj(s, D, 0, N, vm, nm, [&](int j, double2 acc) {
            if (!act || !((g.vmask >> j) & 1u)) return;
            const int64_t addr = dp_read_addr(sh, g, j, s);
            Fb[addr] = cadd(__ldcg(Fb + addr), acc);
        });
        if (act) {
            double2 fpb = make_double2(0, 0);
            for (int i = 0; i < N; ++i)
                if ((g.nmask >> i) & 1u) fpb = cfma_conj(s.bs[i], load_adj(s, D, i, t), fpb);
            Fb[g.rdiag] = cadd(__ldcg(Fb + g.rdiag), fpb);
        }
        reduce_partials(a, s, tl.circ, 0, N, true, nm, vm);
    }

    // ------------------------------------------- reverse on the tensor cores
    // Per warp: reads and scaled output adjoints land in the warp's buffers,
    // the warp's partial dL/dA (and dL/db) is formed from them, then the read
    // adjoints conj(A) Y overwrite the read buffer and each lane scatters its
    // own pivot's.
    static __device__ void tc_partb(const DiagArgs &a, const Smem &s, int circ, int row0, int N)
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, D = 2 * a.sh.M;
        const size_t slot = (size_t)blockIdx.x * (TPB / 32) + warp;
        double2 *pb = a.partb + ((size_t)circ * a.slots + slot) * D;
        const double *wy = s.wy + (size_t)warp * XS * WBS;
        for (int w = lane; w < N; w += 32) {
            double2 acc = make_double2(0, 0);
            for (int tt = 0; tt < 32; ++tt)
                acc = cfma_conj(s.FP[warp * 32 + tt], make_double2(wy[(2 * w) * WBS + tt], wy[(2 * w + 1) * WBS + tt]),
                                acc);
            atomicAdd(&pb[row0 + w].x, acc.x);   // one writer, ordered as above
            atomicAdd(&pb[row0 + w].y, acc.y);
        }
    }

    // Row exponents of the warp's partial dL/dA: for row w the largest
    // exponent field of Y_w(t) 2^(e_t - 1022) over the warp's pivots (0: none).
    static __device__ __forceinline__ void tc_row_exponents(Smem &s, int D, int N, int fx)
    {
        const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
        s.wf[t] = fx;
        for (int w = 0; w < N; ++w) {
            int gw = 0;
            if (fx != 0) {
                const double2 y = load_adj(s, D, w, t);
                const int fy = max(fexp(y.x), fexp(y.y));
                if (fy != 0) gw = max(fy + fx - 1022, 0);
            }
            gw = __reduce_max_sync(0xffffffffu, gw);
            if (lane == 0) s.wg[warp * 32 + w] = gw;
        }
        __syncwarp();
    }

    // Reverse step of an AP(K) tile on the tensor engine (the walk): scaled
    // output adjoints into the warp's buffer (the DIAG one formed here and kept
    // in Fbar for the partial pass), the read adjoints conj(A) Y in place, then
    // each lane scatters its pivot's.
    template <bool HASB>
    static __device__ void ap_reverse_tile_tc(const DiagArgs &a, Smem &s, const TileId &tl, int K, int lev)
    {
        const DiagShape &sh = a.sh;
        const int t = threadIdx.x, lane = t & 31, D = 2 * sh.M, N = 2 * (sh.M - K);
        load_circuit(a, s, tl.circ);
        double2 *Fb = a.Fbar + (size_t)tl.circ * sh.circ_alloc;
        const unsigned r = tl.rank0 + t;
        const bool act = r < tl.count;
        const bool up = pivots_run_w(a, tl.circ, lev + 1);   // level lev + 1 ran in reverse
        Dig e;
        ApGeom g{};
        if (act) {
            g = ap_pivot(a, s, K, lev, r, e);
            gather(
                N,
                [&](int i) {
                    if (!((g.nmask >> i) & 1u)) return make_double2(0, 0);
                    int den;
                    const int64_t addr = ap_write_addr(sh, g, e, K, i, s, &den);
                    double2 y;
                    if (i == 1) {
                        y = diag_adjoint<HASB>(a, s, tl.circ, K, lev, g, e, up);
                        Fb[addr] = y;   // complete: the partial pass reads it back
                    } else {
                        // T2 and P values of a level whose pivots did not run have no
                        // reader: their adjoint is zero (Fbar is not cleared for b = 0)
                        y = up ? __ldcg(Fb + addr) : make_double2(0, 0);
                    }
                    return rscale(y, s.inv[den]);
                },
                [&](int i, double2 v) { store_adj(s, D, i, t, v); });
        } else {
            for (int j = 0; j < N; ++j) store_adj(s, D, j, t, make_double2(0, 0));
        }
        double2 fpb = make_double2(0, 0);
        if (HASB && act)
            for (int i = 0; i < N; ++i)
                if ((g.nmask >> i) & 1u) fpb = cfma_conj(s.bs[2 * K + i], load_adj(s, D, i, t), fpb);
        __syncwarp();
        double *wy = s.wy + (size_t)(t >> 5) * XS * WBS;
        tc_products<true>(s, D, 2 * K, N, wy, wy);
        if (act) {
            for (int j = 0; j < N; ++j) {
                if (!((g.vmask >> j) & 1u)) continue;
                const double2 acc = make_double2(wy[(2 * j) * WBS + lane], wy[(2 * j + 1) * WBS + lane]);
                if (j == 0) {
                    const int64_t ia = g.lk0 + g.r;
                    a.scratch[(size_t)tl.circ * sh.n_ap + box_ap(sh, K, sh.off_ap[K] + ia)] = acc;
                } else {
                    Fb[ap_read_addr(sh, g, K, j, s)] = acc;   // the value's only reader
                }
            }
            if (HASB) Fb[g.fp] = cadd(__ldcg(Fb + g.fp), fpb);
        }
        __syncwarp();
    }

    static __device__ void dp_reverse_tile_tc(const DiagArgs &a, Smem &s, const TileId &tl, int lev)
    {
        const DiagShape &sh = a.sh;
        const int t = threadIdx.x, lane = t & 31, D = 2 * sh.M, N = D;
        load_circuit(a, s, tl.circ);
        double2 *Fb = a.Fbar + (size_t)tl.circ * sh.circ_alloc;
        const unsigned r = tl.rank0 + t;
        const bool act = r < tl.count;
        Dig d;
        DpGeom g{};
        if (act) {
            d = unrank(sh, s, 0, 1, lev, r);
            g = dp_geom(sh, d, s, lev, (int64_t)r);
            gather(
                N,
                [&](int i) {
                    if (!((g.nmask >> i) & 1u)) return make_double2(0, 0);
                    int den;
                    const int64_t addr = dp_write_addr(sh, g, d, i, s, &den);
                    return rscale(__ldcg(Fb + addr), s.inv[den]);
                },
                [&](int i, double2 v) { store_adj(s, D, i, t, v); });
        } else {
            for (int j = 0; j < N; ++j) store_adj(s, D, j, t, make_double2(0, 0));
        }
        double2 fpb = make_double2(0, 0);
        if (act)
            for (int i = 0; i < N; ++i)
                if ((g.nmask >> i) & 1u) fpb = cfma_conj(s.bs[i], load_adj(s, D, i, t), fpb);
        __syncwarp();
        double *wy = s.wy + (size_t)(t >> 5) * XS * WBS;
        tc_products<true>(s, D, 0, N, wy, wy);
        if (act) {
            for (int j = 0; j < N; ++j) {
                if (!((g.vmask >> j) & 1u)) continue;
                const double2 acc = make_double2(wy[(2 * j) * WBS + lane], wy[(2 * j + 1) * WBS + lane]);
                const int64_t addr = dp_read_addr(sh, g, j, s);
                Fb[addr] = cadd(__ldcg(Fb + addr), acc);
            }
            Fb[g.rdiag] = cadd(__ldcg(Fb + g.rdiag), fpb);
        }
        __syncwarp();
    }

    // ------------------------------------------ partial dL/dA, dL/db (tensor)
    // After the reverse walk every adjoint is final, so the partial sums
    // sum_t Y_w(t) conj(X_j(t)) (and the dL/db terms) of all pivots are formed
    // in one pass without level barriers: reads X and scaled output adjoints Y
    // are gathered again (the DIAG adjoint from where the walk left it).
    template <bool HASB>
    static __device__ void ap_partial_tile(const DiagArgs &a, Smem &s, const TileId &tl, int K, int lev)
    {
        const DiagShape &sh = a.sh;
        const int t = threadIdx.x, D = 2 * sh.M, N = 2 * (sh.M - K);
        const double2 *F = a.F + (size_t)tl.circ * sh.circ_alloc;
        const double2 *Fb = a.Fbar + (size_t)tl.circ * sh.circ_alloc;
        const unsigned r = tl.rank0 + t;
        const bool act = r < tl.count;
        const bool up = pivots_run_w(a, tl.circ, lev + 1);
        int fx = 0;
        double2 FPv = make_double2(0, 0);
        if (act) {
            Dig e;
            ApRel q;
            const ApGeom g = ap_pivot_regs(a, s, K, lev, r, e, q);
            gather(
                N,
                [&](int j) {
                    return ((g.vmask >> j) & 1u) ? __ldcg(F + ap_read_addr_q(sh, g, K, j, q))
                                                 : make_double2(0, 0);
                },
                [&](int j, double2 v) {
                    fx = max(fx, max(fexp(v.x), fexp(v.y)));
                    store_read(s, D, j, t, v, true);
                });
            gather(
                N,
                [&](int i) {
                    if (!((g.nmask >> i) & 1u)) return make_double2(0, 0);
                    int den;
                    const int64_t addr = ap_write_addr(sh, g, e, K, i, s, &den);
                    const double2 y = (i == 1 || up) ? __ldcg(Fb + addr) : make_double2(0, 0);
                    return rscale(y, s.inv[den]);
                },
                [&](int i, double2 v) { store_adj(s, D, i, t, v); });
            if (HASB) FPv = __ldcg(F + g.fp);
        } else {
            for (int j = 0; j < N; ++j) {
                store_read(s, D, j, t, make_double2(0, 0), true);
                store_adj(s, D, j, t, make_double2(0, 0));
            }
        }
        if (HASB) s.FP[t] = FPv;
        tc_row_exponents(s, D, N, fx);
        tc_partials(a, s, tl.circ, 2 * K, N);
        if (HASB) tc_partb(a, s, tl.circ, 2 * K, N);
        __syncwarp();
    }

    static __device__ void dp_partial_tile(const DiagArgs &a, Smem &s, const TileId &tl, int lev)
    {
        const DiagShape &sh = a.sh;
        const int t = threadIdx.x, D = 2 * sh.M, N = D;
        const double2 *F = a.F + (size_t)tl.circ * sh.circ_alloc;
        const double2 *Fb = a.Fbar + (size_t)tl.circ * sh.circ_alloc;
        const unsigned r = tl.rank0 + t;
        const bool act = r < tl.count;
        int fx = 0;
        double2 FPv = make_double2(0, 0);
        if (act) {
            const Dig d = unrank(sh, s, 0, 1, lev, r);
            const DpGeom g = dp_geom(sh, d, s, lev, (int64_t)r);
            gather(
                N,
                [&](int j) {
                    return ((g.vmask >> j) & 1u) ? __ldcg(F + dp_read_addr(sh, g, j, s)) : make_double2(0, 0);
                },
                [&](int j, double2 v) {
                    fx = max(fx, max(fexp(v.x), fexp(v.y)));
                    store_read(s, D, j, t, v, true);
                });
            gather(
                N,
                [&](int i) {
                    if (!((g.nmask >> i) & 1u)) return make_double2(0, 0);
                    int den;
                    const int64_t addr = dp_write_addr(sh, g, d, i, s, &den);
                    return rscale(__ldcg(Fb + addr), s.inv[den]);
                },
                [&](int i, double2 v) { store_adj(s, D, i, t, v); });
            FPv = __ldcg(F + g.rdiag);
        } else {
            for (int j = 0; j < N; ++j) {
                store_read(s, D, j, t, make_double2(0, 0), true);
                store_adj(s, D, j, t, make_double2(0, 0));
            }
        }
        s.FP[t] = FPv;
        tc_row_exponents(s, D, N, fx);
        tc_partials(a, s, tl.circ, 0, N);
        tc_partb(a, s, tl.circ, 0, N);
        __syncwarp();
    }

    // ------------------------------------------------------------------ kernels
    static __device__ void forward(const DiagArgs &a)
    {
        const DiagShape &sh = a.sh;
        if (skip_walk(a.ctl)) return;
        Smem s = carve_smem(sh, kFwd);
        build_tables(sh, s);
        prologue(a, s, true);
        if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
        if (a.geo != nullptr && blockIdx.x == 0 && threadIdx.x == 0) a.ctl->geo_key = a.geo_key;
        const int hb = *(volatile int *)&a.ctl->has_b;
        if (hb && !sh.has_b) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&a.ctl->status, 0, (int)FK_EBZERO);
            return;
        }
        if (a.pc) {
            for (int c = next_circuit(a.ctr + 2 * sh.L); c < a.B; c = next_circuit(a.ctr + 2 * sh.L)) {
                for (int lev = 0; lev < sh.L; ++lev) {
                    if (hb) {
                        circuit_tiles(a, c, phase_tiles(a, s, 1, lev), [&](int tile) {
                            const TileId tl = decode_tile(a, s, 1, lev, tile);
                            if (pivots_run(a, c, lev)) dp_forward_tile(a, s, tl, lev);
                        });
                    }
                    circuit_tiles(a, c, phase_tiles(a, s, 0, lev), [&](int tile) {
                        const TileId tl = decode_tile(a, s, 0, lev, tile);
                        if (!pivots_run(a, c, lev)) return;
                        if (a.early) {
                            if (hb) ap_forward_tile<true, true>(a, s, tl, tl.seg, lev);
                            else ap_forward_tile<false, true>(a, s, tl, tl.seg, lev);
                        } else {
                            if (hb) ap_forward_tile<true, false>(a, s, tl, tl.seg, lev);
                            else ap_forward_tile<false, false>(a, s, tl, tl.seg, lev);
                        }
                    });
                }
                if (a.early && a.levels != nullptr && threadIdx.x == 0) {
                    int n = 0;
                    while (n < sh.L && pivots_run(a, c, n)) ++n;
                    a.levels[c] = n + 1;
                }
            }
            return;
        }
        for (int lev = 0; lev < sh.L; ++lev) {
            if (hb) {
                const int nt = phase_tiles(a, s, 1, lev);
                run_tiles(a.ctr + 2 * lev, nt, [&](int tile) {
                    const TileId tl = decode_tile(a, s, 1, lev, tile);
                    if (!pivots_run(a, tl.circ, lev)) return;
                    dp_forward_tile(a, s, tl, lev);
                });
                if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
                trace_mark(a.trace, a.trace_cap, kTraceFwd | (lev << 8) | 1u);
            }
            const int nt = phase_tiles(a, s, 0, lev);
            run_tiles(a.ctr + 2 * lev + 1, nt, [&](int tile) {
                const TileId tl = decode_tile(a, s, 0, lev, tile);
                if (!pivots_run(a, tl.circ, lev)) return;
                if (a.early) {
                    if (hb) ap_forward_tile<true, true>(a, s, tl, tl.seg, lev);
                    else ap_forward_tile<false, true>(a, s, tl, tl.seg, lev);
                } else {
                    if (hb) ap_forward_tile<true, false>(a, s, tl, tl.seg, lev);
                    else ap_forward_tile<false, false>(a, s, tl, tl.seg, lev);
                }
            });
            if ((lev + 1 < sh.L || a.early) && !grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
            trace_mark(a.trace, a.trace_cap, kTraceFwd | (lev << 8));
        }
        if (a.early && a.levels != nullptr && blockIdx.x == 0) {
            // photon numbers completed: 0 .. (first level whose pivots did not run)
            for (int c = threadIdx.x; c < a.B; c += blockDim.x) {
                int n = 0;
                while (n < sh.L && pivots_run(a, c, n)) ++n;
                a.levels[c] = n + 1;
            }
        }
    }

    static __device__ void vjp(const DiagArgs &a)
    {
        const DiagShape &sh = a.sh;
        if (skip_walk(a.ctl)) return;
        Smem s = carve_smem(sh, kVjp);
        build_tables(sh, s);
        prologue(a, s, false);
        if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
        const int hb = *(volatile int *)&a.ctl->has_b;
        if (hb && !sh.has_b) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&a.ctl->status, 0, (int)FK_EBZERO);
            return;
        }
        if (a.pc) {
            for (int c = next_circuit(a.ctr + 2 * sh.L); c < a.B; c = next_circuit(a.ctr + 2 * sh.L)) {
                for (int lev = sh.L - 1; lev >= 0; --lev) {
                    circuit_tiles(a, c, phase_tiles(a, s, 0, lev), [&](int tile) {
                        const TileId tl = decode_tile(a, s, 0, lev, tile);
                        if (!pivots_run_w(a, c, lev)) return;
                        if constexpr (TC) {
                            if (hb) ap_reverse_tile_tc<true>(a, s, tl, tl.seg, lev);
                            else ap_reverse_tile_tc<false>(a, s, tl, tl.seg, lev);
                        } else {
                            if (hb) ap_reverse_tile<true>(a, s, tl, tl.seg, lev);
                            else ap_reverse_tile<false>(a, s, tl, tl.seg, lev);
                        }
                    });
                    if (hb) {
                        circuit_tiles(a, c, phase_tiles(a, s, 1, lev), [&](int tile) {
                            const TileId tl = decode_tile(a, s, 1, lev, tile);
                            if (!pivots_run_w(a, c, lev)) return;
                            if constexpr (TC) dp_reverse_tile_tc(a, s, tl, lev);
                            else dp_reverse_tile(a, s, tl, lev);
                        });
                    }
                }
            }
            if constexpr (!TC) finish_vjp(a, hb);
            return;
        }
        for (int lev = sh.L; lev >= 0; --lev) {
            if (lev < sh.L) {
                const int nt = phase_tiles(a, s, 0, lev);
                run_tiles(a.ctr + 2 * lev + 1, nt, [&](int tile) {
                    const TileId tl = decode_tile(a, s, 0, lev, tile);
                    if (!pivots_run_w(a, tl.circ, lev)) return;
                    if constexpr (TC) {
                        if (hb) ap_reverse_tile_tc<true>(a, s, tl, tl.seg, lev);
                        else ap_reverse_tile_tc<false>(a, s, tl, tl.seg, lev);
                    } else {
                        if (hb) ap_reverse_tile<true>(a, s, tl, tl.seg, lev);
                        else ap_reverse_tile<false>(a, s, tl, tl.seg, lev);
                    }
                });
                if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
                trace_mark(a.trace, a.trace_cap, kTraceVjp | (lev << 8));
            }
            if (hb && lev < sh.L) {
                const int nt = phase_tiles(a, s, 1, lev);
                run_tiles(a.ctr + 2 * lev, nt, [&](int tile) {
                    const TileId tl = decode_tile(a, s, 1, lev, tile);
                    if (!pivots_run_w(a, tl.circ, lev)) return;
                    if constexpr (TC) dp_reverse_tile_tc(a, s, tl, lev);
                    else dp_reverse_tile(a, s, tl, lev);
                });
                if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
                trace_mark(a.trace, a.trace_cap, kTraceVjp | (lev << 8) | 1u);
            }
        }
        if constexpr (!TC) finish_vjp(a, hb);   // the tensor engine's partial pass finishes
    }

    // Partial dL/dA and dL/db of every pivot (tensor engine, after the walk):
    // no level barriers, one counter per (level, kind) from the second half of
    // the counter array; then the final reduction.
    static __device__ void vjp_partials(const DiagArgs &a)
    {
        const DiagShape &sh = a.sh;
        if (skip_walk(a.ctl) || ld_status(a.ctl) != 0) return;   // no walk, or it failed
        Smem s = carve_smem(sh, kPart);
        build_tables(sh, s);
        __syncthreads();
        const int hb = *(volatile int *)&a.ctl->has_b;
        int *ctr = a.ctr + 2 * (sh.L + 1);
        for (int lev = 0; lev < sh.L; ++lev) {
            const int nt = phase_tiles(a, s, 0, lev);
            run_tiles(ctr + 2 * lev + 1, nt, [&](int tile) {
                const TileId tl = decode_tile(a, s, 0, lev, tile);
                if (!pivots_run_w(a, tl.circ, lev)) return;
                if (hb) ap_partial_tile<true>(a, s, tl, tl.seg, lev);
                else ap_partial_tile<false>(a, s, tl, tl.seg, lev);
            });
            if (hb) {
                const int nd = phase_tiles(a, s, 1, lev);
                run_tiles(ctr + 2 * lev, nd, [&](int tile) {
                    const TileId tl = decode_tile(a, s, 1, lev, tile);
                    if (!pivots_run_w(a, tl.circ, lev)) return;
                    dp_partial_tile(a, s, tl, lev);
                });
            }
        }
        finish_vjp(a, hb);
    }

    // Final reduction of the partial slots (fixed order -> deterministic),
    // symmetrisation dL/dA <- (dL/dA + dL/dA^T)/2, scatter to the caller's
    // modes, and dL/dc.
    static __device__ void finish_vjp(const DiagArgs &a, int hb)
    {
        zero_grads(a);
        if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
        trace_mark(a.trace, a.trace_cap, kTraceFinish);
        reduce_grads(a, hb);
    }

    static __device__ void zero_grads(const DiagArgs &a)
    {
        const int Do = a.sh.D_orig;
        const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
        for (int64_t e = gtid; e < (int64_t)a.B * Do * Do; e += gsz)
            a.gA[cix(a, (int)(e / (Do * Do))) * Do * Do + e % (Do * Do)] = make_double2(0, 0);
        for (int64_t e = gtid; e < (int64_t)a.B * Do; e += gsz)
            a.gb[cix(a, (int)(e / Do)) * Do + e % Do] = make_double2(0, 0);
    }

    // Sum of a double2 over the 32 lanes (xor butterfly: a fixed order, so
    // the result does not depend on timing).
    static __device__ __forceinline__ double2 warp_sum2(double2 v)
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        }
        return v;
    }

    // One warp per gradient entry: the lanes sum interleaved subsets of the
    // slots (all loads independent), then a butterfly joins them.
    static __device__ void reduce_grads(const DiagArgs &a, int hb)
    {
        const DiagShape &sh = a.sh;
        const int D = 2 * sh.M, Do = sh.D_orig, lane = threadIdx.x & 31;
        const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
        const int64_t nA = (int64_t)a.B * D * D, nb = (int64_t)a.B * D;
        for (int64_t e = gw; e < nA + nb; e += nw) {
            if (e < nA) {
                const int c = (int)(e / (D * D));
                const int w = (int)((e / D) % D), l = (int)(e % D);
                double2 x = make_double2(0, 0), y = make_double2(0, 0);
                const double2 *pA = a.partA + (size_t)c * a.slots * D * D;
                for (int blk = lane; blk < a.slots; blk += 32) {
                    x = cadd(x, __ldcg(pA + (size_t)blk * D * D + (size_t)w * D + l));
                    y = cadd(y, __ldcg(pA + (size_t)blk * D * D + (size_t)l * D + w));
                }
                x = warp_sum2(x);
                y = warp_sum2(y);
                if (lane == 0) {
                    const int ow = 2 * sh.mode_map[w / 2] + (w & 1), ol = 2 * sh.mode_map[l / 2] + (l & 1);
                    a.gA[cix(a, c) * Do * Do + (size_t)ow * Do + ol] =
                        make_double2(0.5 * (x.x + y.x), 0.5 * (x.y + y.y));
                }
            } else {
                const int64_t f = e - nA;
                const int c = (int)(f / D), w = (int)(f % D);
                double2 x = make_double2(0, 0);
                for (int blk = lane; blk < a.slots; blk += 32)
                    x = cadd(x, __ldcg(a.partb + ((size_t)c * a.slots + blk) * D + w));
                x = warp_sum2(x);
                if (lane == 0) a.gb[cix(a, c) * Do + 2 * sh.mode_map[w / 2] + (w & 1)] = x;
            }
        }
        const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
        for (int64_t c = gtid; c < a.B; c += gsz) a.gc[cix(a, (int)c)] = vacuum_adjoint(a, (int)c, hb != 0);
    }

    // ------------------------------------------------ several shapes, one launch
    // Circuits with different cutoffs run in one cooperative launch: they are
    // grouped by shape on the host, each group keeps its own storage, tables
    // and geometry, and every phase (level, kind) hands out the tiles of all
    // groups through one counter (group-major, then circuit-major within a
    // group), so the levels of every shape advance together between the
    // same grid barriers.  A block that takes a tile of another group, level
    // or kind rebuilds its prefix table and phase offsets for it.

    // Word copy of the launch's arguments into each group's view, then the
    // group's fields (one block per group).
    static __device__ void make_views(const DiagArgs &a)
    {
        constexpr int W = (int)(sizeof(DiagArgs) / sizeof(unsigned long long));
        static_assert(sizeof(DiagArgs) % sizeof(unsigned long long) == 0, "DiagArgs is whole words");
        for (int g = blockIdx.x; g < a.G; g += gridDim.x) {
            const unsigned long long *src = (const unsigned long long *)&a;
            unsigned long long *dst = (unsigned long long *)&a.gargs[g];
            for (int i = threadIdx.x; i < W; i += blockDim.x) dst[i] = src[i];
            __syncthreads();
            if (threadIdx.x == 0) {
                const DiagGroup &q = a.grp[g];
                DiagArgs &v = a.gargs[g];
                v.G = 0;
                v.B = q.B;
                v.slots = q.slots;
                v.As = (double2 *)(a.wsbase + q.As);
                v.bs = (double2 *)(a.wsbase + q.bs);
                v.dig = (unsigned char *)(a.wsbase + q.dig);
                v.geo = q.geo >= 0 ? (int *)(a.wsbase + q.geo) : nullptr;
                v.F = (double2 *)(a.wsbase + q.F);
                v.Fbar = q.Fbar >= 0 ? (double2 *)(a.wsbase + q.Fbar) : nullptr;
                v.scratch = q.scratch >= 0 ? (double2 *)(a.wsbase + q.scratch) : nullptr;
                v.partA = q.partA >= 0 ? (double2 *)(a.wsbase + q.partA) : nullptr;
                v.partb = q.partb >= 0 ? (double2 *)(a.wsbase + q.partb) : nullptr;
                v.cidx = a.cidx + q.first;
                v.oidx = a.oidx + q.first;
            }
            __syncthreads();
            // the shape last (many words; one thread per word)
            const unsigned long long *ss = (const unsigned long long *)&a.grp[g].sh;
            unsigned long long *sd = (unsigned long long *)&a.gargs[g].sh;
            for (int i = threadIdx.x; i < (int)(sizeof(DiagShape) / 8); i += blockDim.x) sd[i] = ss[i];
            __syncthreads();
        }
    }

    // Tables of group g for phase (kind, lev) in this block; uniform per block.
    static __device__ const DiagArgs &enter_group(const DiagArgs &a, Smem &s, int g, int kind, int lev)
    {
        const DiagArgs &ag = a.gargs[g];
        const int key = (g * (a.sh.L + 1) + lev) * 2 + kind;
        if (s.multi_key != key) {
            const int prev = s.multi_key < 0 ? -1 : s.multi_key / (2 * (a.sh.L + 1));
            if (prev != g) {
                __syncthreads();
                s.Wn = ag.sh.L + 2;
                build_prefix_table(s.S, s.Wn, ag.sh.C, ag.sh.M);
                s.loaded_circ = -1;
            }
            phase_tiles(ag, s, kind, lev);
            s.multi_key = key;
        }
        return ag;
    }

    // Group and group-local tile of tile `tile` of phase (kind, lev).
    static __device__ __forceinline__ int tile_group(const DiagArgs &a, int kind, int lev, int tile, int *local)
    {
        const int *pre = a.gtiles + (size_t)(2 * lev + kind) * (a.G + 1);
        int g = 0;
        while (g + 1 < a.G && tile >= pre[g + 1]) ++g;
        *local = tile - pre[g];
        return g;
    }

    static __device__ __forceinline__ int multi_tiles(const DiagArgs &a, int kind, int lev)
    {
        return a.gtiles[(size_t)(2 * lev + kind) * (a.G + 1) + a.G];
    }

    // Prologue of every group: views, then each group's A_s, b, digits,
    // geometry and seeds (its prefix table rebuilt first); the tile counters
    // of the launch are cleared once.
    static __device__ bool multi_prologue(const DiagArgs &a, Smem &s, bool seed)
    {
        const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
        make_views(a);
        for (int64_t e = gtid; e < 4 * (int64_t)(a.sh.L + 1); e += gsz) a.ctr[e] = 0;
        if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return false;
        for (int g = 0; g < a.G; ++g) {
            const DiagArgs &ag = a.gargs[g];
            __syncthreads();
            s.Wn = ag.sh.L + 2;
            build_prefix_table(s.S, s.Wn, ag.sh.C, ag.sh.M);
            prologue(ag, s, seed, false);
        }
        s.multi_key = -1;
        s.loaded_circ = -1;
        return grid_sync(a.ctl, gridDim.x, a.timeout_ns);
    }

    static __device__ void forward_multi(const DiagArgs &a)
    {
        const int L = a.sh.L;
        Smem s = carve_smem(a.sh, kFwd);
        build_scalar_tables(s.inv, s.fact);
        if (!multi_prologue(a, s, true)) return;
        const int hb = *(volatile int *)&a.ctl->has_b;
        if (hb && !a.sh.has_b) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&a.ctl->status, 0, (int)FK_EBZERO);
            return;
        }
        for (int lev = 0; lev < L; ++lev) {
            if (hb) {
                run_tiles(a.ctr + 2 * lev, multi_tiles(a, 1, lev), [&](int tile) {
                    int local;
                    const int g = tile_group(a, 1, lev, tile, &local);
                    const DiagArgs &ag = enter_group(a, s, g, 1, lev);
                    dp_forward_tile(ag, s, decode_tile(ag, s, 1, lev, local), lev);
                });
                if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
            }
            run_tiles(a.ctr + 2 * lev + 1, multi_tiles(a, 0, lev), [&](int tile) {
                int local;
                const int g = tile_group(a, 0, lev, tile, &local);
                const DiagArgs &ag = enter_group(a, s, g, 0, lev);
                const TileId tl = decode_tile(ag, s, 0, lev, local);
                if (hb) ap_forward_tile<true, false>(ag, s, tl, tl.seg, lev);
                else ap_forward_tile<false, false>(ag, s, tl, tl.seg, lev);
            });
            if (lev + 1 < L && !grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
        }
    }

    static __device__ void vjp_multi(const DiagArgs &a)
    {
        const int L = a.sh.L;
        Smem s = carve_smem(a.sh, kVjp);
        build_scalar_tables(s.inv, s.fact);
        if (!multi_prologue(a, s, false)) return;
        const int hb = *(volatile int *)&a.ctl->has_b;
        if (hb && !a.sh.has_b) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&a.ctl->status, 0, (int)FK_EBZERO);
            return;
        }
        for (int lev = L - 1; lev >= 0; --lev) {
            run_tiles(a.ctr + 2 * lev + 1, multi_tiles(a, 0, lev), [&](int tile) {
                int local;
                const int g = tile_group(a, 0, lev, tile, &local);
                const DiagArgs &ag = enter_group(a, s, g, 0, lev);
                const TileId tl = decode_tile(ag, s, 0, lev, local);
                if constexpr (TC) {
                    if (hb) ap_reverse_tile_tc<true>(ag, s, tl, tl.seg, lev);
                    else ap_reverse_tile_tc<false>(ag, s, tl, tl.seg, lev);
                } else {
                    if (hb) ap_reverse_tile<true>(ag, s, tl, tl.seg, lev);
                    else ap_reverse_tile<false>(ag, s, tl, tl.seg, lev);
                }
            });
            if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
            if (hb) {
                run_tiles(a.ctr + 2 * lev, multi_tiles(a, 1, lev), [&](int tile) {
                    int local;
                    const int g = tile_group(a, 1, lev, tile, &local);
                    const DiagArgs &ag = enter_group(a, s, g, 1, lev);
                    const TileId tl = decode_tile(ag, s, 1, lev, local);
                    if constexpr (TC) dp_reverse_tile_tc(ag, s, tl, lev);
                    else dp_reverse_tile(ag, s, tl, lev);
                });
                if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
            }
        }
        if constexpr (!TC) finish_multi(a, hb);
    }

    static __device__ void vjp_partials_multi(const DiagArgs &a)
    {
        if (skip_walk(a.ctl) || ld_status(a.ctl) != 0) return;
        const int L = a.sh.L;
        Smem s = carve_smem(a.sh, kPart);
        build_scalar_tables(s.inv, s.fact);
        __syncthreads();
        const int hb = *(volatile int *)&a.ctl->has_b;
        int *ctr = a.ctr + 2 * (L + 1);
        for (int lev = 0; lev < L; ++lev) {
            run_tiles(ctr + 2 * lev + 1, multi_tiles(a, 0, lev), [&](int tile) {
                int local;
                const int g = tile_group(a, 0, lev, tile, &local);
                const DiagArgs &ag = enter_group(a, s, g, 0, lev);
                const TileId tl = decode_tile(ag, s, 0, lev, local);
                if (hb) ap_partial_tile<true>(ag, s, tl, tl.seg, lev);
                else ap_partial_tile<false>(ag, s, tl, tl.seg, lev);
            });
            if (hb) {
                run_tiles(ctr + 2 * lev, multi_tiles(a, 1, lev), [&](int tile) {
                    int local;
                    const int g = tile_group(a, 1, lev, tile, &local);
                    const DiagArgs &ag = enter_group(a, s, g, 1, lev);
                    dp_partial_tile(ag, s, decode_tile(ag, s, 1, lev, local), lev);
                });
            }
        }
        finish_multi(a, hb);
    }

    static __device__ void finish_multi(const DiagArgs &a, int hb)
    {
        for (int g = 0; g < a.G; ++g) zero_grads(a.gargs[g]);
        if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
        for (int g = 0; g < a.G; ++g) reduce_grads(a.gargs[g], hb);
    }

    // Vacuum-only problem (every cutoff is 1): p = c.
};

template <int TPB, int CH, int KS>
__global__ void __launch_bounds__(TPB, (KS > 2 ? 2 : (KS > 0 ? 4 : 1))) diag_forward_kernel(const __grid_constant__ DiagArgs a)
{
    FK_DBG_BEGIN(a.ctl);
    if (a.G == 0) Walk<TPB, CH, KS>::forward(a);
    else if (!skip_walk(a.ctl)) Walk<TPB, CH, KS>::forward_multi(a);
}

template <int TPB, int CH, int KS>
__global__ void __launch_bounds__(TPB, (KS > 2 ? 2 : (KS > 0 ? 4 : 1))) diag_vjp_kernel(const __grid_constant__ DiagArgs a)
{
    FK_DBG_BEGIN(a.ctl);
    if (a.G == 0) Walk<TPB, CH, KS>::vjp(a);
    else if (!skip_walk(a.ctl)) Walk<TPB, CH, KS>::vjp_multi(a);
}

template <int TPB, int CH, int KS>
__global__ void __launch_bounds__(TPB, (KS > 2 ? 2 : (KS > 0 ? 3 : 1))) diag_vjp_partials_kernel(const __grid_constant__ DiagArgs a)
{
    FK_DBG_BEGIN(a.ctl);
    if constexpr (KS > 0) {
        if (a.G == 0) Walk<TPB, CH, KS>::vjp_partials(a);
        else Walk<TPB, CH, KS>::vjp_partials_multi(a);
    }
}

}  // namespace
}  // namespace fk
