// walk_cond_impl.cuh -- device code of the conditional-state walk
// (Algorithm 2 of arXiv 2303.08879, Sec. 3.2) and its reverse-mode adjoint,
// as templates over the product engine (KS = 0: FP64; KS = 1..3: the
// tensor-core digits); walk_cond_k0.cu .. walk_cond_k3.cu instantiate one
// engine each (parallel translation units) and walk_cond.cu holds the host
// side.
//
// Every circuit of a batch may have its own cutoffs; all share the mode count
// and the detected/undetected split.  Amplitudes are carried as
// F = G / sqrt(k!) (see walk_diag.cu); the amplitude at (u, y) -- u a point
// of the undetected sub-lattice, y a position of the Algorithm-1 structure of
// the detected modes -- lives at F[y * U2 + u], so the u-block of one
// detected position is contiguous and a warp of consecutive u reads and
// writes coalesced lines.
//
// Step 1 (zero photons detected): one block per circuit runs eq. (recrel)
// over the undetected sub-lattice level by level.  Step 2: the detected
// levels of Algorithm 1 (diagonal pivots, then off-diagonal pivots), each
// pivot applied to every u of its block (Algorithm 2); a
// thread owns one (pivot, u) pair and reads (u, P - 1_l) for detected l,
// (u - 1_t, P) for undetected t and, when b != 0, (u, P).  All pairs of one
// detected level are independent.
#pragma once

#include <cuda_runtime.h>

#include "fk_internal.h"
#include "walk_common.cuh"
#include "walk_digits.cuh"
#include "../../include/fockdiag.h"

namespace fk {

namespace {

constexpr int TPB = kCondTPB;
constexpr int RS = TPB + 1;
constexpr int MAXB = 1024;                        // circuits per launch

struct PGeom;

struct CondArgs {
    int B, Md, Dmax, grid, Lmax, D_orig;
    int spb, slots;                 // partial-sum slots per block (1, or one per warp for the
                                    // tensor engine) and per circuit (grid x spb)
    unsigned char *dig;             // tensor engine: per-circuit digit fragments of the reduced A
    const CondCirc *plan;
    const unsigned *Wall;
    const double2 *A, *b, *c;
    double2 *rho;
    Control *ctl;
    double2 *Ar, *br, *F;
    PGeom *geo;                     // pivot geometry of every circuit (built by the prologue)
    const double2 *grho;
    double2 *Fbar, *scratch, *partA, *partb;
    double2 *gA, *gb, *gc;
    unsigned long long timeout_ns;
};

// Positions (in the detected structure) of one pivot's reads and writes;
// every thread of a tile shares the pivot, so thread 0 computes them once per
// tile into shared memory.
struct PGeom {
    int64_t yP;                 // pivot position
    int64_t ia;                 // AP pivot: its entry in the diagonal-read scratch
    int64_t yr[2 * FK_MAXM];    // read positions, column j
    int64_t yw[2 * FK_MAXM];    // write positions, row i
    int den[2 * FK_MAXM];       // P_w + 1 of row i
    unsigned vmask, nmask;      // valid detected reads / needed writes
    int N;                      // rows = detected read columns
    int row0;                   // first detected lattice index of rows/cols (2K or 0)
    double fdiag;               // prod d_j! of the diagonal written by row 1 (AP)
};

struct CSmem {
    double *inv, *fact, *sqf;   // 1/v, v!, sqrt(v!)
    double2 *Ar, *br;           // current circuit's reduced A (Dmax x Dmax) and b
    double *A3;                 // FP64 engine: [3][Dmax][Dmax]: Re A, Re A + Im A, Im A - Re A
    double *R3, *Y3;            // FP64 engine: [3][Dmax][RS] reads (Re x, Im x, Re x + Im x), scaled
                                // output adjoints (Re y, Im y, Re y + Im y)
    double2 *FP;                // [RS] pivot values (VJP)
    uint4 *Af;                  // tensor engine: [KS][KS][7][32] digit fragments of the real form
                                // of the reduced A (m16n8k16 A-operand order)
    int *fA;                    // tensor engine: [16 KS] row exponent fields
    double *wx, *wy;            // tensor engine: per-warp [16 KS][kCWBS] reads (products in place)
                                // and scaled output adjoints (VJP)
    int *wf, *wg;               // tensor VJP: exponent of each pair's largest read; per-warp [32]
                                // row exponents of the partial dL/dA
    PGeom *geo;                 // the current tile's pivot
    int *ctiles;                // [MAXB + 1] tile prefix over circuits
    unsigned char *s1;          // the per-tile buffers, free while step 1 runs: its
    size_t s1_bytes;            // staging area (amplitudes and levels of the u-block)
    int loaded;
};

constexpr int kCWBS = 34;       // column stride (doubles) of a tensor-engine per-warp buffer

// K steps of 16 real rows the tensor engine needs for Dmax reduced indices:
// the real form of the augmented (Dmax + 1) x (Dmax + 1) matrix [[A, b], [b^T, 0]].
__host__ __device__ inline int cond_ks(int Dmax)
{
    return (2 * (Dmax + 1) + 15) / 16;
}

// Shared-memory plan (host sizing and device carving use the same one).
// KS = 0: the FP64 engine; KS > 0: the tensor engine with 16 KS real rows.
struct CondSmemPlan {
    size_t tab, Ar, br, A3, R3, Y3, FP, Af, fA, wx, wy, wf, wg, geo, ctiles, bytes;
};

__host__ __device__ inline CondSmemPlan cond_smem_plan(int Dmax, bool vjp, int KS)
{
    CondSmemPlan q;
    const size_t Dm = (size_t)Dmax, none = ~(size_t)0;
    q.A3 = q.R3 = q.Y3 = q.FP = q.Af = q.fA = q.wx = q.wy = q.wf = q.wg = none;
    size_t n = 0;
    const auto al = [&n]() { n = (n + 15) & ~(size_t)15; };
    q.tab = n; n += 3 * kTabN * sizeof(double); al();
    q.Ar = n; n += Dm * Dm * sizeof(double2);
    q.br = n; n += Dm * sizeof(double2); al();
    if (KS == 0) {
        q.A3 = n; n += 3 * Dm * Dm * sizeof(double); al();
        q.R3 = n; n += 3 * Dm * RS * sizeof(double); al();   // at most 2M matrix columns per pivot
        if (vjp) {
            q.Y3 = n; n += 3 * Dm * RS * sizeof(double); al();
            q.FP = n; n += RS * sizeof(double2); al();
        }
    } else {
        const size_t buf = (size_t)(TPB / 32) * 16 * KS * kCWBS * sizeof(double);
        q.Af = n; n += (size_t)KS * KS * kNDig * 32 * sizeof(uint4); al();
        q.fA = n; n += 16 * (size_t)KS * sizeof(int); al();
        q.wx = n; n += buf; al();
        if (vjp) {
            q.wy = n; n += buf; al();
            q.FP = n; n += TPB * sizeof(double2); al();
            q.wf = n; n += TPB * sizeof(int); al();
            q.wg = n; n += TPB * sizeof(int); al();
        }
    }
    q.geo = n; n += sizeof(PGeom); al();
    q.ctiles = n; n += (MAXB + 1) * sizeof(int);
    q.bytes = n + 64;
    return q;
}

__host__ __device__ inline size_t cond_smem_bytes(int Dmax, bool vjp, int KS)
{
    return cond_smem_plan(Dmax, vjp, KS).bytes;
}

__device__ CSmem carve(const CondArgs &a, bool vjp, int KS)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CondSmemPlan q = cond_smem_plan(a.Dmax, vjp, KS);
    const auto at = [&](size_t o) { return o == ~(size_t)0 ? nullptr : (void *)(smem_raw + o); };
    CSmem s;
    s.inv = (double *)at(q.tab);
    s.fact = s.inv + kTabN;
    s.sqf = s.fact + kTabN;
    s.Ar = (double2 *)at(q.Ar);
    s.br = (double2 *)at(q.br);
    s.A3 = (double *)at(q.A3);
    s.R3 = (double *)at(q.R3);
    s.Y3 = (double *)at(q.Y3);
    s.FP = (double2 *)at(q.FP);
    s.Af = (uint4 *)at(q.Af);
    s.fA = (int *)at(q.fA);
    s.wx = (double *)at(q.wx);
    s.wy = (double *)at(q.wy);
    s.wf = (int *)at(q.wf);
    s.wg = (int *)at(q.wg);
    s.geo = (PGeom *)at(q.geo);
    s.ctiles = (int *)at(q.ctiles);
    const size_t lo = KS > 0 ? q.wx : q.R3;   // per-tile buffers up to the tile's geometry
    s.s1 = smem_raw + lo;
    s.s1_bytes = q.geo - lo;
    s.loaded = -1;
    return s;
}

// Plane k (0: Re, 1: Im, 2: Re + Im) of column j of a per-thread buffer.
__device__ __forceinline__ double &pl(double *buf, int Dm, int k, int j, int t)
{
    return buf[((size_t)k * Dm + j) * RS + t];
}

__device__ __forceinline__ void put3(double *buf, int Dm, int j, int t, double2 v)
{
    pl(buf, Dm, 0, j, t) = v.x;
    pl(buf, Dm, 1, j, t) = v.y;
    pl(buf, Dm, 2, j, t) = v.x + v.y;
}

__device__ __forceinline__ double2 get2(double *buf, int Dm, int j, int t)
{
    return make_double2(pl(buf, Dm, 0, j, t), pl(buf, Dm, 1, j, t));
}

__device__ void build_tables(CSmem &s)
{
    build_scalar_tables(s.inv, s.fact);
    for (int v = threadIdx.x; v < kTabN; v += blockDim.x) {
        double f = 1.0;
        for (int u = 2; u <= v; ++u) f *= sqrt((double)u);
        s.sqf[v] = f;
    }
    __syncthreads();
}

__device__ __forceinline__ LevelTab ltab(const CondArgs &a, const CondCirc &cc)
{
    return LevelTab{a.Wall + cc.W_off, cc.Wn};
}

__device__ void load_circuit(const CondArgs &a, CSmem &s, int c)
{
    if (s.loaded == c) return;
    __syncthreads();
    const int Dm = a.Dmax;
    for (int e = threadIdx.x; e < Dm * Dm; e += blockDim.x) {
        const double2 v = a.Ar[(size_t)c * Dm * Dm + e];
        s.Ar[e] = v;
        if (s.A3 != nullptr) {
            s.A3[e] = v.x;
            s.A3[Dm * Dm + e] = v.x + v.y;
            s.A3[2 * Dm * Dm + e] = v.y - v.x;
        }
    }
    for (int e = threadIdx.x; e < Dm; e += blockDim.x) s.br[e] = a.br[(size_t)c * Dm + e];
    if (s.Af != nullptr) {
        // tensor engine: the digit fragments and row exponents written by the prologue
        const int KS = cond_ks(Dm);
        const unsigned char *src = a.dig + (size_t)c * kDigBytes;
        const uint4 *gf = (const uint4 *)(src + 256);
        for (int e = threadIdx.x; e < KS * KS * kNDig * 32; e += blockDim.x) s.Af[e] = __ldcg(gf + e);
        for (int r = threadIdx.x; r < 16 * KS; r += blockDim.x) s.fA[r] = __ldcg((const int *)src + r);
    }
    __syncthreads();
    s.loaded = c;
}

// Checked indices (debug-checks build, see walk_common.cuh): amplitude
// (y, u) of circuit cc in F / Fbar, with y a position of the detected
// structure and u a point of the u-block; an entry of its output block; of
// its diagonal-read scratch.
__device__ __forceinline__ int64_t fpos(const CondCirc &cc, int64_t y, int64_t u)
{
    return FK_BOX(FK_BOX(y, 0, cc.dsh.circ_size) * cc.U2 + FK_BOX(u, 0, cc.U2), 0, cc.dsh.circ_size * cc.U2);
}

__device__ __forceinline__ int64_t rpos(const CondCirc &cc, int64_t i)
{
    return cc.off_rho + FK_BOX(i, 0, cc.n_patterns * cc.NUo * cc.NUo);
}

__device__ __forceinline__ int64_t spos(const CondCirc &cc, int64_t ia, int64_t u)
{
    return cc.off_scratch + FK_BOX(FK_BOX(ia, 0, cc.dsh.n_ap) * cc.U2 + u, 0, cc.dsh.n_ap * cc.U2);
}

// u-block digit t of flat index u.
__device__ __forceinline__ int udigit(const CondCirc &cc, int u, int t)
{
    return (u / cc.ustride[t]) % cc.CU[t >> 1];
}

// sqrt(prod_t u_t!) and the output (ket, bra) flat indices of u.
__device__ __forceinline__ double uscale(const CondCirc &cc, const CSmem &s, int u, int *ket,
                                         int *bra)
{
    double f = 1.0;
    int k = 0, b = 0;
    for (int a = 0; a < cc.nU; ++a) {
        const int uk = udigit(cc, u, 2 * a), ub = udigit(cc, u, 2 * a + 1);
        f *= s.sqf[uk] * s.sqf[ub];
        k = k * cc.CU[a] + uk;
        b = b * cc.CU[a] + ub;
    }
    *ket = k;
    *bra = b;
    return f;
}

// ------------------------------------------------------------- prologue
__device__ void prologue(const CondArgs &a)
{
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int Dm = a.Dmax, Do = a.D_orig;
    int nz = 0;
    for (int64_t e = gtid; e < (int64_t)a.B * Dm * Dm; e += gsz) {
        const int c = (int)(e / (Dm * Dm));
        const int w = (int)((e / Dm) % Dm), l = (int)(e % Dm);
        const CondCirc &cc = a.plan[c];
        double2 v = czero();
        if (w < cc.Dred && l < cc.Dred) {
            const int ow = cc.red_to_orig[w], ol = cc.red_to_orig[l];
            const double2 x = a.A[(size_t)c * Do * Do + (size_t)ow * Do + ol];
            const double2 y = a.A[(size_t)c * Do * Do + (size_t)ol * Do + ow];
            v = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y + y.y));
        }
        a.Ar[e] = v;
    }
    for (int64_t e = gtid; e < (int64_t)a.B * Dm; e += gsz) {
        const int c = (int)(e / Dm), w = (int)(e % Dm);
        const CondCirc &cc = a.plan[c];
        double2 v = czero();
        if (w < cc.Dred) v = a.b[(size_t)c * Do + cc.red_to_orig[w]];
        a.br[e] = v;
        if (v.x != 0.0 || v.y != 0.0) nz = 1;
    }
    if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(&a.ctl->has_b, 1);
}

// ------------------------------------------------------------ step 1
// The zero-photon block (detected part 0): eq. (recrel) over the undetected
// sub-lattice, written from the pivot u - 1_w with w its first nonzero index.
// One block per circuit, level by level.  When the u-block fits, its values
// and levels are staged in the block's per-tile buffers (free during step 1),
// so a level reads the two below it from shared memory; otherwise it reads
// them from F.

// Strides and cutoffs of the u-block positions, copied to shared memory.
__device__ void stage_ubox(const CondCirc &cc, int *ust, int *ucu)
{
    __syncthreads();
    if (threadIdx.x < 2 * cc.nU) {
        ust[threadIdx.x] = cc.ustride[threadIdx.x];
        ucu[threadIdx.x] = cc.CU[threadIdx.x >> 1];
    }
    __syncthreads();
}

// Whether the u-block's values (16 B) and levels (1 B) fit the staging area.
__device__ __forceinline__ bool step1_staged(const CSmem &s, const CondCirc &cc)
{
    return cc.Lu < 256 && (size_t)cc.U2 * 17 <= s.s1_bytes;
}

template <bool SMEM>
__device__ __forceinline__ double2 ld_u(const double2 *p)
{
    if constexpr (SMEM) return *p;
    else return __ldcg(p);
}

// Digits of u (dig[0, tU)), their sum and the first nonzero position (tU: none).
__device__ __forceinline__ int u_digits(int u, int tU, const int *ust, const int *ucu, int *dig, int *first)
{
    int sum = 0, f0 = tU;
    for (int t = 0; t < tU; ++t) {
        dig[t] = (u / ust[t]) % ucu[t];
        sum += dig[t];
        if (f0 == tU && dig[t] > 0) f0 = t;
    }
    *first = f0;
    return sum;
}

// X: where the values live (shared staging area or F itself); lv: levels of
// the staged u-block (SMEM only).
template <bool SMEM>
__device__ void step1_forward_levels(const CondArgs &a, CSmem &s, int c, bool hb, double2 *X,
                                     const unsigned char *lv, const int *ust, const int *ucu)
{
    const CondCirc &cc = a.plan[c];
    double2 *F = a.F + cc.off_F;
    const int tU = 2 * cc.nU, Db = 2 * cc.dsh.M, U2 = cc.U2, Lu = cc.Lu, nU = cc.nU;
    for (int lev = 0; lev <= Lu; ++lev) {
        for (int u = threadIdx.x; u < U2; u += blockDim.x) {
            if (SMEM && lv[u] != lev) continue;
            int dig[2 * FK_MAXU], w;
            const int sum = u_digits(u, tU, ust, ucu, dig, &w);
            if (sum != lev) continue;
            double2 v;
            if (lev == 0) {
                v = a.c[c];
            } else {
                const int P = u - ust[w];
                double2 acc = hb ? cmul(s.br[Db + w], ld_u<SMEM>(X + (SMEM ? P : fpos(cc, 0, P)))) : czero();
                for (int t = 0; t < tU; ++t) {
                    const int Pt = dig[t] - (t == w ? 1 : 0);
                    if (Pt <= 0) continue;
                    const int r = P - ust[t];
                    acc = cfma(s.Ar[(Db + w) * a.Dmax + Db + t], ld_u<SMEM>(X + (SMEM ? r : fpos(cc, 0, r))), acc);
                }
                v = rscale(acc, s.inv[dig[w]]);
            }
            if (SMEM) X[u] = v;
            F[fpos(cc, 0, u)] = v;
            // output (ket, bra) of u and sqrt(prod u_t!)
            double f = 1.0;
            int ket = 0, bra = 0;
            for (int q = 0; q < nU; ++q) {
                const int uk = dig[2 * q], ub = dig[2 * q + 1];
                f *= s.sqf[uk] * s.sqf[ub];
                ket = ket * ucu[2 * q] + uk;
                bra = bra * ucu[2 * q] + ub;
            }
            a.rho[rpos(cc, (int64_t)ket * cc.NUo + bra)] = rscale(v, f);
        }
        __syncthreads();
    }
}

__device__ void step1_forward(const CondArgs &a, CSmem &s, int c, bool hb)
{
    __shared__ int ust[2 * FK_MAXU], ucu[2 * FK_MAXU];
    const CondCirc &cc = a.plan[c];
    load_circuit(a, s, c);
    stage_ubox(cc, ust, ucu);
    if (step1_staged(s, cc)) {
        const int tU = 2 * cc.nU, U2 = cc.U2;
        double2 *X = (double2 *)s.s1;
        unsigned char *lv = (unsigned char *)(X + U2);
        for (int u = threadIdx.x; u < U2; u += blockDim.x) {
            int dig[2 * FK_MAXU], f0;
            lv[u] = (unsigned char)u_digits(u, tU, ust, ucu, dig, &f0);
        }
        __syncthreads();
        step1_forward_levels<true>(a, s, c, hb, X, lv, ust, ucu);
    } else {
        step1_forward_levels<false>(a, s, c, hb, a.F + cc.off_F, nullptr, ust, ucu);
    }
}

// ------------------------------------------------------- tile bookkeeping
// kind: 0 = off-diagonal pivots AP(K), 1 = diagonal pivots DP, 2 = diagonal
// positions (reverse walk).  Per circuit: segments (K for AP) x pivots x
// u-chunks.
__device__ __forceinline__ unsigned seg_count(const CondArgs &a, const CondCirc &cc, int kind,
                                              int seg, int lev)
{
    const DiagShape &ds = cc.dsh;
    if (ds.M == 0 || lev >= ds.L + (kind == 2 ? 1 : 0)) return 0u;
    const LevelTab W = ltab(a, cc);
    if (kind == 0) return level_count(ds.C, W, seg, 1, lev);
    if (kind == 1) return level_count(ds.C, W, 0, 1, lev);
    return level_count(ds.C, W, 0, 0, lev);
}

__device__ int phase_tiles(const CondArgs &a, CSmem &s, int kind, int lev)
{
    __syncthreads();
    for (int c = threadIdx.x; c < a.B; c += blockDim.x) {
        const CondCirc &cc = a.plan[c];
        const int nseg = (kind == 0) ? cc.dsh.M : 1;
        int n = 0;
        for (int k = 0; k < nseg; ++k) n += (int)seg_count(a, cc, kind, k, lev) * cc.nchunk;
        s.ctiles[c + 1] = n;
    }
    __syncthreads();
    // prefix sums over the circuits by warp 0: each lane a contiguous run of
    // entries, then an exclusive scan of the runs' totals across the lanes
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, per = (a.B + 31) / 32;
        const int lo = 1 + lane * per, hi = min(lo + per, a.B + 1);
        int run = 0;
        for (int c = lo; c < hi; ++c) {
            run += s.ctiles[c];
            s.ctiles[c] = run;
        }
        int ex = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, ex, o);
            if (lane >= o) ex += v;
        }
        ex -= run;   // exclusive: the runs of the lanes before this one
        for (int c = lo; c < hi; ++c) s.ctiles[c] += ex;
        if (lane == 0) s.ctiles[0] = 0;
    }
    __syncthreads();
    return s.ctiles[a.B];
}

// Tiles [*t0, *t1) of a phase of nt tiles for this block: contiguous ranges,
// so the consecutive tiles of one circuit (numbered circuit-major) stay in
// one block and its A is loaded once per phase, not once per tile.
__device__ __forceinline__ void tile_range(int nt, int *t0, int *t1)
{
    *t0 = (int)((int64_t)nt * blockIdx.x / gridDim.x);
    *t1 = (int)((int64_t)nt * (blockIdx.x + 1) / gridDim.x);
}

struct CTile {
    int circ, seg, chunk;
    unsigned rank;
    unsigned pbase;     // pivots of the segments before seg in this phase of the circuit
};

__device__ CTile decode(const CondArgs &a, const CSmem &s, int kind, int lev, int tile)
{
    int lo = 0, hi = a.B - 1;
    while (lo < hi) {                      // last c with ctiles[c] <= tile
        const int mid = (lo + hi + 1) >> 1;
        if (s.ctiles[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    CTile t;
    t.circ = lo;
    const CondCirc &cc = a.plan[lo];
    int rem = tile - s.ctiles[lo];
    const int nseg = (kind == 0) ? cc.dsh.M : 1;
    int k = 0;
    unsigned pb = 0;
    for (; k < nseg; ++k) {
        const unsigned c = seg_count(a, cc, kind, k, lev);
        const int n = (int)c * cc.nchunk;
        if (rem < n) break;
        rem -= n;
        pb += c;
    }
    t.seg = k;
    t.pbase = pb;
    t.rank = (unsigned)(rem / cc.nchunk);
    t.chunk = rem % cc.nchunk;
    return t;
}

// ----------------------------------------------------- pivot geometry
__device__ PGeom ap_geom(const DiagShape &ds, const Dig &e, int K, const CSmem &s)
{
    PGeom g;
    g.ia = ds.off_ap[K] + box_index(ds, e, K, K, 1, -1, 0);
    const int M = ds.M;
    g.N = 2 * (M - K);
    g.row0 = 2 * K;
    const int eK = e(K);
    int64_t gd = 0;
    for (int i = K; i < M; ++i) gd += (int64_t)e(i) * ds.stride[i];
    const int64_t t2 = box_index(ds, e, K, K, 2, -1, 0);
    g.yP = ds.off_t1k[K] + box_index(ds, e, 0, 0, 1, K > 0 ? K : -1, 1);
    g.vmask = 1u | (eK >= 1 ? 2u : 0u);
    g.nmask = 2u | (eK <= ds.C[K] - 3 ? 1u : 0u);
    g.yr[0] = gd;
    g.yr[1] = ds.off_t2[K] + t2 - ds.stride[K];
    g.yw[0] = ds.off_t2[K] + t2;
    g.den[0] = eK + 2;
    g.yw[1] = gd + ds.stride[K];
    g.den[1] = eK + 1;
    double f = 1.0;
    for (int i = K; i < M; ++i) f *= s.fact[e(i)];
    g.fdiag = f * (double)(eK + 1);
    for (int m = K + 1; m < M; ++m) {
        const int j = 2 * (m - K);
        const int64_t ip = box_index(ds, e, K, K, 1, m, 1);
        const int em = e(m);
        g.yr[j] = ds.off_1001[K][m] + 2 * (ip - ds.stride[m]);   // P1010/P1001 interleaved
        g.yr[j + 1] = ds.off_1010[K][m] + 2 * (ip - ds.stride[m]);
        g.yw[j] = ds.off_1010[K][m] + 2 * ip;
        g.yw[j + 1] = ds.off_1001[K][m] + 2 * ip;
        g.den[j] = g.den[j + 1] = em + 1;
        if (em >= 1) g.vmask |= 3u << j;
        if (em <= ds.C[m] - 2) g.nmask |= 3u << j;
    }
    return g;
}

__device__ PGeom dp_geom(const DiagShape &ds, const Dig &d)
{
    PGeom g;
    const int M = ds.M;
    g.ia = 0;
    g.N = 2 * M;
    g.row0 = 0;
    g.fdiag = 0.0;
    int64_t gd = 0;
    for (int i = 0; i < M; ++i) gd += (int64_t)d(i) * ds.stride[i];
    g.yP = gd;
    g.vmask = g.nmask = 0;
    const int64_t t1b0 = box_index(ds, d, 0, 0, 2, -1, 0);
    for (int q = 0; q < M; ++q) {
        const int64_t iq = box_index(ds, d, 0, 0, 1, q > 0 ? q : -1, 1);
        const int64_t ib = (q == 0) ? t1b0 : iq;
        const int dq = d(q);
        g.yr[2 * q] = ds.off_t1b[q] + ib - ds.stride[q];
        g.yr[2 * q + 1] = ds.off_t1k[q] + iq - ds.stride[q];
        g.yw[2 * q] = ds.off_t1k[q] + iq;
        g.yw[2 * q + 1] = ds.off_t1b[q] + ib;
        g.den[2 * q] = g.den[2 * q + 1] = dq + 1;
        if (dq >= 1) g.vmask |= 3u << (2 * q);
        if (q == 0) {
            g.nmask |= 1u;
            if (dq <= ds.C[0] - 3) g.nmask |= 2u;
        } else if (dq <= ds.C[q] - 2) {
            g.nmask |= 3u << (2 * q);
        }
    }
    return g;
}

// Column j of the pivot's matrix -> index in the reduced lattice.
__device__ __forceinline__ int col_index(const PGeom &g, int Db, int j)
{
    return j < g.N ? g.row0 + j : Db + (j - g.N);
}

// Record of pivot `rank` of segment `seg` of phase (kind, lev) in circuit c's
// geometry table: AP pivots of every level first, then DP pivots.
__device__ __forceinline__ int64_t geo_index(const CondArgs &a, const CondCirc &cc, int kind, int lev,
                                             unsigned pbase, unsigned rank)
{
    const unsigned *pre = a.Wall + cc.gp_off;
    return cc.geo_off + (int64_t)pre[kind * (cc.dsh.L + 1) + lev] + pbase + rank;
}

// The pivot geometry of every circuit, once per launch: one block per
// (circuit, kind, level), a thread per pivot of each segment.
__device__ void build_geo(const CondArgs &a, const CSmem &s)
{
    const int nitem = a.B * 2 * a.Lmax;
    for (int it = blockIdx.x; it < nitem; it += gridDim.x) {
        const int c = it / (2 * a.Lmax), kind = (it / a.Lmax) & 1, lev = it % a.Lmax;
        const CondCirc &cc = a.plan[c];
        const DiagShape &ds = cc.dsh;
        if (ds.M == 0 || lev >= ds.L) continue;
        const LevelTab W = ltab(a, cc);
        unsigned pb = 0;
        const int nseg = kind == 0 ? ds.M : 1;
        for (int k = 0; k < nseg; ++k) {
            const unsigned cnt = seg_count(a, cc, kind, k, lev);
            for (unsigned r = threadIdx.x; r < cnt; r += blockDim.x) {
                const Dig e = unrank(ds.C, ds.M, W, kind == 0 ? k : 0, 1, lev, r);
                a.geo[geo_index(a, cc, kind, lev, pb, r)] = kind == 0 ? ap_geom(ds, e, k, s) : dp_geom(ds, e);
            }
            pb += cnt;
        }
    }
}

// The current tile's pivot geometry (shared by every thread of the tile).
__device__ __forceinline__ const PGeom &tile_geometry(const CondArgs &a, const CTile &tl, int kind, int lev)
{
    const CondCirc &cc = a.plan[tl.circ];
    return a.geo[geo_index(a, cc, kind, lev, tl.pbase, tl.rank)];
}

// -------------------------------------------------------------- forward
// One (pivot, u) pair per thread: rows = detected writes, columns = detected
// reads then undetected reads, plus the b-term on the pivot value.  Gauss's
// three-multiplication complex product (A in the planes Re A, Re A + Im A,
// Im A - Re A; reads as Re x, Im x, Re x + Im x): three DFMA per term.
template <bool HASB>
__device__ void pair_forward(const CondArgs &a, CSmem &s, const CTile &tl, int kind, int lev)
{
    const CondCirc &cc = a.plan[tl.circ];
    const DiagShape &ds = cc.dsh;
    load_circuit(a, s, tl.circ);
    const PGeom &g = tile_geometry(a, tl, kind, lev);
    const int t = threadIdx.x, Dm = a.Dmax;
    const int u = tl.chunk * TPB + t;
    const bool act = u < cc.U2;
    const int Db = 2 * ds.M, tU = 2 * cc.nU, N = g.N, NC = N + tU, row0 = g.row0;
    const unsigned vmask = g.vmask, nm = g.nmask;   // uniform: every thread of the tile shares the pivot
    const int64_t yP = g.yP;
    const double2 *F = a.F + cc.off_F;
    unsigned umask = 0;
    double2 PV = czero();
    if (act) {
        for (int j = 0; j < N; ++j)
            put3(s.R3, Dm, j, t, ((vmask >> j) & 1u) ? __ldcg(F + fpos(cc, g.yr[j], u)) : czero());
        for (int q = 0; q < tU; ++q) {
            double2 v = czero();
            if (udigit(cc, u, q) >= 1) {
                umask |= 1u << q;
                v = __ldcg(F + fpos(cc, yP, u - cc.ustride[q]));
            }
            put3(s.R3, Dm, N + q, t, v);
        }
        if (HASB) PV = __ldcg(F + fpos(cc, yP, u));
    } else {
        for (int j = 0; j < NC; ++j) put3(s.R3, Dm, j, t, czero());
    }
    const unsigned cm = __reduce_or_sync(0xffffffffu, act ? (vmask | (umask << N)) : 0u);
    double2 *Fw = a.F + cc.off_F;
    const size_t DD = (size_t)Dm * Dm;
    const double *Ar = s.A3, *Ap = s.A3 + DD, *Am = s.A3 + 2 * DD;
    constexpr int CH = 8;
    for (int i0 = 0; i0 < N; i0 += CH) {
        if (((nm >> i0) & 0xffu) == 0) continue;
        double p1[CH], p2[CH], p3[CH];
#pragma unroll
        for (int ii = 0; ii < CH; ++ii) p1[ii] = p2[ii] = p3[ii] = 0.0;
        for (int j = 0; j < NC; ++j) {
            if (!((cm >> j) & 1u)) continue;
            const double xr = pl(s.R3, Dm, 0, j, t), xi = pl(s.R3, Dm, 1, j, t), xs = pl(s.R3, Dm, 2, j, t);
            const int cj = col_index(g, Db, j);
#pragma unroll
            for (int ii = 0; ii < CH; ++ii)
                if (i0 + ii < N && ((nm >> (i0 + ii)) & 1u)) {
                    const size_t o = (size_t)(row0 + i0 + ii) * Dm + cj;
                    p1[ii] = fma(Ar[o], xs, p1[ii]);
                    p2[ii] = fma(Ap[o], xi, p2[ii]);
                    p3[ii] = fma(Am[o], xr, p3[ii]);
                }
        }
        if (!act) continue;
#pragma unroll
        for (int ii = 0; ii < CH; ++ii) {
            const int i = i0 + ii;
            if (i < N && ((nm >> i) & 1u)) {
                double2 acc = make_double2(p1[ii] - p2[ii], p1[ii] + p3[ii]);
                if (HASB) acc = cadd(acc, cmul(s.br[row0 + i], PV));
                const double2 v = rscale(acc, s.inv[g.den[i]]);
                Fw[fpos(cc, g.yw[i], u)] = v;
                if (kind == 0 && i == 1) {          // a diagonal of the detected modes
                    int ket, bra;
                    const double f = uscale(cc, s, u, &ket, &bra) * g.fdiag;
                    a.rho[rpos(cc, (g.yw[1] * cc.NUo + ket) * cc.NUo + bra)] = rscale(v, f);
                }
            }
        }
    }
}

// ------------------------------------------------------ tensor-core engine
// The same sums on the fp16 tensor cores as in the all-detected walk
// (walk_digits.cuh: exact base-256 digit products, recombined in int64).  A
// tile is one pivot and 128 points u of its u-block; a warp takes 32 of
// them.  The pivot's reads are the reduced indices [row0, Dred) -- detected
// reads from row0, undetected ones from Db = row0 + N on -- and its writes
// the rows [row0, Db), so one digit image of the real form R of each
// circuit's reduced A (row 2i: Re A_ij at column 2j, -Im A_ij at 2j + 1;
// row 2i + 1: Im A_ij, Re A_ij), padded to 16 KS x 16 KS, serves every
// pivot: the products use the aligned 16 x 16 tiles of R that these rows and
// columns meet, with zeros for the inputs outside.

// Entry (w, l) of the augmented symmetric matrix [[A_s, b], [b^T, 0]] of
// circuit c on the reduced indices, index Dred standing for the pivot value
// (the arithmetic of the prologue's copies of A_s and b).
__device__ __forceinline__ double2 red_entry(const CondArgs &a, const CondCirc &cc, int c, int w, int l)
{
    const int Do = a.D_orig, Dr = cc.Dred;
    if (w == Dr && l == Dr) return czero();
    if (w == Dr || l == Dr) return a.b[(size_t)c * Do + cc.red_to_orig[w == Dr ? l : w]];
    const int ow = cc.red_to_orig[w], ol = cc.red_to_orig[l];
    const double2 x = a.A[(size_t)c * Do * Do + (size_t)ow * Do + ol];
    const double2 y = a.A[(size_t)c * Do * Do + (size_t)ol * Do + ow];
    return make_double2(0.5 * (x.x + y.x), 0.5 * (x.y + y.y));
}

// Digit fragments of every circuit's augmented R (one block per circuit):
// the row exponent fields (largest over the complex row) first, then the
// seven digit planes in the register order of the A operand of mma
// m16n8k16.  With b folded in as the column (and row) of the pivot value,
// the forward's b-term b_w G_P and the reverse walk's pivot-value adjoint
// sum_w conj(b_w) ybar_w come out of the same exact products.
template <int KS>
__device__ void build_cond_digits(const CondArgs &a, CSmem &s)
{
    constexpr int P = 16 * KS;
    for (int c = blockIdx.x; c < a.B; c += gridDim.x) {
        const CondCirc &cc = a.plan[c];
        const int Dr = cc.Dred + 1;   // augmented
        int *gA = (int *)(a.dig + (size_t)c * kDigBytes);
        uint32_t *Af = (uint32_t *)(a.dig + (size_t)c * kDigBytes + 256);
        __syncthreads();
        for (int r = threadIdx.x; r < P; r += blockDim.x) s.fA[r] = 0;
        __syncthreads();
        for (int e = threadIdx.x; e < Dr * Dr; e += blockDim.x) {
            const double2 v = red_entry(a, cc, c, e / Dr, e % Dr);
            const int f = max(fexp(v.x), fexp(v.y));
            if (f != 0) atomicMax(&s.fA[2 * (e / Dr)], f);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < Dr; i += blockDim.x) s.fA[2 * i + 1] = s.fA[2 * i];
        __syncthreads();
        for (int r = threadIdx.x; r < P; r += blockDim.x) gA[r] = s.fA[r];
        for (int e = threadIdx.x; e < P * P / 2; e += blockDim.x) {
            const int r = e / (P / 2), col = 2 * (e % (P / 2));
            uint32_t wd[kNDig];
            if (r < 2 * Dr && col < 2 * Dr) {
                const double2 v = red_entry(a, cc, c, r >> 1, col >> 1);
                const double x0 = (r & 1) ? v.y : v.x, x1 = (r & 1) ? v.x : -v.y;
                digit_words(to_fixed(x0, s.fA[r]), to_fixed(x1, s.fA[r]), wd);
            } else {
#pragma unroll
                for (int sl = 0; sl < kNDig; ++sl) wd[sl] = 0u;
            }
            const int rr = r & 15, cl = col & 15;
            const int lane = (rr & 7) * 4 + ((cl & 7) >> 1), k = (rr >> 3) | ((cl >> 3) << 1);
            const int tile = (r >> 4) * KS + (col >> 4);
#pragma unroll
            for (int sl = 0; sl < kNDig; ++sl) Af[(((tile * kNDig + sl) * 32 + lane) << 2) + k] = wd[sl];
        }
    }
    __syncthreads();
    s.loaded = -1;
}

// out[r][p] = sum_{c < ncol} R[2 row0 + r][2 row0 + c] in[c][p] for the 32
// pairs p of this warp and real rows r < nrow (CONJ: with conj(A), whose
// real form flips the sign of the Im A digits); in and out are the warp's
// buffers (row = real index relative to 2 row0, column = lane) and may
// alias: an N tile is read before its products land.
template <int KS, bool CONJ>
__device__ __forceinline__ void cond_products(const CSmem &s, int row0, int nrow, int ncol, double *in,
                                              double *out)
{
    const int lane = threadIdx.x & 31, grp = lane >> 2, tig = lane & 3;
    const int r0 = 2 * row0;
    const int m0 = r0 >> 4, m1 = (r0 + nrow + 15) >> 4;   // M tiles (output rows)
    const int k0 = r0 >> 4, k1 = (r0 + ncol + 15) >> 4;   // K tiles (input rows)
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
                const bool ok = ks >= k0 && ks < k1 && c >= 0 && c < ncol;
                xv[ks][h][0] = ok ? in[c * kCWBS + p] : 0.0;
                xv[ks][h][1] = ok ? in[(c + 1) * kCWBS + p] : 0.0;
                fm = max(fm, max(fexp(xv[ks][h][0]), fexp(xv[ks][h][1])));
            }
        fm = max(fm, __shfl_xor_sync(0xffffffffu, fm, 1));
        fm = max(fm, __shfl_xor_sync(0xffffffffu, fm, 2));
        // an N tile whose inputs all count as zero (points past the u-block's
        // end) has zero products: write them without the MMAs
        if (!__any_sync(0xffffffffu, fm >= 26)) {
            for (int r = tig; r < nrow; r += 4) out[r * kCWBS + p] = 0.0;
            continue;
        }
        uint32_t bq[kNDig][KS][2];
#pragma unroll
        for (int ks = 0; ks < KS; ++ks)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t wd[kNDig];
                digit_words(to_fixed(xv[ks][h][0], fm), to_fixed(xv[ks][h][1], fm), wd);
#pragma unroll
                for (int sl = 0; sl < kNDig; ++sl) bq[sl][ks][h] = wd[sl];
            }
        __syncwarp();   // every lane has read this N tile's inputs
        const int fx0 = __shfl_sync(0xffffffffu, fm, 8 * tig) - 2096;
        const int fx1 = __shfl_sync(0xffffffffu, fm, 8 * tig + 4) - 2096;
#pragma unroll 1
        for (int mt = m0; mt < m1; ++mt) {
            float acc[kNDig][4];
#pragma unroll
            for (int d = 0; d < kNDig; ++d)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[d][q] = 0.f;
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                if (ks < k0 || ks >= k1) continue;
#pragma unroll
                for (int sa = 0; sa < kNDig; ++sa) {
                    const uint4 f = Af[((mt * KS + ks) * kNDig + sa) * 32];
                    const uint32_t af[4] = {f.x ^ cflip, f.y ^ cflip, f.z ^ cflip, f.w ^ cflip};
#pragma unroll
                    for (int u = 0; u + sa < kNDig; ++u) mma_f16(acc[sa + u], af, bq[u][ks]);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int ra = 16 * mt + grp + 8 * (q >> 1), r = ra - r0;
                const int pc = nt * 8 + 2 * tig + (q & 1);
                if (r >= 0 && r < nrow) {
                    // up to 7 x 16 KS x 2^14 per diagonal: below 2^22 for KS <= 2
                    const long long Y = KS > 2 ? combine_digits_wide(acc, q) : combine_digits(acc, q);
                    out[r * kCWBS + pc] = scale2(__ll2double_rn(Y), s.fA[ra] + ((q & 1) ? fx1 : fx0));
                }
            }
        }
    }
    __syncwarp();
}

// Partial dL/dA of this warp's 32 pairs, P[w][j] = sum_t Y_w(t) conj(X_j(t))
// for rows w < N and read columns j < NC (reduced indices row0 + w and
// row0 + j), on six-digit products (the reading of the all-detected walk's
// partial pass): each pair's reads are scaled by 2^(1022 - e_t) and its
// adjoints by the inverse, and the adjoints share one power of two per row
// over the warp.  The matrices are small here (N <= 2 Md rows), so the real
// parts go into the MMA's M and N dimensions and the pairs into K: rows
// (w, Re/Im of Y) = the warp buffer's rows of Y, columns (j, Re/Im of X) =
// its rows of X, K = 16 pairs per MMA.  Re P = Yr Xr + Yi Xi and
// Im P = Yi Xr - Yr Xi then join the accumulators of lanes 4 apart (the
// Re/Im rows of one w), exactly in int64.  Each diagonal sums at most
// 6 x 32 products below 2^14, so the fp32 accumulators stay below 2^22.
// The result is added to the warp's own slot (single writer, fixed order).
template <int KS>
__device__ void cond_partials(const CondArgs &a, const CSmem &s, int circ, int row0, int N, int NC)
{
    constexpr int NDP = 6, NT = 2 * KS;   // N tiles of 8 real columns (2 NC <= 16 KS)
    const int lane = threadIdx.x & 31, grp = lane >> 2, tig = lane & 3, warp = threadIdx.x >> 5;
    const int Dm = a.Dmax, nmt = (2 * N + 15) >> 4, nnt = (2 * NC + 7) >> 3;
    const double *wx = s.wx + (size_t)warp * 16 * KS * kCWBS;
    const double *wy = s.wy + (size_t)warp * 16 * KS * kCWBS;
    const int *ef = s.wf + warp * 32;
    const int *gy = s.wg + warp * 32;
    const size_t slot = (size_t)blockIdx.x * a.spb + warp;
    double *pA = (double *)(a.partA + ((size_t)circ * a.slots + slot) * Dm * Dm);
    const int ri = grp & 1;   // Re (0) or Im (1) part of Y on this lane's rows
#pragma unroll 1
    for (int mt = 0; mt < nmt; ++mt) {
        float acc[NDP][NT][4];
#pragma unroll
        for (int d = 0; d < NDP; ++d)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[d][nt][q] = 0.f;
        // this lane's rows of Y: real rows ra0 = 16 mt + grp and ra1 = ra0 + 8
        const int ra0 = 16 * mt + grp, ra1 = ra0 + 8;
        const int w0 = ra0 >> 1, w1 = ra1 >> 1;
        const int g0 = w0 < N ? gy[w0] : 0, g1 = w1 < N ? gy[w1] : 0;
#pragma unroll 1
        for (int ks = 0; ks < 2; ++ks) {
            // pairs of the k-step: 16 ks + 2 tig (+1) and 16 ks + 2 tig + 8 (+1)
            const int tA = 16 * ks + 2 * tig, tB = tA + 8;
            const int eA0 = ef[tA], eA1 = ef[tA + 1], eB0 = ef[tB], eB1 = ef[tB + 1];
            uint32_t aq[NDP][4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                // A operand registers: k bit 0 = row half, bit 1 = K half
                const int ra = (k & 1) ? ra1 : ra0, w = (k & 1) ? w1 : w0, g = (k & 1) ? g1 : g0;
                const int t = (k & 2) ? tB : tA;
                const int e0 = (k & 2) ? eB0 : eA0, e1 = (k & 2) ? eB1 : eA1;
                double y0 = 0.0, y1 = 0.0;
                if (w < N && g != 0) {
                    if (e0 != 0) y0 = wy[ra * kCWBS + t];
                    if (e1 != 0) y1 = wy[ra * kCWBS + t + 1];
                }
                uint32_t wd[NDP];
                digit_words<NDP>(to_fixed_rel<NDP>(y0, g - e0 + 1022), to_fixed_rel<NDP>(y1, g - e1 + 1022), wd);
#pragma unroll
                for (int sl = 0; sl < NDP; ++sl) aq[sl][k] = wd[sl];
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                if (nt >= nnt) continue;
                const int n = 8 * nt + grp;   // B column = real row of X
                uint32_t bq[NDP][2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int t = h ? tB : tA;
                    const int e0 = h ? eB0 : eA0, e1 = h ? eB1 : eA1;
                    double x0 = 0.0, x1 = 0.0;
                    if (n < 2 * NC) {
                        x0 = wx[n * kCWBS + t];
                        x1 = wx[n * kCWBS + t + 1];
                    }
                    uint32_t wd[NDP];
                    digit_words<NDP>(to_fixed<NDP>(x0, e0), to_fixed<NDP>(x1, e1), wd);
#pragma unroll
                    for (int sl = 0; sl < NDP; ++sl) bq[sl][h] = wd[sl];
                }
#pragma unroll
                for (int u = 0; u < NDP; ++u)
#pragma unroll
                    for (int sa = 0; sa + u < NDP; ++sa) mma_f16(acc[sa + u][nt], aq[sa], bq[u]);
            }
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            if (nt >= nnt) continue;
            const int j = 4 * nt + tig;   // columns 2 tig (Re X) and 2 tig + 1 (Im X) of the tile
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int w = h ? w1 : w0, g = h ? g1 : g0;
                float t6[NDP][4];
#pragma unroll
                for (int d = 0; d < NDP; ++d) {
                    t6[d][0] = acc[d][nt][2 * h];
                    t6[d][1] = acc[d][nt][2 * h + 1];
                }
                const long long v0 = combine_digits<NDP>(t6, 0);   // Y_ri X_re
                const long long v1 = combine_digits<NDP>(t6, 1);   // Y_ri X_im
                // the other part of Y of the same w sits on the lane 4 apart
                const long long o1 = __shfl_xor_sync(0xffffffffu, v1, 4);
                const long long y = ri ? v0 - o1 : v0 + o1;   // Im P = Yi Xr - Yr Xi, Re P = Yr Xr + Yi Xi
                if (w < N && j < NC && g >= 26) {
                    // reductions without return into the warp's own slot; Y
                    // carries the product of the two fixed points over 2^48
                    double *dst = pA + 2 * ((size_t)(row0 + w) * Dm + row0 + j) + ri;
                    atomicAdd(dst, scale2(__ll2double_rn(y), g - 1074 + 8 * (kNDig - NDP)));
                }
            }
        }
    }
}

// Forward tile on the tensor engine: the pairs' reads into the warp's
// buffer, the products in place, each lane writes its pair's rows.
template <int KS, bool HASB>
__device__ void pair_forward_tc(const CondArgs &a, CSmem &s, const CTile &tl, int kind, int lev)
{
    const CondCirc &cc = a.plan[tl.circ];
    load_circuit(a, s, tl.circ);
    const PGeom &g = tile_geometry(a, tl, kind, lev);
    const int t = threadIdx.x, lane = t & 31;
    const int u = tl.chunk * TPB + t;
    const bool act = u < cc.U2;
    const int tU = 2 * cc.nU, N = g.N, NC = N + tU, row0 = g.row0;
    const unsigned vmask = g.vmask, nm = g.nmask;
    const int64_t yP = g.yP;
    const double2 *F = a.F + cc.off_F;
    double *wb = s.wx + (size_t)(t >> 5) * 16 * KS * kCWBS + lane;
    double2 PV = czero();
    if (act) {
        double2 v[8 * KS];
#pragma unroll
        for (int j = 0; j < 8 * KS; ++j) {
            v[j] = czero();
            if (j < N) {
                if ((vmask >> j) & 1u) v[j] = __ldcg(F + fpos(cc, g.yr[j], u));
            } else if (j < NC) {
                const int q = j - N;
                if (udigit(cc, u, q) >= 1) v[j] = __ldcg(F + fpos(cc, yP, u - cc.ustride[q]));
            }
        }
        if (HASB) PV = __ldcg(F + fpos(cc, yP, u));
#pragma unroll
        for (int j = 0; j < 8 * KS; ++j)
            if (j < NC) {
                wb[(2 * j) * kCWBS] = v[j].x;
                wb[(2 * j + 1) * kCWBS] = v[j].y;
            }
    } else {
        for (int j = 0; j < NC; ++j) wb[(2 * j) * kCWBS] = wb[(2 * j + 1) * kCWBS] = 0.0;
    }
    // the pivot value as the read of column Dred (b in the augmented matrix)
    wb[(2 * NC) * kCWBS] = PV.x;
    wb[(2 * NC + 1) * kCWBS] = PV.y;
    __syncwarp();
    double *wbw = s.wx + (size_t)(t >> 5) * 16 * KS * kCWBS;
    cond_products<KS, false>(s, row0, 2 * N, 2 * (NC + 1), wbw, wbw);
    if (act) {
        double2 *Fw = a.F + cc.off_F;
        for (int i = 0; i < N; ++i) {
            if (!((nm >> i) & 1u)) continue;
            const double2 acc = make_double2(wb[(2 * i) * kCWBS], wb[(2 * i + 1) * kCWBS]);
            const double2 val = rscale(acc, s.inv[g.den[i]]);
            Fw[fpos(cc, g.yw[i], u)] = val;
            if (kind == 0 && i == 1) {          // a diagonal of the detected modes
                int ket, bra;
                const double f = uscale(cc, s, u, &ket, &bra) * g.fdiag;
                a.rho[rpos(cc, (g.yw[1] * cc.NUo + ket) * cc.NUo + bra)] = rscale(val, f);
            }
        }
    }
    __syncwarp();
}

// Reverse tile on the tensor engine: reads and scaled output adjoints into
// the warp's buffers; the warp's partial dL/dA (digits) and dL/db (FP64);
// the detected read adjoints conj(A)^T Y in place; the pivot position pulls
// its adjoint from this u (b-term) and from u + 1_t (FP64) as in the FP64
// engine.
template <int KS, bool HASB>
__device__ void pair_reverse_tc(const CondArgs &a, CSmem &s, const CTile &tl, int kind, int lev)
{
    const CondCirc &cc = a.plan[tl.circ];
    const DiagShape &ds = cc.dsh;
    load_circuit(a, s, tl.circ);
    const PGeom &g = tile_geometry(a, tl, kind, lev);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int u = tl.chunk * TPB + t;
    const bool act = u < cc.U2;
    const int Db = 2 * ds.M, tU = 2 * cc.nU, N = g.N, NC = N + tU, Dm = a.Dmax, row0 = g.row0;
    const unsigned vmask = g.vmask, nm = g.nmask;
    const int64_t yP = g.yP;
    const double2 *F = a.F + cc.off_F;
    double2 *Fb = a.Fbar + cc.off_F;
    double *wxl = s.wx + (size_t)warp * 16 * KS * kCWBS + lane;
    double *wyl = s.wy + (size_t)warp * 16 * KS * kCWBS + lane;
    unsigned upmask = 0;
    int fx = 0;
    double2 FPv = czero();
    if (act) {
        double2 v[8 * KS];
#pragma unroll
        for (int j = 0; j < 8 * KS; ++j) {
            v[j] = czero();
            if (j < N) {
                if ((vmask >> j) & 1u) v[j] = __ldcg(F + fpos(cc, g.yr[j], u));
            } else if (j < NC) {
                const int q = j - N, dq = udigit(cc, u, q);
                if (dq >= 1) v[j] = __ldcg(F + fpos(cc, yP, u - cc.ustride[q]));
                if (dq + 1 < cc.CU[q >> 1]) upmask |= 1u << q;
            }
        }
        double2 y[8 * KS];
#pragma unroll
        for (int i = 0; i < 8 * KS; ++i) {
            y[i] = czero();
            if (i < N && ((nm >> i) & 1u)) y[i] = rscale(__ldcg(Fb + fpos(cc, g.yw[i], u)), s.inv[g.den[i]]);
        }
        if (HASB) FPv = __ldcg(F + fpos(cc, yP, u));
#pragma unroll
        for (int j = 0; j < 8 * KS; ++j)
            if (j < NC) {
                fx = max(fx, max(fexp(v[j].x), fexp(v[j].y)));
                wxl[(2 * j) * kCWBS] = v[j].x;
                wxl[(2 * j + 1) * kCWBS] = v[j].y;
            }
#pragma unroll
        for (int i = 0; i < 8 * KS; ++i)
            if (i < N) {
                wyl[(2 * i) * kCWBS] = y[i].x;
                wyl[(2 * i + 1) * kCWBS] = y[i].y;
            }
    } else {
        for (int j = 0; j < NC; ++j) wxl[(2 * j) * kCWBS] = wxl[(2 * j + 1) * kCWBS] = 0.0;
        for (int i = 0; i < N; ++i) wyl[(2 * i) * kCWBS] = wyl[(2 * i + 1) * kCWBS] = 0.0;
    }
    if (HASB) s.FP[t] = FPv;
    // row exponents of the partial dL/dA: for row w the largest exponent
    // field of Y_w(t) 2^(e_t - 1022) over the warp's pairs (0: none)
    s.wf[t] = fx;
    for (int w = 0; w < N; ++w) {
        int gw = 0;
        if (fx != 0) {
            const int fy = max(fexp(wyl[(2 * w) * kCWBS]), fexp(wyl[(2 * w + 1) * kCWBS]));
            if (fy != 0) gw = max(fy + fx - 1022, 0);
        }
        gw = __reduce_max_sync(0xffffffffu, gw);
        if (lane == 0) s.wg[warp * 32 + w] = gw;
    }
    __syncwarp();
    cond_partials<KS>(a, s, tl.circ, row0, N, NC);
    if (HASB) {
        // dL/db partial of the warp: sum_t conj(P(t)) Y_w(t), lanes over rows
        double2 *pb = a.partb + ((size_t)tl.circ * a.slots + (size_t)blockIdx.x * a.spb + warp) * Dm;
        const double *wyw = s.wy + (size_t)warp * 16 * KS * kCWBS;
        for (int w = lane; w < N; w += 32) {
            double2 acc = czero();
            for (int tt = 0; tt < 32; ++tt)
                acc = cfma_conj(s.FP[warp * 32 + tt], make_double2(wyw[(2 * w) * kCWBS + tt], wyw[(2 * w + 1) * kCWBS + tt]),
                                acc);
            atomicAdd(&pb[row0 + w].x, acc.x);   // one writer, ordered by the warp's barriers
            atomicAdd(&pb[row0 + w].y, acc.y);
        }
    }
    __syncwarp();
    // conj(M)^T Y on the augmented matrix, rows [row0, Dred]: the detected
    // read adjoints (j < N), the values this pair sends to the pivot
    // positions u - 1_t through its undetected reads (N <= j < NC), and the
    // b-term of its own pivot-value adjoint (j = NC)
    double *wyw = s.wy + (size_t)warp * 16 * KS * kCWBS;
    cond_products<KS, true>(s, row0, 2 * (NC + 1), 2 * N, wyw, wyw);
    __syncthreads();   // the tile's products are visible to every warp
    if (act) {
        double2 pv = make_double2(wyl[(2 * NC) * kCWBS], wyl[(2 * NC + 1) * kCWBS]);
        for (int j = 0; j < N; ++j) {
            if (!((vmask >> j) & 1u)) continue;
            const double2 acc = make_double2(wyl[(2 * j) * kCWBS], wyl[(2 * j + 1) * kCWBS]);
            if (kind == 0 && j == 0) {
                a.scratch[spos(cc, g.ia, u)] = acc;
            } else {
                double2 *dst = Fb + fpos(cc, g.yr[j], u);
                *dst = cadd(__ldcg(dst), acc);
            }
        }
        // the pivot position (u, P) pulls from the pairs u + 1_t: from the
        // tile's products when that pair is in the tile, else in FP64
        for (int q = 0; q < tU; ++q) {
            if (!((upmask >> q) & 1u)) continue;
            const int tn = t + cc.ustride[q];
            if (tn < TPB) {
                const double *src = s.wy + (size_t)(tn >> 5) * 16 * KS * kCWBS + (tn & 31);
                pv = cadd(pv, make_double2(src[(2 * (N + q)) * kCWBS], src[(2 * (N + q) + 1) * kCWBS]));
                continue;
            }
            const int un = u + cc.ustride[q];
            for (int i = 0; i < N; ++i) {
                if (!((nm >> i) & 1u)) continue;
                const double2 yn = rscale(__ldcg(Fb + fpos(cc, g.yw[i], un)), s.inv[g.den[i]]);
                pv = cfma_conj(s.Ar[(row0 + i) * Dm + Db + q], yn, pv);
            }
        }
        double2 *dst = Fb + fpos(cc, yP, u);
        *dst = cadd(__ldcg(dst), pv);
    }
    __syncthreads();   // every warp has read the buffers before the next tile
}

// KS = 0: the FP64 engine; KS = 1..3: the tensor engine with 16 KS real rows.
template <int KS>
__global__ void __launch_bounds__(TPB, (KS == 1 ? 4 : 1)) cond_forward_kernel(const __grid_constant__ CondArgs a)
{
    FK_DBG_BEGIN(a.ctl);
    if (skip_walk(a.ctl)) return;   // the input scan found a NaN or Inf
    CSmem s = carve(a, false, KS);
    build_tables(s);
    prologue(a);
    build_geo(a, s);
    if constexpr (KS > 0) build_cond_digits<KS>(a, s);
    if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
    const bool hb = *(volatile int *)&a.ctl->has_b != 0;
    for (int c = blockIdx.x; c < a.B; c += gridDim.x) step1_forward(a, s, c, hb);
    if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
    for (int lev = 0; lev < a.Lmax; ++lev) {
        for (int kind = 1; kind >= 0; --kind) {     // diagonal pivots, then off-diagonal
            const int nt = phase_tiles(a, s, kind, lev);
            int t0, t1;
            tile_range(nt, &t0, &t1);
            for (int tile = t0; tile < t1; ++tile) {
                const CTile tl = decode(a, s, kind, lev, tile);
                if constexpr (KS > 0) {
                    if (hb) pair_forward_tc<KS, true>(a, s, tl, kind, lev);
                    else pair_forward_tc<KS, false>(a, s, tl, kind, lev);
                } else {
                    if (hb) pair_forward<true>(a, s, tl, kind, lev);
                    else pair_forward<false>(a, s, tl, kind, lev);
                }
            }
            if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
        }
    }
}

// -------------------------------------------------------------- reverse
// Per (pivot, u): scaled output adjoints ybar_i = Fbar(u, y_i) / (P_w + 1);
// detected reads get conj(A)^T ybar (each is read by exactly one (pivot, u),
// except the diagonal read of an off-diagonal pivot, which goes to scratch);
// the pivot position (u, P) pulls its adjoint from this u (b-term) and from
// u + 1_t (undetected reads of the neighbours), so no two threads write one
// location; dL/dA and dL/db are reduced over the tile into block partials.
template <bool HASB>
__device__ void pair_reverse(const CondArgs &a, CSmem &s, const CTile &tl, int kind, int lev)
{
    const CondCirc &cc = a.plan[tl.circ];
    const DiagShape &ds = cc.dsh;
    load_circuit(a, s, tl.circ);
    const PGeom &g = tile_geometry(a, tl, kind, lev);
    const int t = threadIdx.x;
    const int u = tl.chunk * TPB + t;
    const bool act = u < cc.U2;
    const int Db = 2 * ds.M, tU = 2 * cc.nU, N = g.N, NC = N + tU, Dm = a.Dmax, row0 = g.row0;
    const unsigned vmask = g.vmask, nm = g.nmask;
    const int64_t yP = g.yP;
    const double2 *F = a.F + cc.off_F;
    double2 *Fb = a.Fbar + cc.off_F;
    unsigned upmask = 0;
    if (act) {
        for (int j = 0; j < N; ++j)
            put3(s.R3, Dm, j, t, ((vmask >> j) & 1u) ? __ldcg(F + fpos(cc, g.yr[j], u)) : czero());
        for (int q = 0; q < tU; ++q) {
            const int dq = udigit(cc, u, q);
            double2 v = czero();
            if (dq >= 1) v = __ldcg(F + fpos(cc, yP, u - cc.ustride[q]));
            if (dq + 1 < cc.CU[q >> 1]) upmask |= 1u << q;
            put3(s.R3, Dm, N + q, t, v);
        }
        for (int i = 0; i < N; ++i)
            put3(s.Y3, Dm, i, t, ((nm >> i) & 1u) ? rscale(__ldcg(Fb + fpos(cc, g.yw[i], u)), s.inv[g.den[i]])
                                                   : czero());
        s.FP[t] = HASB ? __ldcg(F + fpos(cc, yP, u)) : czero();
    } else {
        for (int j = 0; j < NC; ++j) put3(s.R3, Dm, j, t, czero());
        for (int i = 0; i < N; ++i) put3(s.Y3, Dm, i, t, czero());
        s.FP[t] = czero();
    }
    // detected reads: Rbar_j = sum_i conj(A_{w_i l_j}) y_i, with y = yr + i yi,
    // ys = yr + yi:  Re = sum Ar ys + sum (Ai - Ar) yi,  Im = sum Ar ys - sum (Ar + Ai) yr
    const size_t DD = (size_t)Dm * Dm;
    const double *Ar = s.A3, *Ap = s.A3 + DD, *Am = s.A3 + 2 * DD;
    constexpr int CH = 8;
    for (int j0 = 0; j0 < N; j0 += CH) {
        if (((vmask >> j0) & 0xffu) == 0) continue;
        double p1[CH], q2[CH], q3[CH];
#pragma unroll
        for (int jj = 0; jj < CH; ++jj) p1[jj] = q2[jj] = q3[jj] = 0.0;
        for (int i = 0; i < N; ++i) {
            if (!((nm >> i) & 1u)) continue;
            const double yr = pl(s.Y3, Dm, 0, i, t), yi = pl(s.Y3, Dm, 1, i, t), ys = pl(s.Y3, Dm, 2, i, t);
#pragma unroll
            for (int jj = 0; jj < CH; ++jj)
                if (j0 + jj < N && ((vmask >> (j0 + jj)) & 1u)) {
                    const size_t o = (size_t)(row0 + i) * Dm + row0 + j0 + jj;
                    p1[jj] = fma(Ar[o], ys, p1[jj]);
                    q2[jj] = fma(Am[o], yi, q2[jj]);
                    q3[jj] = fma(Ap[o], yr, q3[jj]);
                }
        }
        if (!act) continue;
#pragma unroll
        for (int jj = 0; jj < CH; ++jj) {
            const int j = j0 + jj;
            if (j < N && ((vmask >> j) & 1u)) {
                const double2 acc = make_double2(p1[jj] + q2[jj], p1[jj] - q3[jj]);
                if (kind == 0 && j == 0) {
                    a.scratch[spos(cc, g.ia, u)] = acc;
                } else {
                    double2 *dst = Fb + fpos(cc, g.yr[j], u);
                    *dst = cadd(__ldcg(dst), acc);
                }
            }
        }
    }
    // pivot position: pull from this u and from u + 1_t
    if (act) {
        double2 pv = czero();
        if (HASB)
            for (int i = 0; i < N; ++i)
                if ((nm >> i) & 1u) pv = cfma_conj(s.br[row0 + i], get2(s.Y3, Dm, i, t), pv);
        for (int q = 0; q < tU; ++q) {
            if (!((upmask >> q) & 1u)) continue;
            const int un = u + cc.ustride[q];
            for (int i = 0; i < N; ++i) {
                if (!((nm >> i) & 1u)) continue;
                const double2 yn = rscale(__ldcg(Fb + fpos(cc, g.yw[i], un)), s.inv[g.den[i]]);
                pv = cfma_conj(s.Ar[(row0 + i) * Dm + Db + q], yn, pv);
            }
        }
        double2 *dst = Fb + fpos(cc, yP, u);
        *dst = cadd(__ldcg(dst), pv);
    }
    // dL/dA (rows = detected writes, columns = all reads) and dL/db partials:
    // one warp per entry, lanes over the tile's pairs, a fixed butterfly sum
    __syncthreads();
    const int lane = t & 31, warp = t >> 5;
    double2 *pA = a.partA + ((size_t)tl.circ * a.slots + blockIdx.x * a.spb) * Dm * Dm;
    for (int ent = warp; ent < N * NC; ent += TPB / 32) {
        const int i = ent / NC, j = ent % NC;
        if (!((nm >> i) & 1u)) continue;
        if (j < N && !((vmask >> j) & 1u)) continue;
        double2 acc = czero();
        for (int tt = lane; tt < TPB; tt += 32) acc = cfma_conj(get2(s.R3, Dm, j, tt), get2(s.Y3, Dm, i, tt), acc);
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) {
            double2 &d = pA[(row0 + i) * Dm + col_index(g, Db, j)];
            d = cadd(d, acc);
        }
    }
    if (HASB) {
        double2 *pb = a.partb + ((size_t)tl.circ * a.slots + blockIdx.x * a.spb) * Dm;
        for (int i = warp; i < N; i += TPB / 32) {
            if (!((nm >> i) & 1u)) continue;
            double2 acc = czero();
            for (int tt = lane; tt < TPB; tt += 32) acc = cfma_conj(s.FP[tt], get2(s.Y3, Dm, i, tt), acc);
            for (int o = 16; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (lane == 0) pb[row0 + i] = cadd(pb[row0 + i], acc);
        }
    }
    __syncthreads();
}

// Adjoint of the diagonal positions of level `lev` for every u: upstream
// seed plus the diagonal-read contributions left in scratch.
__device__ void diag_reverse(const CondArgs &a, CSmem &s, const CTile &tl, int lev)
{
    const CondCirc &cc = a.plan[tl.circ];
    const DiagShape &ds = cc.dsh;
    const int u = tl.chunk * TPB + threadIdx.x;
    if (u >= cc.U2) return;
    const Dig d = unrank(ds.C, ds.M, ltab(a, cc), 0, 0, lev, tl.rank);
    int64_t idx = 0;
    double f = 1.0;
    int fnz = ds.M;
    for (int i = 0; i < ds.M; ++i) {
        const int v = d(i);
        idx += (int64_t)v * ds.stride[i];
        f *= s.fact[v];
        if (v > 0 && fnz == ds.M) fnz = i;
    }
    int ket, bra;
    f *= uscale(cc, s, u, &ket, &bra);
    double2 acc = rscale(a.grho[rpos(cc, (idx * cc.NUo + ket) * cc.NUo + bra)], f);
    const int kmax = fnz < ds.M ? fnz : ds.M - 1;
    for (int K = 0; K <= kmax; ++K)
        if (d(K) <= ds.C[K] - 2) {
            const int64_t ia = ds.off_ap[K] + box_index(ds, d, K, K, 1, -1, 0);
            acc = cadd(acc, __ldcg(a.scratch + spos(cc, ia, u)));
        }
    double2 *dst = a.Fbar + cc.off_F + fpos(cc, idx, u);
    *dst = cadd(__ldcg(dst), acc);
}

// Sum of a double2 over the 32 lanes (xor butterfly: a fixed order, so the
// result does not depend on timing).
__device__ __forceinline__ double2 warp_sum(double2 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Sum of one double2 per thread over the block, in a fixed order; every
// thread gets the result.
__device__ double2 block_sum(double2 v)
{
    __shared__ double2 part[TPB / 32];
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    double2 r = czero();
    for (int k = 0; k < TPB / 32; ++k) r = cadd(r, part[k]);
    return r;
}

// Step 1 in reverse, one block per circuit, the levels of the undetected
// sub-lattice from the top down.  Every reader of a point v lies one level
// above it (u = v + 1_w, the b term) or two (u = v + 1_t + 1_w with t >= w,
// the A term), w being the first nonzero index of u, i.e. w <= the first
// nonzero index of v.  Each thread owns the points of the level and pulls
// their adjoint from those readers, whose adjoints are final; no two threads
// write one point.  X holds the adjoints: the shared staging area (with the
// levels lv) when the u-block fits it, else Fbar itself.
template <bool SMEM>
__device__ void step1_reverse_levels(const CondArgs &a, const CSmem &s, int c, bool hb, double2 *X,
                                     const unsigned char *lv, const int *ust, const int *ucu)
{
    const CondCirc &cc = a.plan[c];
    const int tU = 2 * cc.nU, Db = 2 * cc.dsh.M, Dm = a.Dmax, U2 = cc.U2;
    for (int lev = cc.Lu - 1; lev >= 0; --lev) {   // the top level has no readers
        for (int v = threadIdx.x; v < U2; v += blockDim.x) {
            if (SMEM && lv[v] != lev) continue;
            int dv[2 * FK_MAXU], f0;
            if (u_digits(v, tU, ust, ucu, dv, &f0) != lev) continue;
            double2 acc = czero();
            for (int w = 0; w < tU && w <= f0; ++w) {
                if (dv[w] + 1 >= ucu[w]) continue;   // v + 1_w leaves the box
                const int u1 = v + ust[w];
                if (hb)
                    acc = cfma_conj(s.br[Db + w],
                                    rscale(ld_u<SMEM>(X + (SMEM ? u1 : fpos(cc, 0, u1))), s.inv[dv[w] + 1]), acc);
                for (int t = w; t < tU; ++t) {
                    const int dt = dv[t] + 1 + (t == w ? 1 : 0);   // digit t of u = v + 1_t + 1_w
                    if (dt >= ucu[t]) continue;
                    const int dw = dv[w] + 1 + (t == w ? 1 : 0);   // its digit w
                    const int u2 = u1 + ust[t];
                    acc = cfma_conj(s.Ar[(Db + w) * Dm + Db + t],
                                    rscale(ld_u<SMEM>(X + (SMEM ? u2 : fpos(cc, 0, u2))), s.inv[dw]), acc);
                }
            }
            double2 *dst = X + (SMEM ? v : fpos(cc, 0, v));
            *dst = cadd(ld_u<SMEM>(dst), acc);
        }
        __syncthreads();
    }
}

__device__ void step1_reverse(const CondArgs &a, CSmem &s, int c, bool hb)
{
    __shared__ int ust[2 * FK_MAXU], ucu[2 * FK_MAXU];
    const CondCirc &cc = a.plan[c];
    load_circuit(a, s, c);
    stage_ubox(cc, ust, ucu);
    const double2 *F = a.F + cc.off_F;
    double2 *Fb = a.Fbar + cc.off_F;
    const int tU = 2 * cc.nU, Db = 2 * cc.dsh.M, Dm = a.Dmax, U2 = cc.U2;
    const bool staged = step1_staged(s, cc);
    double2 *X = staged ? (double2 *)s.s1 : Fb;
    unsigned char *lv = staged ? (unsigned char *)(X + U2) : nullptr;
    // the adjoints so far (and, with no detected mode, the upstream seed)
    for (int u = threadIdx.x; u < U2; u += blockDim.x) {
        int dig[2 * FK_MAXU], f0;
        const int lev = u_digits(u, tU, ust, ucu, dig, &f0);
        double2 y = __ldcg(Fb + fpos(cc, 0, u));
        if (cc.dsh.M == 0) {
            int ket, bra;
            const double f = uscale(cc, s, u, &ket, &bra);
            y = cadd(y, rscale(a.grho[rpos(cc, (int64_t)ket * cc.NUo + bra)], f));
        }
        if (staged) {
            X[u] = y;
            lv[u] = (unsigned char)lev;
        } else if (cc.dsh.M == 0) {
            Fb[fpos(cc, 0, u)] = y;
        }
    }
    __syncthreads();
    if (staged) {
        step1_reverse_levels<true>(a, s, c, hb, X, lv, ust, ucu);
        for (int u = threadIdx.x; u < U2; u += blockDim.x) Fb[fpos(cc, 0, u)] = X[u];
    } else {
        step1_reverse_levels<false>(a, s, c, hb, X, nullptr, ust, ucu);
    }
    // partial sums: entry (w, t) with t >= w of dL/dA, t = tU the b term,
    // each a sum over u formed in a fixed order
    double2 *pA = a.partA + ((size_t)c * a.slots + blockIdx.x * a.spb) * Dm * Dm;
    double2 *pb = a.partb + ((size_t)c * a.slots + blockIdx.x * a.spb) * Dm;
    for (int w = 0; w < tU; ++w)
        for (int t = w; t <= tU; ++t) {
            if (t == tU && !hb) continue;
            double2 acc = czero();
            for (int u = threadIdx.x; u < U2; u += blockDim.x) {
                int du[2 * FK_MAXU], f0;
                u_digits(u, tU, ust, ucu, du, &f0);
                if (f0 != w) continue;   // u = 0, or another first index
                const int P = u - ust[w];
                const double2 y = rscale(staged ? X[u] : __ldcg(Fb + fpos(cc, 0, u)), s.inv[du[w]]);
                if (t == tU) {
                    acc = cfma_conj(__ldcg(F + fpos(cc, 0, P)), y, acc);
                } else if (du[t] - (t == w ? 1 : 0) > 0) {
                    acc = cfma_conj(__ldcg(F + fpos(cc, 0, P - ust[t])), y, acc);
                }
            }
            acc = block_sum(acc);
            if (threadIdx.x == 0) {
                double2 *dst = (t == tU) ? pb + Db + w : pA + (Db + w) * Dm + Db + t;
                *dst = cadd(*dst, acc);
            }
        }
    __syncthreads();
}

template <int KS>
__global__ void __launch_bounds__(TPB, (KS == 1 ? 4 : 1)) cond_vjp_kernel(const __grid_constant__ CondArgs a)
{
    FK_DBG_BEGIN(a.ctl);
    if (skip_walk(a.ctl)) return;   // the input scan found a NaN or Inf
    CSmem s = carve(a, true, KS);
    build_tables(s);
    prologue(a);
    build_geo(a, s);
    if constexpr (KS > 0) build_cond_digits<KS>(a, s);
    if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
    const bool hb = *(volatile int *)&a.ctl->has_b != 0;
    for (int lev = a.Lmax; lev >= 0; --lev) {
        if (lev < a.Lmax) {
            const int nt = phase_tiles(a, s, 0, lev);
            int t0, t1;
            tile_range(nt, &t0, &t1);
            for (int tile = t0; tile < t1; ++tile) {
                const CTile tl = decode(a, s, 0, lev, tile);
                if constexpr (KS > 0) {
                    if (hb) pair_reverse_tc<KS, true>(a, s, tl, 0, lev);
                    else pair_reverse_tc<KS, false>(a, s, tl, 0, lev);
                } else {
                    if (hb) pair_reverse<true>(a, s, tl, 0, lev);
                    else pair_reverse<false>(a, s, tl, 0, lev);
                }
            }
            if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
        }
        {
            const int nt = phase_tiles(a, s, 2, lev);
            int t0, t1;
            tile_range(nt, &t0, &t1);
            for (int tile = t0; tile < t1; ++tile) diag_reverse(a, s, decode(a, s, 2, lev, tile), lev);
            if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
        }
        if (lev < a.Lmax) {
            const int nt = phase_tiles(a, s, 1, lev);
            int t0, t1;
            tile_range(nt, &t0, &t1);
            for (int tile = t0; tile < t1; ++tile) {
                const CTile tl = decode(a, s, 1, lev, tile);
                if constexpr (KS > 0) {
                    if (hb) pair_reverse_tc<KS, true>(a, s, tl, 1, lev);
                    else pair_reverse_tc<KS, false>(a, s, tl, 1, lev);
                } else {
                    if (hb) pair_reverse<true>(a, s, tl, 1, lev);
                    else pair_reverse<false>(a, s, tl, 1, lev);
                }
            }
            if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
        }
    }
    for (int c = blockIdx.x; c < a.B; c += gridDim.x) step1_reverse(a, s, c, hb);
    // final reduction, symmetrisation and scatter to the caller's lattice order
    const int Dm = a.Dmax, Do = a.D_orig;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = gtid; e < (int64_t)a.B * Do * Do; e += gsz) a.gA[e] = czero();
    for (int64_t e = gtid; e < (int64_t)a.B * Do; e += gsz) a.gb[e] = czero();
    if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
    // one warp per entry (w <= l of the symmetric dL/dA, then dL/db): the lanes
    // sum interleaved subsets of the slots, a butterfly joins them
    const int lane = threadIdx.x & 31;
    const int64_t gw = gtid >> 5, nw = gsz >> 5, nA = (int64_t)a.B * Dm * Dm;
    for (int64_t e = gw; e < nA + (int64_t)a.B * Dm; e += nw) {
        if (e < nA) {
            const int c = (int)(e / (Dm * Dm));
            const int w = (int)((e / Dm) % Dm), l = (int)(e % Dm);
            const CondCirc &cc = a.plan[c];
            if (w > l || l >= cc.Dred) continue;
            double2 x = czero(), y = czero();
            const double2 *pA = a.partA + (size_t)c * a.slots * Dm * Dm;
            for (int blk = lane; blk < a.slots; blk += 32) {
                x = cadd(x, __ldcg(pA + (size_t)blk * Dm * Dm + (size_t)w * Dm + l));
                y = cadd(y, __ldcg(pA + (size_t)blk * Dm * Dm + (size_t)l * Dm + w));
            }
            x = warp_sum(x);
            y = warp_sum(y);
            if (lane == 0) {
                const double2 g = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y + y.y));
                const int ow = cc.red_to_orig[w], ol = cc.red_to_orig[l];
                a.gA[(size_t)c * Do * Do + (size_t)ow * Do + ol] = g;
                a.gA[(size_t)c * Do * Do + (size_t)ol * Do + ow] = g;
            }
        } else {
            const int c = (int)((e - nA) / Dm), w = (int)((e - nA) % Dm);
            const CondCirc &cc = a.plan[c];
            if (w >= cc.Dred) continue;
            double2 x = czero();
            for (int blk = lane; blk < a.slots; blk += 32)
                x = cadd(x, __ldcg(a.partb + ((size_t)c * a.slots + blk) * Dm + w));
            x = warp_sum(x);
            if (lane == 0) a.gb[(size_t)c * Do + cc.red_to_orig[w]] = x;
        }
    }
    for (int64_t c = gtid; c < a.B; c += gsz) a.gc[c] = __ldcg(a.Fbar + a.plan[c].off_F);
}

}  // namespace

// Kernels of one product engine, for the host side.
struct CondKernels {
    const void *forward, *vjp;
};

}  // namespace fk
