// walk_cond.cu -- persistent sm_103a kernels for conditional states
// (Algorithm 2 of arXiv 2303.08879, Sec. 3.2) and their reverse-mode adjoint.
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
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "fk_internal.h"
#include "walk_common.cuh"
#include "../../include/fockdiag.h"

namespace fk {

namespace {

constexpr int TPB = kCondTPB;
constexpr int RS = TPB + 1;
constexpr int MAXB = 1024;                        // circuits per launch

struct PGeom;

struct CondArgs {
    int B, Md, Dmax, grid, Lmax, D_orig;
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
    double *A3;                 // [3][Dmax][Dmax]: Re A, Re A + Im A, Im A - Re A
    double *R3, *Y3;            // [3][Dmax][RS] reads (Re x, Im x, Re x + Im x), scaled
                                // output adjoints (Re y, Im y, Re y + Im y)
    double2 *FP;                // [RS] pivot values (VJP)
    PGeom *geo;                 // the current tile's pivot
    int *ctiles;                // [MAXB + 1] tile prefix over circuits
    int loaded;
};

__host__ __device__ inline size_t cond_smem_bytes(int Dmax, bool vjp)
{
    size_t n = 3 * kTabN * sizeof(double);
    n += (size_t)Dmax * Dmax * sizeof(double2) + (size_t)Dmax * sizeof(double2);
    n += 3 * (size_t)Dmax * Dmax * sizeof(double);
    n += 3 * (size_t)Dmax * RS * sizeof(double);    // at most 2M matrix columns per pivot
    if (vjp) n += 3 * (size_t)Dmax * RS * sizeof(double) + RS * sizeof(double2);
    n = (n + 15) & ~(size_t)15;
    n += sizeof(PGeom);
    n += (MAXB + 1) * sizeof(int);
    return n + 64;
}

__device__ CSmem carve(const CondArgs &a, bool vjp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CSmem s;
    unsigned char *p = smem_raw;
    const size_t Dm = (size_t)a.Dmax;
    s.inv = (double *)p; p += kTabN * sizeof(double);
    s.fact = (double *)p; p += kTabN * sizeof(double);
    s.sqf = (double *)p; p += kTabN * sizeof(double);
    s.Ar = (double2 *)p; p += Dm * Dm * sizeof(double2);
    s.br = (double2 *)p; p += Dm * sizeof(double2);
    s.A3 = (double *)p; p += 3 * Dm * Dm * sizeof(double);
    s.R3 = (double *)p; p += 3 * Dm * RS * sizeof(double);
    if (vjp) {
        s.Y3 = (double *)p; p += 3 * Dm * RS * sizeof(double);
        s.FP = (double2 *)p; p += RS * sizeof(double2);
    } else {
        s.Y3 = nullptr;
        s.FP = nullptr;
    }
    p = smem_raw + ((p - smem_raw + 15) & ~(size_t)15);
    s.geo = (PGeom *)p; p += sizeof(PGeom);
    s.ctiles = (int *)p;
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
        s.A3[e] = v.x;
        s.A3[Dm * Dm + e] = v.x + v.y;
        s.A3[2 * Dm * Dm + e] = v.y - v.x;
    }
    for (int e = threadIdx.x; e < Dm; e += blockDim.x) s.br[e] = a.br[(size_t)c * Dm + e];
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
__device__ void step1_forward(const CondArgs &a, CSmem &s, int c, bool hb)
{
    const CondCirc &cc = a.plan[c];
    load_circuit(a, s, c);
    double2 *F = a.F + cc.off_F;
    const int tU = 2 * cc.nU, Db = 2 * cc.dsh.M;
    for (int lev = 0; lev <= cc.Lu; ++lev) {
        for (int u = threadIdx.x; u < cc.U2; u += blockDim.x) {
            int dig[2 * FK_MAXU], sum = 0, w = -1;
            for (int t = 0; t < tU; ++t) {
                dig[t] = udigit(cc, u, t);
                sum += dig[t];
                if (w < 0 && dig[t] > 0) w = t;
            }
            if (sum != lev) continue;
            double2 v;
            if (lev == 0) {
                v = a.c[c];
            } else {
                const int P = u - cc.ustride[w];
                const int Pw = dig[w] - 1;
                double2 acc = hb ? cmul(s.br[Db + w], __ldcg(F + fpos(cc, 0, P))) : czero();
                for (int t = 0; t < tU; ++t) {
                    const int Pt = dig[t] - (t == w ? 1 : 0);
                    if (Pt <= 0) continue;
                    acc = cfma(s.Ar[(Db + w) * a.Dmax + Db + t], __ldcg(F + fpos(cc, 0, P - cc.ustride[t])), acc);
                }
                v = rscale(acc, s.inv[Pw + 1]);
            }
            F[fpos(cc, 0, u)] = v;
            int ket, bra;
            const double f = uscale(cc, s, u, &ket, &bra);
            a.rho[rpos(cc, (int64_t)ket * cc.NUo + bra)] = rscale(v, f);
        }
        __syncthreads();
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
    if (threadIdx.x == 0) {
        s.ctiles[0] = 0;
        for (int c = 0; c < a.B; ++c) s.ctiles[c + 1] += s.ctiles[c];
    }
    __syncthreads();
    return s.ctiles[a.B];
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
// circuit, a thread per pivot of each (kind, level, segment).
__device__ void build_geo(const CondArgs &a, const CSmem &s)
{
    for (int c = blockIdx.x; c < a.B; c += gridDim.x) {
        const CondCirc &cc = a.plan[c];
        const DiagShape &ds = cc.dsh;
        if (ds.M == 0) continue;
        const LevelTab W = ltab(a, cc);
        for (int kind = 0; kind < 2; ++kind)
            for (int lev = 0; lev < ds.L; ++lev) {
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

__global__ void __launch_bounds__(TPB) cond_forward_kernel(const __grid_constant__ CondArgs a)
{
    FK_DBG_BEGIN(a.ctl);
    if (skip_walk(a.ctl)) return;   // the input scan found a NaN or Inf
    CSmem s = carve(a, false);
    build_tables(s);
    prologue(a);
    build_geo(a, s);
    if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
    const bool hb = *(volatile int *)&a.ctl->has_b != 0;
    for (int c = blockIdx.x; c < a.B; c += gridDim.x) step1_forward(a, s, c, hb);
    if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
    for (int lev = 0; lev < a.Lmax; ++lev) {
        for (int kind = 1; kind >= 0; --kind) {     // diagonal pivots, then off-diagonal
            const int nt = phase_tiles(a, s, kind, lev);
            for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
                const CTile tl = decode(a, s, kind, lev, tile);
                if (hb) pair_forward<true>(a, s, tl, kind, lev);
                else pair_forward<false>(a, s, tl, kind, lev);
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
    double2 *pA = a.partA + ((size_t)tl.circ * a.grid + blockIdx.x) * Dm * Dm;
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
        double2 *pb = a.partb + ((size_t)tl.circ * a.grid + blockIdx.x) * Dm;
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

// Step 1 in reverse, one thread per circuit, u in decreasing flat order (every
// reader of u has a larger flat index).
__device__ void step1_reverse(const CondArgs &a, CSmem &s, int c, bool hb)
{
    const CondCirc &cc = a.plan[c];
    load_circuit(a, s, c);
    if (threadIdx.x != 0) return;
    const double2 *F = a.F + cc.off_F;
    double2 *Fb = a.Fbar + cc.off_F;
    const int tU = 2 * cc.nU, Db = 2 * cc.dsh.M, Dm = a.Dmax;
    double2 *pA = a.partA + ((size_t)c * a.grid + blockIdx.x) * Dm * Dm;
    double2 *pb = a.partb + ((size_t)c * a.grid + blockIdx.x) * Dm;
    if (cc.dsh.M == 0) {   // no detected mode: the upstream seed lands here
        for (int u = 0; u < cc.U2; ++u) {
            int ket, bra;
            const double f = uscale(cc, s, u, &ket, &bra);
            Fb[fpos(cc, 0, u)] = cadd(Fb[u], rscale(a.grho[rpos(cc, (int64_t)ket * cc.NUo + bra)], f));
        }
    }
    for (int u = cc.U2 - 1; u >= 1; --u) {
        int dig[2 * FK_MAXU], w = -1;
        for (int q = 0; q < tU; ++q) {
            dig[q] = udigit(cc, u, q);
            if (w < 0 && dig[q] > 0) w = q;
        }
        const int P = u - cc.ustride[w];
        const double2 y = rscale(Fb[u], s.inv[dig[w]]);
        if (hb) {
            Fb[fpos(cc, 0, P)] = cfma_conj(s.br[Db + w], y, Fb[P]);
            pb[Db + w] = cfma_conj(F[P], y, pb[Db + w]);
        }
        for (int q = 0; q < tU; ++q) {
            const int Pq = dig[q] - (q == w ? 1 : 0);
            if (Pq <= 0) continue;
            const int r = P - cc.ustride[q];
            Fb[fpos(cc, 0, r)] = cfma_conj(s.Ar[(Db + w) * Dm + Db + q], y, Fb[r]);
            double2 &dA = pA[(Db + w) * Dm + Db + q];
            dA = cfma_conj(F[r], y, dA);
        }
    }
}

__global__ void __launch_bounds__(TPB) cond_vjp_kernel(const __grid_constant__ CondArgs a)
{
    FK_DBG_BEGIN(a.ctl);
    if (skip_walk(a.ctl)) return;   // the input scan found a NaN or Inf
    CSmem s = carve(a, true);
    build_tables(s);
    prologue(a);
    build_geo(a, s);
    if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
    const bool hb = *(volatile int *)&a.ctl->has_b != 0;
    for (int lev = a.Lmax; lev >= 0; --lev) {
        if (lev < a.Lmax) {
            const int nt = phase_tiles(a, s, 0, lev);
            for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
                const CTile tl = decode(a, s, 0, lev, tile);
                if (hb) pair_reverse<true>(a, s, tl, 0, lev);
                else pair_reverse<false>(a, s, tl, 0, lev);
            }
            if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
        }
        {
            const int nt = phase_tiles(a, s, 2, lev);
            for (int tile = blockIdx.x; tile < nt; tile += gridDim.x)
                diag_reverse(a, s, decode(a, s, 2, lev, tile), lev);
            if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
        }
        if (lev < a.Lmax) {
            const int nt = phase_tiles(a, s, 1, lev);
            for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
                const CTile tl = decode(a, s, 1, lev, tile);
                if (hb) pair_reverse<true>(a, s, tl, 1, lev);
                else pair_reverse<false>(a, s, tl, 1, lev);
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
    for (int64_t e = gtid; e < (int64_t)a.B * Dm * Dm; e += gsz) {
        const int c = (int)(e / (Dm * Dm));
        const int w = (int)((e / Dm) % Dm), l = (int)(e % Dm);
        const CondCirc &cc = a.plan[c];
        if (w >= cc.Dred || l >= cc.Dred) continue;
        double2 x = czero(), y = czero();
        for (int blk = 0; blk < a.grid; ++blk) {
            const double2 *pA = a.partA + ((size_t)c * a.grid + blk) * Dm * Dm;
            x = cadd(x, pA[(size_t)w * Dm + l]);
            y = cadd(y, pA[(size_t)l * Dm + w]);
        }
        const int ow = cc.red_to_orig[w], ol = cc.red_to_orig[l];
        a.gA[(size_t)c * Do * Do + (size_t)ow * Do + ol] =
            make_double2(0.5 * (x.x + y.x), 0.5 * (x.y + y.y));
    }
    for (int64_t e = gtid; e < (int64_t)a.B * Dm; e += gsz) {
        const int c = (int)(e / Dm), w = (int)(e % Dm);
        const CondCirc &cc = a.plan[c];
        if (w >= cc.Dred) continue;
        double2 x = czero();
        for (int blk = 0; blk < a.grid; ++blk) x = cadd(x, a.partb[((size_t)c * a.grid + blk) * Dm + w]);
        a.gb[(size_t)c * Do + cc.red_to_orig[w]] = x;
    }
    for (int64_t c = gtid; c < a.B; c += gsz) a.gc[c] = a.Fbar[a.plan[c].off_F];
}

// --------------------------------------------------------- host plumbing
struct PlanEntry {
    CondPlan plan;
    std::vector<unsigned char> bytes;
    void *pinned = nullptr;
};

std::mutex g_plan_mu;
std::map<std::string, std::unique_ptr<PlanEntry>> g_plans;

int build_plan(int B, int M, const int *cut, const unsigned char *mask, PlanEntry *pe)
{
    if (B < 1 || B > MAXB || M < 1 || M > FK_MAXM + FK_MAXU || !cut || !mask) return FK_EINVAL;
    int Md = 0;
    for (int j = 0; j < M; ++j) Md += mask[j] ? 1 : 0;
    std::vector<CondCirc> cc(B);
    std::vector<unsigned> tabs;
    int64_t offF = 0, offR = 0, offS = 0, offG = 0;
    int Lmax = 0;
    for (int c = 0; c < B; ++c) {
        CondCirc &x = cc[c];
        std::memset(&x, 0, sizeof(x));
        const int *C = cut + (size_t)c * M;
        int dcut[FK_MAXM + FK_MAXU], dmode[FK_MAXM + FK_MAXU], nd = 0;
        int nu = 0;
        int64_t NUo = 1;
        for (int j = 0; j < M; ++j) {
            if (C[j] < 1) return FK_EINVAL;
            if (C[j] > FK_MAX_CUTOFF) return FK_EUNSUPPORTED;
            if (mask[j]) {
                dcut[nd] = C[j];
                dmode[nd] = j;
                ++nd;
            } else if (C[j] > 1) {
                if (nu >= FK_MAXU) return FK_EUNSUPPORTED;
                x.CU[nu] = C[j];
                dmode[FK_MAXM + nu] = j;
                NUo *= C[j];
                ++nu;
            }
        }
        x.nU = nu;
        DiagShape &ds = x.dsh;
        bool any_det = false;
        for (int i = 0; i < nd; ++i) any_det |= dcut[i] > 1;
        if (any_det) {
            int rc = build_diag_shape(nd, dcut, true, &ds);
            if (rc) return rc;
            for (int i = 0; i < ds.M; ++i) ds.mode_map[i] = dmode[ds.mode_map[i]];
        } else {
            std::memset(&ds, 0, sizeof(ds));
            ds.n_diag = 1;
            ds.circ_size = 1;
        }
        int64_t U2 = 1;
        for (int a2 = 0; a2 < nu; ++a2) U2 *= (int64_t)x.CU[a2] * x.CU[a2];
        if (U2 > (1 << 24)) return FK_EUNSUPPORTED;
        x.U2 = (int)U2;
        int st = 1;
        for (int t = 2 * nu - 1; t >= 0; --t) {
            x.ustride[t] = st;
            st *= x.CU[t >> 1];
        }
        x.Lu = 0;
        for (int a2 = 0; a2 < nu; ++a2) x.Lu += 2 * (x.CU[a2] - 1);
        x.nchunk = (x.U2 + kCondTPB - 1) / kCondTPB;
        x.NUo = (int)NUo;
        x.Dred = 2 * (ds.M + nu);
        for (int i = 0; i < ds.M; ++i) {
            x.red_to_orig[2 * i] = 2 * ds.mode_map[i];
            x.red_to_orig[2 * i + 1] = 2 * ds.mode_map[i] + 1;
        }
        for (int a2 = 0; a2 < nu; ++a2) {
            x.red_to_orig[2 * ds.M + 2 * a2] = 2 * dmode[FK_MAXM + a2];
            x.red_to_orig[2 * ds.M + 2 * a2 + 1] = 2 * dmode[FK_MAXM + a2] + 1;
        }
        // level table of the detected cutoffs
        x.Wn = ds.L + 2;
        x.W_off = (int)tabs.size();
        const int Mw = ds.M;
        std::vector<unsigned> W((size_t)(Mw + 1) * x.Wn, 0u);
        W[(size_t)Mw * x.Wn] = 1u;
        for (int i = Mw - 1; i >= 0; --i)
            for (int t2 = 0; t2 < x.Wn; ++t2) {
                unsigned acc = 0;
                for (int v = 0; v < ds.C[i] && v <= t2; ++v) acc += W[(size_t)(i + 1) * x.Wn + t2 - v];
                W[(size_t)i * x.Wn + t2] = acc;
            }
        tabs.insert(tabs.end(), W.begin(), W.end());
        // pivot prefix per (kind, level): AP(K) pivots of level s are the vectors
        // over modes K.. with digit K < C_K - 1 summing to s; DP pivots those of K = 0
        auto fam_count = [&](int K, int lev) {
            int64_t n = 0;
            for (int v = 0; v < ds.C[K] - 1 && v <= lev; ++v) n += W[(size_t)(K + 1) * x.Wn + lev - v];
            return n;
        };
        x.gp_off = (int)tabs.size();
        int64_t npiv = 0;
        for (int kind = 0; kind < 2; ++kind)
            for (int lev = 0; lev <= ds.L; ++lev) {
                if (npiv >= (int64_t(1) << 32)) return FK_EUNSUPPORTED;
                tabs.push_back((unsigned)npiv);
                if (lev < ds.L && Mw > 0)
                    for (int K = 0; K < (kind == 0 ? Mw : 1); ++K) npiv += fam_count(K, lev);
            }
        x.geo_off = offG;
        offG += npiv;
        x.n_patterns = ds.n_diag;
        x.off_F = offF;
        x.off_rho = offR;
        x.off_scratch = offS;
        offF += ds.circ_size * U2;
        offR += ds.n_diag * NUo * NUo;
        offS += ds.n_ap * U2;
        if (ds.L > Lmax) Lmax = ds.L;
    }
    PlanEntry &p = *pe;
    p.plan.B = B;
    p.plan.M = M;
    p.plan.Md = Md;
    p.plan.Dmax = 2 * M;
    p.plan.Lmax = Lmax;
    p.plan.F_total = offF;
    p.plan.scratch_total = offS;
    p.plan.rho_total = offR;
    p.plan.geo_total = offG;
    const size_t nb = sizeof(CondCirc) * B + sizeof(unsigned) * tabs.size();
    p.bytes.resize(nb);
    std::memcpy(p.bytes.data(), cc.data(), sizeof(CondCirc) * B);
    std::memcpy(p.bytes.data() + sizeof(CondCirc) * B, tabs.data(), sizeof(unsigned) * tabs.size());
    p.plan.plan_bytes = nb;
    p.plan.host_plan = p.bytes.data();
    return FK_OK;
}

int pinned_plan(const CondPlan &plan, const void **out)
{
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (auto &kv : g_plans) {
        PlanEntry &pe = *kv.second;
        if (&pe.plan != &plan) continue;
        if (!pe.pinned) {
            if (cudaHostAlloc(&pe.pinned, pe.bytes.size(), cudaHostAllocDefault) != cudaSuccess) {
                pe.pinned = nullptr;
                return FK_ECUDA;
            }
            std::memcpy(pe.pinned, pe.bytes.data(), pe.bytes.size());
        }
        *out = pe.pinned;
        return FK_OK;
    }
    return FK_EINVAL;
}

int device_sms(int *sms)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FK_ECUDA;
    if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FK_ECUDA;
    return FK_OK;
}

int launch(const void *fn, int grid, size_t smem, CondArgs *args, cudaStream_t st)
{
    void *params[] = {args};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(TPB), params, smem, st) == cudaSuccess
               ? FK_OK
               : FK_ECUDA;
}

CondArgs make_args(const CondPlan &plan, const void *A, const void *b, const void *c, void *ws,
                   const CondLayout &lay)
{
    CondArgs a{};
    char *w = (char *)ws;
    a.B = plan.B;
    a.Md = plan.Md;
    a.Dmax = plan.Dmax;
    a.Lmax = plan.Lmax;
    a.D_orig = 2 * plan.M;
    a.plan = (const CondCirc *)(w + lay.plan);
    a.Wall = (const unsigned *)(w + lay.plan + sizeof(CondCirc) * plan.B);
    a.A = (const double2 *)A;
    a.b = (const double2 *)b;
    a.c = (const double2 *)c;
    a.ctl = (Control *)(w + lay.ctl);
    a.Ar = (double2 *)(w + lay.Ar);
    a.br = (double2 *)(w + lay.br);
    a.F = (double2 *)(w + lay.F);
    a.geo = (PGeom *)(w + lay.geo);
    a.timeout_ns = kBarrierTimeoutNs;
    return a;
}

}  // namespace

int get_cond_plan(int batch, int M, const int *cutoffs, const unsigned char *mask,
                  const CondPlan **plan)
{
    if (batch < 1 || M < 1 || !cutoffs || !mask || !plan) return FK_EINVAL;
    std::string key((const char *)&batch, sizeof(int));
    key.append((const char *)&M, sizeof(int));
    key.append((const char *)cutoffs, sizeof(int) * (size_t)batch * M);
    key.append((const char *)mask, (size_t)M);
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plans.find(key);
    if (it == g_plans.end()) {
        std::unique_ptr<PlanEntry> pe(new PlanEntry());
        int rc = build_plan(batch, M, cutoffs, mask, pe.get());
        if (rc) return rc;
        it = g_plans.emplace(key, std::move(pe)).first;
    }
    *plan = &it->second->plan;
    return FK_OK;
}

int cond_grid_size(const CondPlan &plan, bool vjp, int *grid)
{
    int sms = 0;
    int rc = device_sms(&sms);
    if (rc) return rc;
    const size_t smem = cond_smem_bytes(plan.Dmax, vjp);
    const void *fn = vjp ? (const void *)cond_vjp_kernel : (const void *)cond_forward_kernel;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return FK_ECUDA;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, TPB, smem) != cudaSuccess) return FK_ECUDA;
    if (per < 1) return FK_EUNSUPPORTED;
    *grid = per * sms;
    return FK_OK;
}

int cond_layout(const CondPlan &plan, bool vjp, CondLayout *lay)
{
    const size_t B = (size_t)plan.B, D = (size_t)plan.Dmax, c16 = 16;
    size_t o = 0;
    lay->ctl = o; o = align_up(o + sizeof(Control));
    lay->plan = o; o = align_up(o + plan.plan_bytes);
    lay->Ar = o; o = align_up(o + B * D * D * c16);
    lay->br = o; o = align_up(o + B * D * c16);
    lay->geo = o; o = align_up(o + (size_t)plan.geo_total * sizeof(PGeom));
    lay->F = o; o = align_up(o + (size_t)plan.F_total * c16);
    lay->grid_vjp = 0;
    if (vjp) {
        int grid = 0;
        int rc = cond_grid_size(plan, true, &grid);
        if (rc) return rc;
        lay->grid_vjp = grid;
        lay->Fbar = o; o = align_up(o + (size_t)plan.F_total * c16);
        lay->scratch = o; o = align_up(o + (size_t)plan.scratch_total * c16);
        lay->partA = o; o = align_up(o + B * (size_t)grid * D * D * c16);
        lay->partb = o; o = align_up(o + B * (size_t)grid * D * c16);
    } else {
        lay->Fbar = lay->scratch = lay->partA = lay->partb = o;
    }
    lay->total = o;
    return FK_OK;
}

static int check_inputs(const CondPlan &plan, unsigned flags, const void *A, const void *b,
                        const void *c, char *w, const CondLayout &lay, cudaStream_t st)
{
    if (!(flags & FK_FLAG_CHECK_FINITE)) return FK_OK;
    const int64_t D = 2 * (int64_t)plan.M;
    return launch_check_finite(A, plan.B * D * D, b, plan.B * D, c, plan.B, (Control *)(w + lay.ctl), st);
}

int launch_cond_forward(const CondPlan &plan, unsigned flags, const void *A, const void *b,
                        const void *c, void *rho, void *ws, const CondLayout &lay, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const void *hp = nullptr;
    int rc = pinned_plan(plan, &hp);
    if (rc) return rc;
    char *w = (char *)ws;
    if (cudaMemsetAsync(w + lay.ctl, 0, sizeof(Control), st) != cudaSuccess) return FK_ECUDA;
    if ((rc = check_inputs(plan, flags, A, b, c, w, lay, st)) != 0) return rc;
    if (cudaMemcpyAsync(w + lay.plan, hp, plan.plan_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FK_ECUDA;
    CondArgs a = make_args(plan, A, b, c, ws, lay);
    a.rho = (double2 *)rho;
    int grid = 0;
    rc = cond_grid_size(plan, false, &grid);
    if (rc) return rc;
    a.grid = grid;
    return launch((const void *)cond_forward_kernel, grid, cond_smem_bytes(plan.Dmax, false), &a, st);
}

int launch_cond_vjp(const CondPlan &plan, unsigned flags, const void *A, const void *b,
                    const void *c, const void *grho, void *gA, void *gb, void *gc, void *ws,
                    const CondLayout &lay, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const void *hp = nullptr;
    int rc = pinned_plan(plan, &hp);
    if (rc) return rc;
    char *w = (char *)ws;
    if (cudaMemsetAsync(w + lay.ctl, 0, sizeof(Control), st) != cudaSuccess) return FK_ECUDA;
    if ((rc = check_inputs(plan, flags, A, b, c, w, lay, st)) != 0) return rc;
    if (cudaMemcpyAsync(w + lay.plan, hp, plan.plan_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FK_ECUDA;
    if (cudaMemsetAsync(w + lay.Fbar, 0, lay.partA - lay.Fbar, st) != cudaSuccess) return FK_ECUDA;
    if (cudaMemsetAsync(w + lay.partA, 0, lay.total - lay.partA, st) != cudaSuccess) return FK_ECUDA;
    CondArgs a = make_args(plan, A, b, c, ws, lay);
    a.grho = (const double2 *)grho;
    a.Fbar = (double2 *)(w + lay.Fbar);
    a.scratch = (double2 *)(w + lay.scratch);
    a.partA = (double2 *)(w + lay.partA);
    a.partb = (double2 *)(w + lay.partb);
    a.gA = (double2 *)gA;
    a.gb = (double2 *)gb;
    a.gc = (double2 *)gc;
    a.grid = lay.grid_vjp;
    return launch((const void *)cond_vjp_kernel, lay.grid_vjp, cond_smem_bytes(plan.Dmax, true), &a, st);
}

}  // namespace fk
