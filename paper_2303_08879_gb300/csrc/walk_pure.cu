// walk_pure.cu -- state-vector walk (Sec. 2.2, "State vector simulations") and
// its reverse-mode adjoint, for pure Gaussian states: psi_k for every k < C
// over M modes from the pure triple (A_psi, b_psi, psi_0).
//
// The kernels carry F_k = psi_k / sqrt(k!), so eq. (recrel) reads
//   F_x = (b_w F_P + sum_{l: P_l > 0} A_wl F_{P - 1_l}) / (P_w + 1),
// with the canonical parent P = x - 1_w, w the first nonzero index of x
// (every amplitude has one writer).  Pivots are applied in order of weight
// (digit sum): a thread owns one amplitude x of the current weight and pulls
// its (<= M + 1) reads from the two weights below.  With b = 0 only even
// weights are nonzero (Sec. 2.4) and odd weights are skipped.
//
// Reverse walk (the chain rule of Sec. 2.5 run backwards), in pull form so
// that every adjoint has one writer: an amplitude y is read
//   * as the parent P = y by x = y + 1_w for every w <= fnz(y) (b term), and
//   * as P - 1_l by x = y + 1_l + 1_w for every l and w <= min(fnz(y), l),
// hence
//   Fbar_y = seed_y + sum_{w <= fnz(y)} conj(b_w) Fbar_{y+1_w} / (y_w + 1)
//          + sum_l sum_{w <= min(fnz(y), l)} conj(A_wl) Fbar_{y+1_l+1_w} / ((y+1_l)_w + 1)
// over the two weights above.  Each x then adds conj(F_{P-1_l}/(P_w+1)) Fbar_x
// to dL/dA_wl and conj(F_P/(P_w+1)) Fbar_x to dL/db_w (block partials,
// reduced in a fixed order), and dL/dc = Fbar_0.
#include <cuda_runtime.h>

#include "fk_internal.h"
#include "walk_common.cuh"
#include "../../include/fockdiag.h"

namespace fk {

namespace {

constexpr int kPureTPB = 128;
constexpr int kPureMaxM = 16;

struct PureArgs {
    int M, L, B, grid;
    int C[kPureMaxM];
    int64_t stride[kPureMaxM];   // row-major strides of the box prod C
    int64_t n;                   // prod C
    unsigned flags;
    const double2 *A, *b, *c;    // caller's [B][M][M], [B][M], [B]
    double2 *psi;                // forward output [B][n]
    const double2 *gpsi;         // VJP input [B][n]
    Control *ctl;
    double2 *As, *bs, *F, *Fbar, *partA, *partb;
    double2 *gA, *gb, *gc;
    unsigned long long timeout_ns;
};

struct PureSmem {
    unsigned *S;                 // [(M+1)][L+2] prefix level counts
    int Wn;
    double *inv, *sqf;           // 1/v, sqrt(v!)
    double2 *A, *b;              // this circuit's A_s, b
    double2 *con;                // [TPB][M] per-thread contributions to a row of dL/dA
    double2 *conb;               // [TPB]   contributions to dL/db
    int *row;                    // [TPB]   their row (-1: none)
    int loaded;
};

__host__ __device__ inline size_t pure_smem_bytes(int M, int L)
{
    size_t n = (size_t)(M + 1) * (L + 2) * sizeof(unsigned);
    n = (n + 15) & ~(size_t)15;
    n += 2 * (size_t)kTabN * sizeof(double);
    n += (size_t)(M * M + M) * sizeof(double2);
    n += (size_t)kPureTPB * M * sizeof(double2) + kPureTPB * sizeof(double2) + kPureTPB * sizeof(int);
    return n + 64;
}

__device__ PureSmem carve(const PureArgs &a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PureSmem s;
    unsigned char *p = smem_raw;
    s.S = (unsigned *)p;
    s.Wn = a.L + 2;
    p += (size_t)(a.M + 1) * s.Wn * sizeof(unsigned);
    p = (unsigned char *)(((uintptr_t)p + 15) & ~(uintptr_t)15);
    s.inv = (double *)p; p += kTabN * sizeof(double);
    s.sqf = (double *)p; p += kTabN * sizeof(double);
    s.A = (double2 *)p; p += (size_t)a.M * a.M * sizeof(double2);
    s.b = (double2 *)p; p += (size_t)a.M * sizeof(double2);
    s.con = (double2 *)p; p += (size_t)kPureTPB * a.M * sizeof(double2);
    s.conb = (double2 *)p; p += kPureTPB * sizeof(double2);
    s.row = (int *)p;
    s.loaded = -1;
    return s;
}

__device__ void pure_tables(const PureArgs &a, PureSmem &s)
{
    double *fact = s.sqf;   // factorials first, square roots below
    build_scalar_tables(s.inv, fact);
    __syncthreads();
    for (int v = threadIdx.x; v < kTabN; v += blockDim.x) s.sqf[v] = sqrt(fact[v]);
    build_prefix_table(s.S, s.Wn, a.C, a.M);
}

__device__ void load_circ(const PureArgs &a, PureSmem &s, int circ)
{
    if (s.loaded == circ) return;
    __syncthreads();
    const int M = a.M;
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) s.A[e] = a.As[(size_t)circ * M * M + e];
    for (int e = threadIdx.x; e < M; e += blockDim.x) s.b[e] = a.bs[(size_t)circ * M + e];
    __syncthreads();
    s.loaded = circ;
}

__device__ __forceinline__ int64_t box_idx(const PureArgs &a, const Dig &x)
{
    int64_t i = 0;
    for (int m = 0; m < a.M; ++m) i += (int64_t)x(m) * a.stride[m];
    return i;
}

__device__ __forceinline__ int first_nz(const PureArgs &a, const Dig &x)
{
    for (int m = 0; m < a.M; ++m)
        if (x(m) > 0) return m;
    return a.M;
}

__device__ __forceinline__ double sqrt_fact(const PureArgs &a, const PureSmem &s, const Dig &x)
{
    double f = 1.0;
    for (int m = 0; m < a.M; ++m) f *= s.sqf[x(m)];
    return f;
}

// A_s = (A + A^T)/2 and b of every circuit; vacuum seeds (forward).
__device__ void pure_prologue(const PureArgs &a, bool seed)
{
    const int M = a.M;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = gtid; e < (int64_t)a.B * M * M; e += gsz) {
        const int64_t c = e / (M * M);
        const int w = (int)((e / M) % M), l = (int)(e % M);
        const double2 x = a.A[c * M * M + (int64_t)w * M + l];
        const double2 y = a.A[c * M * M + (int64_t)l * M + w];
        a.As[e] = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y + y.y));
    }
    for (int64_t e = gtid; e < (int64_t)a.B * M; e += gsz) a.bs[e] = a.b[e];
    if (seed)
        for (int64_t c = gtid; c < a.B; c += gsz) {
            a.F[c * a.n] = a.c[c];
            a.psi[c * a.n] = a.c[c];
        }
}

// Tiles of one weight are circuit-major, TPB amplitudes each, taken round robin.

__global__ void __launch_bounds__(kPureTPB) pure_forward_kernel(const __grid_constant__ PureArgs a)
{
    if (skip_walk(a.ctl)) return;   // the input scan found a NaN or Inf
    PureSmem s = carve(a);
    pure_tables(a, s);
    pure_prologue(a, true);
    const bool b0 = (a.flags & FK_FLAG_B_ZERO) != 0;
    if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
    const PrefixTab tab{s.S, s.Wn};
    const int M = a.M;
    for (int lev = 1; lev <= a.L; ++lev) {
        const unsigned cnt = level_count(a.C, tab, 0, 0, lev);
        const int per = (int)((cnt + kPureTPB - 1) / kPureTPB), nt = a.B * per;
        for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
            const int circ = tile / per;
            const unsigned r = (unsigned)(tile - circ * per) * kPureTPB + threadIdx.x;
            load_circ(a, s, circ);
            if (r >= cnt) continue;
            const Dig x = unrank(a.C, M, tab, 0, 0, lev, r);
            const int64_t xi = box_idx(a, x);
            double2 *F = a.F + (size_t)circ * a.n;
            if (b0 && (lev & 1)) {          // odd weights vanish when b = 0
                F[xi] = czero();
                a.psi[(size_t)circ * a.n + xi] = czero();
                continue;
            }
            const int w = first_nz(a, x);
            const int64_t pi = xi - a.stride[w];
            double2 acc = b0 ? czero() : cmul(s.b[w], __ldcg(F + pi));
            for (int l = w; l < M; ++l) {
                const int Pl = x(l) - (l == w ? 1 : 0);
                if (Pl > 0) acc = cfma(s.A[w * M + l], __ldcg(F + pi - a.stride[l]), acc);
            }
            const double2 v = rscale(acc, s.inv[x(w)]);
            F[xi] = v;
            a.psi[(size_t)circ * a.n + xi] = rscale(v, sqrt_fact(a, s, x));
        }
        if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
    }
}

__global__ void __launch_bounds__(kPureTPB) pure_vjp_kernel(const __grid_constant__ PureArgs a)
{
    if (skip_walk(a.ctl)) return;   // the input scan found a NaN or Inf
    PureSmem s = carve(a);
    pure_tables(a, s);
    pure_prologue(a, false);
    if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
    const PrefixTab tab{s.S, s.Wn};
    const int M = a.M, t = threadIdx.x;
    for (int lev = a.L; lev >= 0; --lev) {
        const unsigned cnt = level_count(a.C, tab, 0, 0, lev);
        const int per = (int)((cnt + kPureTPB - 1) / kPureTPB), nt = a.B * per;
        for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
            const int circ = tile / per;
            const unsigned r = (unsigned)(tile - circ * per) * kPureTPB + t;
            load_circ(a, s, circ);
            s.row[t] = -1;
            if (r < cnt) {
                const Dig y = unrank(a.C, M, tab, 0, 0, lev, r);
                const int64_t yi = box_idx(a, y);
                const int fz = first_nz(a, y);
                const double2 *F = a.F + (size_t)circ * a.n;
                double2 *Fb = a.Fbar + (size_t)circ * a.n;
                double2 acc = rscale(a.gpsi[(size_t)circ * a.n + yi], sqrt_fact(a, s, y));
                // y as the parent of y + 1_w (b term)
                for (int w = 0; w <= fz && w < M; ++w)
                    if (y(w) + 1 < a.C[w])
                        acc = cfma_conj(s.b[w], rscale(__ldcg(Fb + yi + a.stride[w]), s.inv[y(w) + 1]), acc);
                // y as the read P - 1_l of x = y + 1_l + 1_w, w <= min(fnz(y), l)
                for (int l = 0; l < M; ++l) {
                    if (y(l) + 1 >= a.C[l]) continue;
                    const int wmax = fz < l ? fz : l;
                    for (int w = 0; w <= wmax; ++w) {
                        const int pw = y(w) + (w == l ? 1 : 0);       // (y + 1_l)_w
                        if (pw + 1 >= a.C[w]) continue;
                        const double2 xb = __ldcg(Fb + yi + a.stride[l] + a.stride[w]);
                        acc = cfma_conj(s.A[w * M + l], rscale(xb, s.inv[pw + 1]), acc);
                    }
                }
                Fb[yi] = acc;
                // y as a written amplitude x: parent P = y - 1_w, w = fnz(y)
                if (fz < M) {
                    const int w = fz;
                    const int64_t pi = yi - a.stride[w];
                    const double sc = s.inv[y(w)];
                    for (int l = 0; l < M; ++l) {
                        const int Pl = y(l) - (l == w ? 1 : 0);
                        double2 v = czero();
                        if (l >= w && Pl > 0) v = cfma_conj(__ldcg(F + pi - a.stride[l]), rscale(acc, sc), v);
                        s.con[t * M + l] = v;
                    }
                    s.conb[t] = cfma_conj(__ldcg(F + pi), rscale(acc, sc), czero());
                    s.row[t] = w;
                }
            }
            __syncthreads();
            // fixed-order block reduction into this block's partial slot
            double2 *pA = a.partA + ((size_t)circ * a.grid + blockIdx.x) * M * M;
            double2 *pb = a.partb + ((size_t)circ * a.grid + blockIdx.x) * M;
            for (int e = t; e < M * M; e += blockDim.x) {
                const int w = e / M, l = e % M;
                double2 v = czero();
                for (int tt = 0; tt < kPureTPB; ++tt)
                    if (s.row[tt] == w) v = cadd(v, s.con[tt * M + l]);
                pA[e] = cadd(pA[e], v);
            }
            for (int w = t; w < M; w += blockDim.x) {
                double2 v = czero();
                for (int tt = 0; tt < kPureTPB; ++tt)
                    if (s.row[tt] == w) v = cadd(v, s.conb[tt]);
                pb[w] = cadd(pb[w], v);
            }
            __syncthreads();
        }
        if (!grid_sync(a.ctl, gridDim.x, a.timeout_ns)) return;
    }
    // dL/dA = sym(sum of partials), dL/db, dL/dc = Fbar_0
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + t;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = gtid; e < (int64_t)a.B * M * M; e += gsz) {
        const int64_t c = e / (M * M);
        const int w = (int)((e / M) % M), l = (int)(e % M);
        double2 x = czero(), y = czero();
        for (int blk = 0; blk < a.grid; ++blk) {
            const double2 *pA = a.partA + ((size_t)c * a.grid + blk) * M * M;
            x = cadd(x, pA[w * M + l]);
            y = cadd(y, pA[l * M + w]);
        }
        a.gA[e] = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y + y.y));
    }
    for (int64_t e = gtid; e < (int64_t)a.B * M; e += gsz) {
        const int64_t c = e / M;
        const int w = (int)(e % M);
        double2 x = czero();
        for (int blk = 0; blk < a.grid; ++blk) x = cadd(x, a.partb[((size_t)c * a.grid + blk) * M + w]);
        a.gb[e] = x;
    }
    for (int64_t c = gtid; c < a.B; c += gsz) a.gc[c] = a.Fbar[(size_t)c * a.n];
}

}  // namespace
}  // namespace fk

// ------------------------------------------------------------------ host
namespace fk {
namespace {

struct PureLayout {
    size_t ctl, As, bs, F, Fbar, partA, partb, total;
    int grid;
};

struct PureShape {
    int M, L;
    int C[kPureMaxM];
    int64_t stride[kPureMaxM];
    int64_t n;
};

int pure_shape(int M, const int *cutoffs, PureShape *sh)
{
    if (M < 1 || !cutoffs) return FK_EINVAL;
    if (M > kPureMaxM) return FK_EUNSUPPORTED;
    sh->M = M;
    sh->L = 0;
    int64_t n = 1;
    for (int j = M - 1; j >= 0; --j) {
        if (cutoffs[j] < 1) return FK_EINVAL;
        if (cutoffs[j] > FK_MAX_CUTOFF) return FK_EUNSUPPORTED;
        sh->C[j] = cutoffs[j];
        sh->stride[j] = n;
        n *= cutoffs[j];
        if (n >= (int64_t(1) << 31)) return FK_EUNSUPPORTED;
        sh->L += cutoffs[j] - 1;
    }
    if (sh->L > FK_MAX_LEVELS) return FK_EUNSUPPORTED;
    sh->n = n;
    return FK_OK;
}

int pure_grid(const PureShape &sh, bool vjp, int *grid)
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FK_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FK_ECUDA;
    const void *fn = vjp ? (const void *)pure_vjp_kernel : (const void *)pure_forward_kernel;
    const size_t smem = pure_smem_bytes(sh.M, sh.L);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return FK_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kPureTPB, smem) != cudaSuccess) return FK_ECUDA;
    if (per < 1) return FK_EUNSUPPORTED;
    *grid = per * sms;
    return FK_OK;
}

int pure_layout(const PureShape &sh, int batch, bool vjp, PureLayout *lay)
{
    const size_t B = (size_t)batch, M = (size_t)sh.M, c16 = 16;
    size_t o = 0;
    lay->ctl = o; o = align_up(o + sizeof(Control));
    lay->As = o; o = align_up(o + B * M * M * c16);
    lay->bs = o; o = align_up(o + B * M * c16);
    lay->F = o; o = align_up(o + B * (size_t)sh.n * c16);
    lay->grid = 0;
    lay->Fbar = lay->partA = lay->partb = o;
    if (vjp) {
        int grid = 0;
        int rc = pure_grid(sh, true, &grid);
        if (rc) return rc;
        lay->grid = grid;
        lay->Fbar = o; o = align_up(o + B * (size_t)sh.n * c16);
        lay->partA = o; o = align_up(o + B * (size_t)grid * M * M * c16);
        lay->partb = o; o = align_up(o + B * (size_t)grid * M * c16);
    }
    lay->total = o;
    return FK_OK;
}

PureArgs pure_args(const PureShape &sh, int batch, unsigned flags, const void *A, const void *b,
                   const void *c, void *ws, const PureLayout &lay)
{
    PureArgs a{};
    a.M = sh.M;
    a.L = sh.L;
    a.B = batch;
    for (int j = 0; j < sh.M; ++j) {
        a.C[j] = sh.C[j];
        a.stride[j] = sh.stride[j];
    }
    a.n = sh.n;
    a.flags = flags;
    a.A = (const double2 *)A;
    a.b = (const double2 *)b;
    a.c = (const double2 *)c;
    char *w = (char *)ws;
    a.ctl = (Control *)(w + lay.ctl);
    a.As = (double2 *)(w + lay.As);
    a.bs = (double2 *)(w + lay.bs);
    a.F = (double2 *)(w + lay.F);
    a.Fbar = (double2 *)(w + lay.Fbar);
    a.partA = (double2 *)(w + lay.partA);
    a.partb = (double2 *)(w + lay.partb);
    a.timeout_ns = kBarrierTimeoutNs;
    return a;
}

int run_forward(const PureShape &sh, int batch, unsigned flags, const void *A, const void *b,
                const void *c, void *psi, void *ws, const PureLayout &lay, cudaStream_t st)
{
    if (cudaMemsetAsync((char *)ws + lay.ctl, 0, sizeof(Control), st) != cudaSuccess) return FK_ECUDA;
    if ((flags & FK_FLAG_CHECK_FINITE) &&
        launch_check_finite(A, (int64_t)batch * sh.M * sh.M, b, (int64_t)batch * sh.M, c, batch,
                            (Control *)((char *)ws + lay.ctl), st) != FK_OK)
        return FK_ECUDA;
    PureArgs a = pure_args(sh, batch, flags, A, b, c, ws, lay);
    a.psi = (double2 *)psi;
    int grid = 0;
    int rc = pure_grid(sh, false, &grid);
    if (rc) return rc;
    a.grid = grid;
    void *params[] = {&a};
    const cudaError_t e = cudaLaunchCooperativeKernel((const void *)pure_forward_kernel, dim3(grid),
                                                      dim3(kPureTPB), params,
                                                      pure_smem_bytes(sh.M, sh.L), st);
    return e == cudaSuccess ? FK_OK : FK_ECUDA;
}

}  // namespace
}  // namespace fk

using namespace fk;

extern "C" {

int fk_pure_workspace_size(int batch, int M, const int *cutoffs, int op, unsigned flags, size_t *bytes)
{
    (void)flags;
    if (!bytes || batch < 1 || (op != FK_OP_DIAG && op != FK_OP_DIAG_VJP)) return FK_EINVAL;
    PureShape sh;
    int rc = pure_shape(M, cutoffs, &sh);
    if (rc) return rc;
    PureLayout lay;
    rc = pure_layout(sh, batch, op == FK_OP_DIAG_VJP, &lay);
    if (rc) return rc;
    *bytes = lay.total;
    return FK_OK;
}

int fock_pure_amplitudes_batched(int batch, const fk_c128 *A, const fk_c128 *b, const fk_c128 *c,
                                 int M, const int *cutoffs, fk_c128 *psi, unsigned flags, void *ws,
                                 size_t ws_bytes, void *stream)
{
    if (batch < 1 || !A || !b || !c || !psi || !ws) return FK_EINVAL;
    PureShape sh;
    int rc = pure_shape(M, cutoffs, &sh);
    if (rc) return rc;
    PureLayout lay;
    rc = pure_layout(sh, batch, false, &lay);
    if (rc) return rc;
    if (ws_bytes < lay.total || ((uintptr_t)ws & (kAlign - 1))) return FK_EWORKSPACE;
    return run_forward(sh, batch, flags, A, b, c, psi, ws, lay, (cudaStream_t)stream);
}

int fock_pure_amplitudes_vjp_batched(int batch, const fk_c128 *A, const fk_c128 *b,
                                     const fk_c128 *c, int M, const int *cutoffs,
                                     const fk_c128 *grad_psi, fk_c128 *gA, fk_c128 *gb, fk_c128 *gc,
                                     unsigned flags, void *ws, size_t ws_bytes, void *stream)
{
    if (batch < 1 || !A || !b || !c || !grad_psi || !gA || !gb || !gc || !ws) return FK_EINVAL;
    PureShape sh;
    int rc = pure_shape(M, cutoffs, &sh);
    if (rc) return rc;
    PureLayout lay;
    rc = pure_layout(sh, batch, true, &lay);
    if (rc) return rc;
    if (ws_bytes < lay.total || ((uintptr_t)ws & (kAlign - 1))) return FK_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    if (flags & FK_FLAG_RECOMPUTE) {
        // the forward's amplitudes land in the adjoint region, cleared next
        rc = run_forward(sh, batch, flags, A, b, c, (char *)ws + lay.Fbar, ws, lay, st);
        if (rc) return rc;
    }
    if (cudaMemsetAsync((char *)ws + lay.ctl, 0, sizeof(Control), st) != cudaSuccess) return FK_ECUDA;
    if ((flags & FK_FLAG_CHECK_FINITE) &&
        launch_check_finite(A, (int64_t)batch * sh.M * sh.M, b, (int64_t)batch * sh.M, c, batch,
                            (Control *)((char *)ws + lay.ctl), st) != FK_OK)
        return FK_ECUDA;
    if (cudaMemsetAsync((char *)ws + lay.Fbar, 0, lay.total - lay.Fbar, st) != cudaSuccess) return FK_ECUDA;
    PureArgs a = pure_args(sh, batch, flags, A, b, c, ws, lay);
    a.gpsi = (const double2 *)grad_psi;
    a.gA = (double2 *)gA;
    a.gb = (double2 *)gb;
    a.gc = (double2 *)gc;
    a.grid = lay.grid;
    int grid = 0;
    rc = pure_grid(sh, true, &grid);
    if (rc) return rc;
    if (grid != lay.grid) return FK_EWORKSPACE;
    void *params[] = {&a};
    const cudaError_t e = cudaLaunchCooperativeKernel((const void *)pure_vjp_kernel, dim3(grid),
                                                      dim3(kPureTPB), params,
                                                      pure_smem_bytes(sh.M, sh.L), st);
    return e == cudaSuccess ? FK_OK : FK_ECUDA;
}

}  // extern "C"
