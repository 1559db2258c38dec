// api.cpp -- host side of the C ABI declared in include/fockdiag.h:
// argument checking, storage geometry, workspace layout, the Gaussian ->
// Bargmann triple map, and dispatch to the CUDA launchers.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "fk_internal.h"
#include "../../include/fockdiag.h"

namespace fk {

static std::vector<int64_t> level_hist(const std::vector<int> &ext, int L);
static std::vector<int> extents(const DiagShape &sh, int k0, int a, int da, int m, int dm);

// Tile bounds of a shape (see DiagShape::max_phase_tiles): AP(K) pivots of
// level s are the vectors of family K (extents C_K - 1, C_K+1, ...) with digit
// sum s; the DP pivots are those of family 0.
static void set_tile_bounds(DiagShape *sh)
{
    const int tpbs[3] = {64, 128, 256};
    for (int i = 0; i < 3; ++i) sh->max_phase_tiles[i] = 0;
    sh->all_tiles128 = 0;
    if (sh->M == 0) return;
    std::vector<std::vector<int64_t>> h(sh->M);
    for (int K = 0; K < sh->M; ++K) h[K] = level_hist(extents(*sh, K, K, 1, -1, 0), sh->L);
    for (int s = 0; s < sh->L; ++s) {
        for (int i = 0; i < 3; ++i) {
            int64_t t = 0;
            for (int K = 0; K < sh->M; ++K) t += (h[K][s] + tpbs[i] - 1) / tpbs[i];
            if (t > sh->max_phase_tiles[i]) sh->max_phase_tiles[i] = t;
        }
        for (int K = 0; K < sh->M; ++K) sh->all_tiles128 += (h[K][s] + 127) / 128;
        if (sh->has_b) sh->all_tiles128 += (h[0][s] + 127) / 128;
    }
}

int build_diag_shape(int M, const int *cutoffs, bool has_b, DiagShape *sh)
{
    if (M < 1 || !cutoffs || !sh) return FK_EINVAL;
    std::memset(sh, 0, sizeof(*sh));
    sh->M_orig = M;
    sh->D_orig = 2 * M;
    int k = 0;
    int64_t nd = 1;
    for (int j = 0; j < M; ++j) {
        if (cutoffs[j] < 1) return FK_EINVAL;
        if (cutoffs[j] > FK_MAX_CUTOFF) return FK_EUNSUPPORTED;
        if (cutoffs[j] == 1) continue;          // index always 0: never read or written
        if (k >= FK_MAXM) return FK_EUNSUPPORTED;
        sh->C[k] = cutoffs[j];
        sh->mode_map[k] = j;
        nd *= cutoffs[j];
        if (nd >= (int64_t(1) << 31)) return FK_EUNSUPPORTED;
        ++k;
    }
    sh->M = k;
    sh->n_diag = nd;
    sh->has_b = has_b ? 1 : 0;
    int L = 0;
    for (int i = 0; i < k; ++i) L += sh->C[i] - 1;
    if (L > FK_MAX_LEVELS) return FK_EUNSUPPORTED;
    sh->L = L;
    int64_t st = 1;
    for (int i = k - 1; i >= 0; --i) {
        sh->stride[i] = st;
        st *= sh->C[i];
    }
    // amplitude boxes, concatenated: DIAG, T2(K), P1010/P1001(K,m), T1K/T1B(j).
    // P1010(K,m) and P1001(K,m) share their index space and are interleaved
    // (element i of P1010 at off + 2i, of P1001 at off + 2i + 1): a pivot
    // reads and writes both at the same index, so each 32-byte sector it
    // touches holds two of its own values.
    int64_t off = nd;
    for (int K = 0; K < k; ++K) {
        sh->off_t2[K] = off;
        off += box_size(*sh, K, K, 2, -1, 0);
    }
    for (int K = 0; K < k; ++K)
        for (int m = K + 1; m < k; ++m) {
            const int64_t n = box_size(*sh, K, K, 1, m, 1);
            sh->off_1010[K][m] = off;
            sh->off_1001[K][m] = off + 1;
            off += 2 * n;
        }
    if (has_b) {
        for (int j = 0; j < k; ++j) {
            sh->off_t1k[j] = off;
            off += box_size(*sh, 0, 0, 1, j > 0 ? j : -1, 1);
            sh->off_t1b[j] = off;
            off += (j == 0) ? box_size(*sh, 0, 0, 2, -1, 0) : box_size(*sh, 0, 0, 1, j, 1);
        }
    }
    sh->circ_size = off;
    // level-major layout (walk_diag.cu)
    int64_t lo = nd;
    for (int K = 0; K < k; ++K) {
        int64_t f = sh->C[K] - 1;
        for (int i = K + 1; i < k; ++i) f *= sh->C[i];
        sh->fam[K] = f;
    }
    for (int K = 0; K < k; ++K) {
        sh->lm_t2[K] = lo;
        lo += sh->fam[K];
    }
    for (int K = 0; K < k; ++K) {
        sh->lm_p[K] = lo;
        lo += 2 * (int64_t)(k - 1 - K) * sh->fam[K];
    }
    if (has_b)
        for (int j = 0; j < k; ++j) {
            sh->lm_t1[j] = lo;
            lo += 2 * sh->fam[0];
        }
    sh->circ_alloc = lo;
    int64_t ap = 0;
    for (int K = 0; K < k; ++K) {
        sh->off_ap[K] = ap;
        ap += box_size(*sh, K, K, 1, -1, 0);
    }
    sh->n_ap = ap;
    set_tile_bounds(sh);
    return FK_OK;
}

int diag_layout(const DiagShape &sh, int batch, bool vjp, unsigned flags, DiagLayout *lay)
{
    if (int rc = check_diag_flags(flags)) return rc;
    const size_t B = (size_t)batch, D = 2 * (size_t)sh.M;
    const size_t c16 = 16;
    size_t o = 0;
    lay->ctl = o; o = align_up(o + sizeof(Control));
    // per circuit and photon number: fixed-point sums of the probabilities (early stop)
    lay->lvl = o; o = align_up(o + B * (size_t)(sh.L + 2) * sizeof(unsigned long long));
    // tile counters of the phases (two per level for the walk, two more for
    // the tensor engine's partial pass), cleared by the kernels
    lay->ctr = o; o = align_up(o + 4 * (size_t)(sh.L + 1) * sizeof(int));
    lay->As = o; o = align_up(o + B * D * D * c16);
    lay->bs = o; o = align_up(o + B * D * c16);
    lay->dig = o; o = align_up(o + B * diag_digit_bytes(sh.M));
    lay->geo = o; o = align_up(o + diag_geo_bytes(sh));
    lay->F = o; o = align_up(o + B * (size_t)sh.circ_alloc * c16);
    lay->grid_vjp = lay->slots_vjp = 0;
    if (vjp) {
        int grid = 1, slots = 1;
        if (sh.M > 0) {
            int rc = diag_grid_size(sh, true, flags, batch, &grid, &slots);
            if (rc) return rc;
        }
        lay->grid_vjp = grid;
        lay->slots_vjp = slots;
        lay->Fbar = o; o = align_up(o + B * (size_t)sh.circ_alloc * c16);
        lay->scratch = o; o = align_up(o + B * (size_t)sh.n_ap * c16);
        lay->partA = o; o = align_up(o + B * (size_t)slots * D * D * c16);
        lay->partb = o; o = align_up(o + B * (size_t)slots * D * c16);
    } else {
        lay->Fbar = lay->scratch = lay->partA = lay->partb = o;
    }
    lay->total = o;
    return FK_OK;
}

// Number of digit vectors with the given extents summing to each s.
static std::vector<int64_t> level_hist(const std::vector<int> &ext, int L)
{
    std::vector<int64_t> h(L + 1, 0), n(L + 1, 0);
    h[0] = 1;
    for (int e : ext) {
        std::fill(n.begin(), n.end(), 0);
        for (int s = 0; s <= L; ++s)
            if (h[s])
                for (int v = 0; v < e && s + v <= L; ++v) n[s + v] += h[s];
        h.swap(n);
    }
    return h;
}

static std::vector<int> extents(const DiagShape &sh, int k0, int a, int da, int m, int dm)
{
    std::vector<int> e;
    for (int i = k0; i < sh.M; ++i) e.push_back(sh.C[i] - (i == a ? da : 0) - (i == m ? dm : 0));
    for (int &v : e) if (v < 0) v = 0;
    return e;
}

// ------------------------------------------------------------------- a0
// Gaussian state -> (A, b, c); see fk_gaussian_to_triple in fockdiag.h.
using cd = std::complex<double>;

static bool invert_and_det(int n, std::vector<cd> &a, std::vector<cd> &inv, cd *det)
{
    inv.assign((size_t)n * n, cd(0, 0));
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
    cd d = 1.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        double best = std::abs(a[(size_t)col * n + col]);
        for (int r = col + 1; r < n; ++r) {
            const double v = std::abs(a[(size_t)r * n + col]);
            if (v > best) { best = v; piv = r; }
        }
        if (!(best > 0.0)) return false;
        if (piv != col) {
            for (int c = 0; c < n; ++c) {
                std::swap(a[(size_t)piv * n + c], a[(size_t)col * n + c]);
                std::swap(inv[(size_t)piv * n + c], inv[(size_t)col * n + c]);
            }
            d = -d;
        }
        const cd p = a[(size_t)col * n + col];
        d *= p;
        for (int c = 0; c < n; ++c) {
            a[(size_t)col * n + c] /= p;
            inv[(size_t)col * n + c] /= p;
        }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const cd f = a[(size_t)r * n + col];
            if (f == cd(0, 0)) continue;
            for (int c = 0; c < n; ++c) {
                a[(size_t)r * n + c] -= f * a[(size_t)col * n + c];
                inv[(size_t)r * n + c] -= f * inv[(size_t)col * n + c];
            }
        }
    }
    *det = d;
    return true;
}

static int gaussian_to_triple(int M, const double *V, const double *mean, fk_c128 *Aout,
                              fk_c128 *bout, fk_c128 *cout)
{
    const int n = 2 * M;
    // a_j = (x_j + i p_j)/sqrt2, a^dag_j = (x_j - i p_j)/sqrt2:
    // sigma = W V W^dagger, mu = W mean with W = [[I, iI], [I, -iI]]/sqrt2.
    const double r2 = 1.0 / std::sqrt(2.0);
    std::vector<cd> W((size_t)n * n, cd(0, 0));
    for (int j = 0; j < M; ++j) {
        W[(size_t)j * n + j] = r2;
        W[(size_t)j * n + M + j] = cd(0, r2);
        W[(size_t)(M + j) * n + j] = r2;
        W[(size_t)(M + j) * n + M + j] = cd(0, -r2);
    }
    std::vector<cd> WV((size_t)n * n, 0.0), sig((size_t)n * n, 0.0), mu(n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            cd s = 0;
            for (int l = 0; l < n; ++l) s += W[(size_t)i * n + l] * V[(size_t)l * n + k];
            WV[(size_t)i * n + k] = s;
        }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            cd s = 0;
            for (int l = 0; l < n; ++l) s += WV[(size_t)i * n + l] * std::conj(W[(size_t)k * n + l]);
            sig[(size_t)i * n + k] = s;
        }
    for (int i = 0; i < n; ++i) {
        cd s = 0;
        for (int l = 0; l < n; ++l) s += W[(size_t)i * n + l] * mean[l];
        mu[i] = s;
    }
    std::vector<cd> sp = sig, sm = sig, spi;
    for (int i = 0; i < n; ++i) {
        sp[(size_t)i * n + i] += 0.5;
        sm[(size_t)i * n + i] -= 0.5;
    }
    cd det;
    std::vector<cd> tmp = sp;
    if (!invert_and_det(n, tmp, spi, &det)) return FK_EINVAL;
    // A_blk = P sm spi, b_blk = P spi mu; (P X)_{i,.} = X_{(i + M) mod 2M, .}
    std::vector<cd> Ablk((size_t)n * n, 0.0), bblk(n, 0.0);
    for (int i = 0; i < n; ++i) {
        const int pi = (i + M) % n;
        for (int k = 0; k < n; ++k) {
            cd s = 0;
            for (int l = 0; l < n; ++l) s += sm[(size_t)pi * n + l] * spi[(size_t)l * n + k];
            Ablk[(size_t)i * n + k] = s;
        }
        cd s = 0;
        for (int l = 0; l < n; ++l) s += spi[(size_t)pi * n + l] * mu[l];
        bblk[i] = s;
    }
    cd q = 0;
    for (int i = 0; i < n; ++i) {
        cd s = 0;
        for (int l = 0; l < n; ++l) s += spi[(size_t)i * n + l] * mu[l];
        q += std::conj(mu[i]) * s;
    }
    const cd c = std::exp(-0.5 * q) / std::sqrt(det);
    // lattice order: index 2j <- a^dag_j (block M + j), 2j+1 <- a_j (block j),
    // so that index 2j is the row m of <m|rho|n>.
    std::vector<int> perm(n);
    for (int j = 0; j < M; ++j) {
        perm[2 * j] = M + j;
        perm[2 * j + 1] = j;
    }
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < n; ++k) {
            const cd v = Ablk[(size_t)perm[i] * n + perm[k]];
            Aout[(size_t)i * n + k] = {v.real(), v.imag()};
        }
        bout[i] = {bblk[perm[i]].real(), bblk[perm[i]].imag()};
    }
    *cout = {c.real(), c.imag()};
    return FK_OK;
}

static bool aligned(const void *p) { return ((uintptr_t)p % kAlign) == 0; }


// ------------------------------------------------------------ global cutoff
// With a global cutoff the per-mode cutoffs are n_max (never binding below
// digit sum n_max) and the walk stops after level L = n_max - 2 of pivots:
// its DIAG writes at level L + 1 = n_max - 1 complete every pattern with
// fewer than n_max photons.  The level-major families are cut after digit
// sum L + 1, so storage grows like binomial(n_max + M, M) instead of n_max^M.
int build_global_shape(int M, int n_max, bool has_b, DiagShape *sh)
{
    if (M < 1 || n_max < 1 || !sh) return FK_EINVAL;
    if (n_max > FK_MAX_CUTOFF) return FK_EUNSUPPORTED;
    std::memset(sh, 0, sizeof(*sh));
    sh->M_orig = M;
    sh->D_orig = 2 * M;
    sh->global = 1;
    sh->has_b = has_b ? 1 : 0;
    if (n_max == 1) {               // vacuum only
        sh->M = 0;
        sh->n_diag = 1;
        sh->circ_size = sh->circ_alloc = 1;
        return FK_OK;
    }
    if (M > FK_MAXM) return FK_EUNSUPPORTED;
    sh->M = M;
    for (int j = 0; j < M; ++j) {
        sh->C[j] = n_max;
        sh->mode_map[j] = j;
    }
    const int L = n_max - 1;        // pivot levels 0..L-1, stored digit sums 0..L
    if (L > FK_MAX_LEVELS) return FK_EUNSUPPORTED;
    sh->L = L;
    auto total = [&](const std::vector<int64_t> &h) {
        int64_t n = 0;
        for (int t = 0; t <= L; ++t) n += h[t];
        return n;
    };
    std::vector<int> full(M, n_max);
    const int64_t nd = total(level_hist(full, L));
    if (nd >= (int64_t(1) << 31)) return FK_EUNSUPPORTED;
    sh->n_diag = nd;
    int64_t lo = nd;
    for (int K = 0; K < M; ++K) sh->fam[K] = total(level_hist(extents(*sh, K, K, 1, -1, 0), L));
    for (int K = 0; K < M; ++K) {
        sh->lm_t2[K] = lo;
        lo += sh->fam[K];
    }
    for (int K = 0; K < M; ++K) {
        sh->lm_p[K] = lo;
        lo += 2 * (int64_t)(M - 1 - K) * sh->fam[K];
    }
    if (has_b)
        for (int j = 0; j < M; ++j) {
            sh->lm_t1[j] = lo;
            lo += 2 * sh->fam[0];
        }
    sh->circ_size = sh->circ_alloc = lo;
    int64_t ap = 0;
    for (int K = 0; K < M; ++K) {
        sh->off_ap[K] = ap;
        ap += sh->fam[K];
    }
    sh->n_ap = ap;
    set_tile_bounds(sh);
    return FK_OK;
}

// Position of a pattern in the level-major output (digit sum, then
// lexicographic with mode 0 slowest); -1 if its photon number is >= n_max.
static int64_t global_index(int M, int n_max, const int *n)
{
    int s = 0;
    for (int j = 0; j < M; ++j) {
        if (n[j] < 0) return -1;
        s += n[j];
    }
    if (s >= n_max) return -1;
    // W[i][t]: vectors over modes i..M-1 (digits < n_max) with digit sum t
    std::vector<std::vector<int64_t>> W(M + 1, std::vector<int64_t>(n_max, 0));
    W[M][0] = 1;
    for (int i = M - 1; i >= 0; --i)
        for (int t = 0; t < n_max; ++t)
            for (int v = 0; v <= t && v < n_max; ++v) W[i][t] += W[i + 1][t - v];
    int64_t idx = 0;
    for (int t = 0; t < s; ++t) idx += W[0][t];
    int rem = s;
    for (int i = 0; i < M; ++i) {
        for (int v = 0; v < n[i]; ++v) idx += W[i + 1][rem - v];
        rem -= n[i];
    }
    return idx;
}

}  // namespace fk

using namespace fk;

extern "C" {

const char *fk_status_string(int status)
{
    switch (status) {
    case FK_OK: return "ok";
    case FK_EINVAL: return "invalid argument";
    case FK_EUNSUPPORTED: return "size beyond compiled limits";
    case FK_EWORKSPACE: return "workspace too small or misaligned";
    case FK_ENOMEM: return "host allocation failed";
    case FK_ECUDA: return "CUDA runtime error";
    case FK_ETIMEOUT: return "device barrier wait timed out";
    case FK_ENONFINITE: return "non-finite input";
    case FK_EBZERO: return "FK_FLAG_B_ZERO given but b is nonzero";
    default: return "unknown status";
    }
}

int fk_version(void) { return 100; }

int fk_gaussian_to_triple(int M, const double *V, const double *mean, fk_c128 *A, fk_c128 *b,
                          fk_c128 *c)
{
    if (M < 1 || M > 64 || !V || !mean || !A || !b || !c) return FK_EINVAL;
    try {
        return gaussian_to_triple(M, V, mean, A, b, c);
    } catch (...) {
        return FK_ENOMEM;
    }
}

int fk_workspace_size(int M, const int *cutoffs, const unsigned char *mask, int batch, int op,
                      unsigned flags, size_t *bytes)
{
    (void)mask;
    if (!bytes || batch < 1) return FK_EINVAL;
    if (op == FK_OP_DIAG || op == FK_OP_DIAG_VJP) {
        DiagShape sh;
        int rc = build_diag_shape(M, cutoffs, !(flags & FK_FLAG_B_ZERO), &sh);
        if (rc) return rc;
        DiagLayout lay;
        rc = diag_layout(sh, batch, op == FK_OP_DIAG_VJP, flags, &lay);
        if (rc) return rc;
        *bytes = lay.total;
        return FK_OK;
    }
    if (op == FK_OP_COND || op == FK_OP_COND_VJP) {
        if (!cutoffs || !mask) return FK_EINVAL;
        std::vector<int> cut((size_t)batch * M);
        for (int i = 0; i < batch; ++i)
            for (int j = 0; j < M; ++j) cut[(size_t)i * M + j] = cutoffs[j];
        return fk_conditional_workspace_size(batch, M, cut.data(), mask, op, flags, bytes, nullptr);
    }
    return FK_EUNSUPPORTED;
}

int fk_conditional_workspace_size(int batch, int M, const int *cutoffs, const unsigned char *mask,
                                  int op, unsigned flags, size_t *bytes, int64_t *rho_offsets)
{
    if (!bytes || (op != FK_OP_COND && op != FK_OP_COND_VJP)) return FK_EINVAL;
    const CondPlan *plan = nullptr;
    int rc = get_cond_plan(batch, M, cutoffs, mask, &plan);
    if (rc) return rc;
    CondLayout lay;
    rc = cond_layout(*plan, op == FK_OP_COND_VJP, flags, &lay);
    if (rc) return rc;
    *bytes = lay.total;
    if (rho_offsets) {
        int64_t off = 0;
        for (int i = 0; i < batch; ++i) {
            rho_offsets[i] = off;
            int64_t np = 1, nu = 1;
            for (int j = 0; j < M; ++j) {
                const int C = cutoffs[(size_t)i * M + j];
                if (mask[j]) np *= C; else nu *= C;
            }
            off += np * nu * nu;
        }
        rho_offsets[batch] = off;
    }
    return FK_OK;
}

int fock_conditional_dm_batched(int batch, const fk_c128 *A, const fk_c128 *b, const fk_c128 *c,
                                int M, const int *cutoffs, const unsigned char *mask, fk_c128 *rho,
                                unsigned flags, void *ws, size_t ws_bytes, void *stream)
{
    if (batch < 1 || !A || !b || !c || !rho || !ws || !cutoffs || !mask) return FK_EINVAL;
    const CondPlan *plan = nullptr;
    int rc = get_cond_plan(batch, M, cutoffs, mask, &plan);
    if (rc) return rc;
    CondLayout lay;
    rc = cond_layout(*plan, false, flags, &lay);
    if (rc) return rc;
    if (ws_bytes < lay.total || !aligned(ws)) return FK_EWORKSPACE;
    return launch_cond_forward(*plan, flags, A, b, c, rho, ws, lay, stream);
}

int fock_conditional_dm(const fk_c128 *A, const fk_c128 *b, const fk_c128 *c, int M,
                        const int *cutoffs, const unsigned char *mask, fk_c128 *rho, void *ws,
                        size_t ws_bytes, void *stream)
{
    return fock_conditional_dm_batched(1, A, b, c, M, cutoffs, mask, rho, 0u, ws, ws_bytes, stream);
}

int fock_conditional_dm_vjp_batched(int batch, const fk_c128 *A, const fk_c128 *b,
                                    const fk_c128 *c, int M, const int *cutoffs,
                                    const unsigned char *mask, const fk_c128 *grho, fk_c128 *gA,
                                    fk_c128 *gb, fk_c128 *gc, unsigned flags, void *ws,
                                    size_t ws_bytes, void *stream)
{
    if (batch < 1 || !A || !b || !c || !grho || !gA || !gb || !gc || !ws || !cutoffs || !mask)
        return FK_EINVAL;
    const CondPlan *plan = nullptr;
    int rc = get_cond_plan(batch, M, cutoffs, mask, &plan);
    if (rc) return rc;
    CondLayout lay;
    rc = cond_layout(*plan, true, flags, &lay);
    if (rc) return rc;
    if (ws_bytes < lay.total || !aligned(ws)) return FK_EWORKSPACE;
    if (flags & FK_FLAG_RECOMPUTE) {
        // the forward's output lands in the adjoint region, cleared next
        void *tmp = (char *)ws + lay.Fbar;
        if ((size_t)plan->rho_total * 16 > lay.partA - lay.Fbar) return FK_EWORKSPACE;
        rc = launch_cond_forward(*plan, flags, A, b, c, tmp, ws, lay, stream);
        if (rc) return rc;
    }
    return launch_cond_vjp(*plan, flags, A, b, c, grho, gA, gb, gc, ws, lay, stream);
}

int fock_conditional_dm_vjp(const fk_c128 *A, const fk_c128 *b, const fk_c128 *c, int M,
                            const int *cutoffs, const unsigned char *mask, const fk_c128 *grho,
                            fk_c128 *gA, fk_c128 *gb, fk_c128 *gc, void *ws, size_t ws_bytes,
                            void *stream)
{
    return fock_conditional_dm_vjp_batched(1, A, b, c, M, cutoffs, mask, grho, gA, gb, gc, 0u, ws,
                                           ws_bytes, stream);
}

int fock_diag_probs_batched(int batch, const fk_c128 *A, const fk_c128 *b, const fk_c128 *c,
                            int M, const int *cutoffs, fk_c128 *probs, unsigned flags, void *ws,
                            size_t ws_bytes, void *stream)
{
    if (batch < 1 || !A || !b || !c || !probs || !ws) return FK_EINVAL;
    DiagShape sh;
    int rc = build_diag_shape(M, cutoffs, !(flags & FK_FLAG_B_ZERO), &sh);
    if (rc) return rc;
    DiagLayout lay;
    rc = diag_layout(sh, batch, false, flags, &lay);
    if (rc) return rc;
    if (ws_bytes < lay.total || !aligned(ws)) return FK_EWORKSPACE;
    return launch_diag_forward(sh, batch, flags, A, b, c, probs, ws, lay, stream);
}

int fock_diag_probs(const fk_c128 *A, const fk_c128 *b, const fk_c128 *c, int M,
                    const int *cutoffs, fk_c128 *probs, void *ws, size_t ws_bytes, void *stream)
{
    return fock_diag_probs_batched(1, A, b, c, M, cutoffs, probs, 0u, ws, ws_bytes, stream);
}

int fock_diag_probs_vjp_batched(int batch, const fk_c128 *A, const fk_c128 *b, const fk_c128 *c,
                                int M, const int *cutoffs, const fk_c128 *gprobs, fk_c128 *gA,
                                fk_c128 *gb, fk_c128 *gc, unsigned flags, void *ws,
                                size_t ws_bytes, void *stream)
{
    if (batch < 1 || !A || !b || !c || !gprobs || !gA || !gb || !gc || !ws) return FK_EINVAL;
    DiagShape sh;
    int rc = build_diag_shape(M, cutoffs, !(flags & FK_FLAG_B_ZERO), &sh);
    if (rc) return rc;
    DiagLayout lay;
    rc = diag_layout(sh, batch, true, flags, &lay);
    if (rc) return rc;
    if (ws_bytes < lay.total || !aligned(ws)) return FK_EWORKSPACE;
    if (flags & FK_FLAG_RECOMPUTE) {
        // the forward's probabilities land in the adjoint region, cleared next
        void *tmp = (char *)ws + lay.Fbar;
        rc = launch_diag_forward(sh, batch, flags, A, b, c, tmp, ws, lay, stream);
        if (rc) return rc;
    }
    return launch_diag_vjp(sh, batch, flags, A, b, c, gprobs, gA, gb, gc, ws, lay, stream);
}

int fock_diag_probs_vjp(const fk_c128 *A, const fk_c128 *b, const fk_c128 *c, int M,
                        const int *cutoffs, const fk_c128 *gprobs, fk_c128 *gA, fk_c128 *gb,
                        fk_c128 *gc, void *ws, size_t ws_bytes, void *stream)
{
    return fock_diag_probs_vjp_batched(1, A, b, c, M, cutoffs, gprobs, gA, gb, gc, 0u, ws,
                                       ws_bytes, stream);
}

int fk_diag_set_tuning(int tpb, int ch, int blocks_per_sm)
{
    return set_diag_tuning(tpb, ch, blocks_per_sm);
}

int fk_diag_set_engine(int engine)
{
    return set_diag_engine(engine);
}

int fk_diag_tuning_flags(int engine, int tpb, int ch, int blocks_per_sm, unsigned *flags_out)
{
    return diag_tuning_flags(engine, tpb, ch, blocks_per_sm, flags_out);
}

int fk_diag_set_vjp_split_event(void *event)
{
    return set_vjp_split_event(event);
}

int fk_workspace_status(const void *ws, void *stream, int *status)
{
    if (!ws || !status) return FK_EINVAL;
    return read_status(ws, stream, status);
}

int fk_debug_checks(void)
{
#ifdef FK_DEBUG_CHECKS
    return 1;
#else
    return 0;
#endif
}

int fk_workspace_debug(const void *ws, void *stream, long long *out)
{
    if (!ws || !out) return FK_EINVAL;
    return read_debug(ws, stream, out);
}

int fk_debug_set_trace(unsigned long long *d_buf, int capacity)
{
    return set_debug_trace(d_buf, capacity);
}

int fk_selftest_wait_timeout(void *ws, size_t ws_bytes, unsigned long long timeout_ns, void *stream)
{
    if (!ws || ws_bytes < sizeof(Control) || !aligned(ws)) return FK_EWORKSPACE;
    return launch_wait_selftest(ws, timeout_ns, stream);
}

int fk_describe_diag_schedule(int M, const int *cutoffs, unsigned flags, int64_t *out, int out_len)
{
    if (!out || out_len < 3) return FK_EINVAL;
    DiagShape sh;
    int rc = build_diag_shape(M, cutoffs, !(flags & FK_FLAG_B_ZERO), &sh);
    if (rc) return rc;
    const int L = sh.L;
    std::vector<int64_t> rows((size_t)6 * (L + 1), 0);
    auto add = [&](int col, const std::vector<int64_t> &h, int shift) {
        for (int s = 0; s <= L; ++s) {
            const int lev = s + shift;
            if (lev >= 0 && lev <= L) rows[(size_t)6 * lev + col] += h[s];
        }
    };
    int64_t pivots = 0;
    const int k = sh.M;
    add(0, level_hist(extents(sh, 0, -1, 0, -1, 0), L), 0);
    for (int K = 0; K < k; ++K) {
        add(2, level_hist(extents(sh, K, K, 2, -1, 0), L), 1);
        for (int m = K + 1; m < k; ++m) {
            const auto h = level_hist(extents(sh, K, K, 1, m, 1), L);
            add(3, h, 1);
            add(4, h, 1);
        }
        const auto hp = level_hist(extents(sh, K, K, 1, -1, 0), L);
        add(5, hp, 0);
        for (auto v : hp) pivots += v;
    }
    if (sh.has_b && k > 0) {
        for (int j = 0; j < k; ++j) {
            add(1, level_hist(extents(sh, 0, 0, 1, j > 0 ? j : -1, 1), L), 0);
            add(1, level_hist(j == 0 ? extents(sh, 0, 0, 2, -1, 0) : extents(sh, 0, 0, 1, j, 1), L), 0);
        }
        const auto hd = level_hist(extents(sh, 0, 0, 1, -1, 0), L);
        add(5, hd, 0);
        for (auto v : hd) pivots += v;
    }
    out[0] = sh.circ_size;
    out[1] = pivots;
    out[2] = L + 1;
    for (int i = 0; i < (int)rows.size() && 3 + i < out_len; ++i) out[3 + i] = rows[i];
    return FK_OK;
}


int fk_global_size(int M, int n_max, int64_t *count)
{
    if (!count) return FK_EINVAL;
    DiagShape sh;
    int rc = build_global_shape(M, n_max, false, &sh);
    if (rc) return rc;
    *count = sh.n_diag;
    return FK_OK;
}

int fk_global_pattern_index(int M, int n_max, const int *pattern, int64_t *index)
{
    if (M < 1 || n_max < 1 || !pattern || !index) return FK_EINVAL;
    *index = global_index(M, n_max, pattern);
    return FK_OK;
}

int fk_global_workspace_size(int batch, int M, int n_max, int op, unsigned flags, size_t *bytes)
{
    if (!bytes || batch < 1 || (op != FK_OP_DIAG && op != FK_OP_DIAG_VJP)) return FK_EINVAL;
    DiagShape sh;
    int rc = build_global_shape(M, n_max, !(flags & FK_FLAG_B_ZERO), &sh);
    if (rc) return rc;
    DiagLayout lay;
    rc = diag_layout(sh, batch, op == FK_OP_DIAG_VJP, flags, &lay);
    if (rc) return rc;
    *bytes = lay.total;
    return FK_OK;
}

int fock_diag_probs_global_batched(int batch, const fk_c128 *A, const fk_c128 *b, const fk_c128 *c,
                                   int M, int n_max, fk_c128 *probs, unsigned flags, void *ws,
                                   size_t ws_bytes, void *stream)
{
    if (batch < 1 || !A || !b || !c || !probs || !ws) return FK_EINVAL;
    DiagShape sh;
    int rc = build_global_shape(M, n_max, !(flags & FK_FLAG_B_ZERO), &sh);
    if (rc) return rc;
    DiagLayout lay;
    rc = diag_layout(sh, batch, false, flags, &lay);
    if (rc) return rc;
    if (ws_bytes < lay.total || !aligned(ws)) return FK_EWORKSPACE;
    return launch_diag_forward(sh, batch, flags, A, b, c, probs, ws, lay, stream);
}

int fock_diag_probs_global_vjp_batched(int batch, const fk_c128 *A, const fk_c128 *b,
                                       const fk_c128 *c, int M, int n_max, const fk_c128 *gprobs,
                                       fk_c128 *gA, fk_c128 *gb, fk_c128 *gc, unsigned flags,
                                       void *ws, size_t ws_bytes, void *stream)
{
    if (batch < 1 || !A || !b || !c || !gprobs || !gA || !gb || !gc || !ws) return FK_EINVAL;
    DiagShape sh;
    int rc = build_global_shape(M, n_max, !(flags & FK_FLAG_B_ZERO), &sh);
    if (rc) return rc;
    DiagLayout lay;
    rc = diag_layout(sh, batch, true, flags, &lay);
    if (rc) return rc;
    if (ws_bytes < lay.total || !aligned(ws)) return FK_EWORKSPACE;
    if (flags & FK_FLAG_RECOMPUTE) {
        void *tmp = (char *)ws + lay.Fbar;
        rc = launch_diag_forward(sh, batch, flags, A, b, c, tmp, ws, lay, stream);
        if (rc) return rc;
    }
    return launch_diag_vjp(sh, batch, flags, A, b, c, gprobs, gA, gb, gc, ws, lay, stream);
}

int fk_describe_global_schedule(int M, int n_max, unsigned flags, int64_t *out, int out_len)
{
    if (!out || out_len < 3) return FK_EINVAL;
    DiagShape sh;
    int rc = build_global_shape(M, n_max, !(flags & FK_FLAG_B_ZERO), &sh);
    if (rc) return rc;
    int64_t pivots = 0;
    for (int K = 0; K < sh.M; ++K) {
        const auto h = level_hist(extents(sh, K, K, 1, -1, 0), sh.L);
        for (int s = 0; s < sh.L; ++s) pivots += h[s];
    }
    if (sh.has_b && sh.M > 0) {
        const auto h = level_hist(extents(sh, 0, 0, 1, -1, 0), sh.L);
        for (int s = 0; s < sh.L; ++s) pivots += h[s];
    }
    out[0] = sh.circ_alloc;
    out[1] = pivots;
    out[2] = sh.n_diag;
    return FK_OK;
}


int fock_diag_probs_stop_batched(int batch, const fk_c128 *A, const fk_c128 *b, const fk_c128 *c,
                                 int M, const int *cutoffs, double eps, fk_c128 *probs, int *levels,
                                 unsigned flags, void *ws, size_t ws_bytes, void *stream)
{
    if (batch < 1 || !A || !b || !c || !probs || !ws || !(eps >= 0.0 && eps <= 1.0)) return FK_EINVAL;
    DiagShape sh;
    int rc = build_diag_shape(M, cutoffs, !(flags & FK_FLAG_B_ZERO), &sh);
    if (rc) return rc;
    DiagLayout lay;
    rc = diag_layout(sh, batch, false, flags, &lay);
    if (rc) return rc;
    if (ws_bytes < lay.total || !aligned(ws)) return FK_EWORKSPACE;
    const EarlyStop es{eps, levels};
    return launch_diag_forward(sh, batch, flags, A, b, c, probs, ws, lay, stream, &es);
}

int fock_diag_probs_stop_vjp_batched(int batch, const fk_c128 *A, const fk_c128 *b,
                                     const fk_c128 *c, int M, const int *cutoffs, double eps,
                                     const fk_c128 *gprobs, fk_c128 *gA, fk_c128 *gb, fk_c128 *gc,
                                     unsigned flags, void *ws, size_t ws_bytes, void *stream)
{
    if (batch < 1 || !A || !b || !c || !gprobs || !gA || !gb || !gc || !ws || !(eps >= 0.0 && eps <= 1.0))
        return FK_EINVAL;
    DiagShape sh;
    int rc = build_diag_shape(M, cutoffs, !(flags & FK_FLAG_B_ZERO), &sh);
    if (rc) return rc;
    DiagLayout lay;
    rc = diag_layout(sh, batch, true, flags, &lay);
    if (rc) return rc;
    if (ws_bytes < lay.total || !aligned(ws)) return FK_EWORKSPACE;
    const EarlyStop es{eps, nullptr};
    if (flags & FK_FLAG_RECOMPUTE) {
        void *tmp = (char *)ws + lay.Fbar;
        rc = launch_diag_forward(sh, batch, flags, A, b, c, tmp, ws, lay, stream, &es);
        if (rc) return rc;
    }
    return launch_diag_vjp(sh, batch, flags, A, b, c, gprobs, gA, gb, gc, ws, lay, stream, &es);
}


int fk_gaussian_to_pure_triple(int M, const double *V, const double *mean, fk_c128 *A, fk_c128 *b,
                               fk_c128 *c)
{
    if (M < 1 || M > 64 || !V || !mean || !A || !b || !c) return FK_EINVAL;
    const int D = 2 * M;
    std::vector<fk_c128> Ar((size_t)D * D), br(D);
    fk_c128 cr;
    int rc;
    try {
        rc = gaussian_to_triple(M, V, mean, Ar.data(), br.data(), &cr);
    } catch (...) {
        return FK_ENOMEM;
    }
    if (rc) return rc;
    // a pure state's density triple has no ket-bra coupling: A_rho = A_psi (+) conj(A_psi)
    double amax = 0.0, cross = 0.0;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            const fk_c128 v = Ar[(size_t)i * D + j];
            const double m = std::hypot(v.re, v.im);
            amax = std::max(amax, m);
            if ((i & 1) != (j & 1)) cross = std::max(cross, m);
        }
    if (cross > 1e-9 * std::max(amax, 1.0) || !(cr.re > 0.0)) return FK_EINVAL;
    for (int i = 0; i < M; ++i) {
        for (int j = 0; j < M; ++j) A[(size_t)i * M + j] = Ar[(size_t)(2 * i) * D + 2 * j];
        b[i] = br[2 * i];
    }
    c->re = std::sqrt(cr.re);   // psi_0 = sqrt(rho_0) up to a global phase (Sec. 2.2)
    c->im = 0.0;
    return FK_OK;
}

}  // extern "C"

// ----------------------------------------------- per-circuit cutoffs (several shapes)
extern "C" {

int fk_multi_workspace_size(int batch, int M, const int *cutoffs, int op, unsigned flags, size_t *bytes,
                            int64_t *out_offsets)
{
    if (!bytes || (op != FK_OP_DIAG && op != FK_OP_DIAG_VJP)) return FK_EINVAL;
    const MultiPlan *p = nullptr;
    int rc = get_multi_plan(batch, M, cutoffs, flags, &p);
    if (rc) return rc;
    *bytes = op == FK_OP_DIAG_VJP ? p->total_vjp : p->total_fwd;
    if (out_offsets)
        for (int i = 0; i <= batch; ++i) out_offsets[i] = p->out_offsets[i];
    return FK_OK;
}

int fock_diag_probs_multi_batched(int batch, const fk_c128 *A, const fk_c128 *b, const fk_c128 *c, int M,
                                  const int *cutoffs, fk_c128 *probs, unsigned flags, void *ws,
                                  size_t ws_bytes, void *stream)
{
    if (batch < 1 || !A || !b || !c || !probs || !ws) return FK_EINVAL;
    const MultiPlan *p = nullptr;
    int rc = get_multi_plan(batch, M, cutoffs, flags, &p);
    if (rc) return rc;
    if (ws_bytes < p->total_fwd || !aligned(ws)) return FK_EWORKSPACE;
    return launch_multi_forward(*p, flags, A, b, c, probs, ws, stream);
}

int fock_diag_probs_multi_vjp_batched(int batch, const fk_c128 *A, const fk_c128 *b, const fk_c128 *c,
                                      int M, const int *cutoffs, const fk_c128 *gprobs, fk_c128 *gA,
                                      fk_c128 *gb, fk_c128 *gc, unsigned flags, void *ws, size_t ws_bytes,
                                      void *stream)
{
    if (batch < 1 || !A || !b || !c || !gprobs || !gA || !gb || !gc || !ws) return FK_EINVAL;
    const MultiPlan *p = nullptr;
    int rc = get_multi_plan(batch, M, cutoffs, flags, &p);
    if (rc) return rc;
    if (ws_bytes < p->total_vjp || !aligned(ws)) return FK_EWORKSPACE;
    if (flags & FK_FLAG_RECOMPUTE) {
        // the forward's probabilities land in the adjoint region, which the
        // VJP either clears (b != 0) or overwrites before reading (b = 0)
        if ((size_t)p->n_out * 16 > p->total_vjp - p->off_vjp) return FK_EWORKSPACE;
        rc = launch_multi_forward(*p, flags, A, b, c, (char *)ws + p->off_vjp, ws, stream);
        if (rc) return rc;
    }
    return launch_multi_vjp(*p, flags, A, b, c, gprobs, gA, gb, gc, ws, stream);
}

}  // extern "C"
