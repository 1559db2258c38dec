/*
 * fock_oracle.c -- plain, slow, obviously-correct CPU oracle for the Fock
 * amplitude recurrence of De Prins et al., "A Quadratic Speedup in the
 * Optimization of Noisy Quantum Optical Circuits" (arXiv 2303.08879).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library.  It shares no code with
 * the CUDA path (paper_2303_08879_gb300/csrc) and includes none of its headers.
 *
 * Arithmetic: IEEE complex128 (C99 double complex), compiled without
 * fast-math and with FP contraction off, summation in the order written.
 *
 * Lattice convention: D = 2M indices; mode j owns indices 2j and 2j+1
 * (Sec. 2.1: "every pair of consecutive elements in k corresponds to a mode").
 * The library-wide reading of the pair order is G_{..m n..} = <m|rho|n>.
 *
 * What is here
 *   O1  or_full_lattice : eq. (recrel) applied to every index of the box
 *       0 <= k < dims, each amplitude written from the pivot k - 1_w with
 *       w = the first nonzero index of k; a row-major sweep visits every read
 *       and pivot before the amplitude that needs it (Sec. 2.2).
 *       Optional forward-mode tangent along one direction (dA, db, dc):
 *       eqs. (recrel_dB) and (recrel_dA) of Sec. 2.5 contracted with that
 *       direction.
 *   O2  or_walk_*       : Algorithm 1 (all modes detected, Sec. 3.1.3) and
 *       Algorithm 2 (conditional states, Sec. 3.2), written naively as a
 *       memoised recursion over the pivot each amplitude is written from.
 *       The pivot rule is the one Algorithm 1 applies (see parent_index()).
 *       Amplitudes live in a hash map keyed by the full lattice index, so
 *       nothing about the compact storage of Sec. 3.1.4 is used.
 *
 * A is symmetrised on entry, As = (A + A^T)/2: the amplitudes are the Taylor
 * coefficients of c exp(z^T A z / 2 + b^T z), which depend on As only.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define OR_MAXD 64

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_ERULE = 3 };

static void symmetrise(int D, const cplx *A, cplx *As)
{
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j)
            As[i * D + j] = 0.5 * (A[i * D + j] + A[j * D + i]);
}

static int all_zero(int D, const cplx *b)
{
    for (int i = 0; i < D; ++i)
        if (creal(b[i]) != 0.0 || cimag(b[i]) != 0.0) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* O1: the recurrence over the whole box 0 <= k < dims                       */
/* ------------------------------------------------------------------------ */
int or_full_lattice(int D, const int *dims, const cplx *A, const cplx *b, const cplx *c,
                    const cplx *dA, const cplx *db, const cplx *dc,
                    cplx *G, cplx *Gdot)
{
    if (D < 1 || D > OR_MAXD) return OR_EINVAL;
    int64_t stride[OR_MAXD];
    int64_t N = 1;
    for (int i = D - 1; i >= 0; --i) {
        if (dims[i] < 1) return OR_EINVAL;
        stride[i] = N;
        N *= dims[i];
    }
    cplx *As = malloc(sizeof(cplx) * D * D);
    cplx *dAs = malloc(sizeof(cplx) * D * D);
    if (!As || !dAs) { free(As); free(dAs); return OR_ENOMEM; }
    symmetrise(D, A, As);
    const int tangent = (Gdot != NULL);
    if (tangent) symmetrise(D, dA, dAs);

    int k[OR_MAXD];
    memset(k, 0, sizeof(k));
    for (int64_t f = 0; f < N; ++f) {
        if (f == 0) {
            G[0] = *c;
            if (tangent) Gdot[0] = *dc;
        } else {
            int w = 0;
            while (k[w] == 0) ++w;               /* first nonzero index   */
            const int64_t fP = f - stride[w];      /* pivot P = k - 1_w     */
            const int Pw = k[w] - 1;
            cplx acc = b[w] * G[fP];
            cplx tacc = 0;
            if (tangent) tacc = db[w] * G[fP] + b[w] * Gdot[fP];
            for (int l = 0; l < D; ++l) {
                const int Pl = k[l] - (l == w ? 1 : 0);
                if (Pl <= 0) continue;
                const int64_t fr = fP - stride[l];  /* read P - 1_l         */
                const double s = sqrt((double)Pl);
                acc += s * As[w * D + l] * G[fr];
                if (tangent) tacc += s * (dAs[w * D + l] * G[fr] + As[w * D + l] * Gdot[fr]);
            }
            const double den = sqrt((double)(Pw + 1));
            G[f] = acc / den;
            if (tangent) Gdot[f] = tacc / den;
        }
        /* advance the row-major multi-index */
        for (int i = D - 1; i >= 0; --i) {
            if (++k[i] < dims[i]) break;
            k[i] = 0;
        }
    }
    free(As);
    free(dAs);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* O2: naive Algorithms 1 and 2 as a memoised walk                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t key;      /* lattice code + 1; 0 marks an empty slot */
    cplx g, t;
} slot_t;

typedef struct {
    uint64_t *keys;
    uint64_t cap, used;
} keyset_t;

typedef struct {
    int M, D;
    int dims[OR_MAXD];
    uint64_t radix[OR_MAXD];
    int detected[OR_MAXD / 2];
    int has_b, has_t;
    cplx *As, *dAs, *b, *db;
    cplx c, dc;
    slot_t *tab;
    uint64_t cap, used;
    keyset_t pivots;
    int err;
    int64_t type_count[6];   /* diag, 1-ket, 1-bra, 2, 1010, 1001 (detected part) */
} walk_t;

static uint64_t mix64(uint64_t x)
{
    x ^= x >> 33; x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

static int ks_insert(keyset_t *s, uint64_t key)   /* returns 1 if new */
{
    if (2 * (s->used + 1) > s->cap) {
        uint64_t ncap = s->cap ? 2 * s->cap : 1024;
        uint64_t *nk = calloc(ncap, sizeof(uint64_t));
        if (!nk) return -1;
        for (uint64_t i = 0; i < s->cap; ++i) {
            uint64_t k = s->keys[i];
            if (!k) continue;
            uint64_t h = mix64(k) & (ncap - 1);
            while (nk[h]) h = (h + 1) & (ncap - 1);
            nk[h] = k;
        }
        free(s->keys);
        s->keys = nk;
        s->cap = ncap;
    }
    uint64_t h = mix64(key) & (s->cap - 1);
    while (s->keys[h]) {
        if (s->keys[h] == key) return 0;
        h = (h + 1) & (s->cap - 1);
    }
    s->keys[h] = key;
    s->used++;
    return 1;
}

static slot_t *tab_find(walk_t *w, uint64_t key)
{
    if (!w->cap) return NULL;
    uint64_t h = mix64(key) & (w->cap - 1);
    while (w->tab[h].key) {
        if (w->tab[h].key == key) return &w->tab[h];
        h = (h + 1) & (w->cap - 1);
    }
    return NULL;
}

static int tab_insert(walk_t *w, uint64_t key, cplx g, cplx t)
{
    if (2 * (w->used + 1) > w->cap) {
        uint64_t ncap = w->cap ? 2 * w->cap : 4096;
        slot_t *nt = calloc(ncap, sizeof(slot_t));
        if (!nt) return OR_ENOMEM;
        for (uint64_t i = 0; i < w->cap; ++i) {
            if (!w->tab[i].key) continue;
            uint64_t h = mix64(w->tab[i].key) & (ncap - 1);
            while (nt[h].key) h = (h + 1) & (ncap - 1);
            nt[h] = w->tab[i];
        }
        free(w->tab);
        w->tab = nt;
        w->cap = ncap;
    }
    uint64_t h = mix64(key) & (w->cap - 1);
    while (w->tab[h].key) h = (h + 1) & (w->cap - 1);
    w->tab[h].key = key;
    w->tab[h].g = g;
    w->tab[h].t = t;
    w->used++;
    return OR_OK;
}

static uint64_t encode(const walk_t *w, const int *x)
{
    uint64_t code = 0;
    for (int i = 0; i < w->D; ++i) code += (uint64_t)x[i] * w->radix[i];
    return code;
}

/*
 * The pivot an amplitude x is written from, P = x - 1_w; returns w.
 *
 * Detected part (Algorithm 1; App. B.2 types).  With excess e_j = x_{2j} -
 * x_{2j+1} over the detected modes j:
 *   e == 0 (diagonal d): K = first detected mode with x_{2K} > 0, w = 2K+1;
 *       P = (d - 1_K) + 1_{2K} is the off-diagonal pivot of Algorithm 1
 *       whose earlier modes are all zero.
 *   e = +1_j or -1_j (type offset_1): w = 2j or 2j+1; P is a diagonal
 *       pivot of Algorithm 1.
 *   e = +2_K (offset_2): w = 2K; e_K = +1, e_i = +1, K < i (offset_1010):
 *   w = 2i; e_K = +1, e_i = -1, K < i (offset_1001): w = 2i+1.  These are
 *   the writes of the off-diagonal pivot anchored at K.
 *   Any other pattern is not reachable from the diagonal (App. B.2: 0110
 *   does not occur) and is an error.
 * Undetected part (Algorithm 2, step 1): when every detected index is zero,
 *   w = the last nonzero undetected index.
 */
static int parent_index(walk_t *w, const int *x, int *type)
{
    int nz = 0, jj[2] = {-1, -1}, ee[2] = {0, 0};
    int any_det = 0;
    for (int j = 0; j < w->M; ++j) {
        if (!w->detected[j]) continue;
        if (x[2 * j] || x[2 * j + 1]) any_det = 1;
        const int e = x[2 * j] - x[2 * j + 1];
        if (e != 0) {
            if (nz < 2) { jj[nz] = j; ee[nz] = e; }
            ++nz;
        }
    }
    if (!any_det) {
        *type = -1;
        for (int i = w->D - 1; i >= 0; --i)
            if (!w->detected[i / 2] && x[i] > 0) return i;
        return -2;                     /* x == 0 */
    }
    if (nz == 0) {
        *type = 0;
        for (int j = 0; j < w->M; ++j)
            if (w->detected[j] && x[2 * j] > 0) return 2 * j + 1;
        return -3;
    }
    if (nz == 1) {
        if (ee[0] == 1) { *type = 1; return 2 * jj[0]; }
        if (ee[0] == -1) { *type = 2; return 2 * jj[0] + 1; }
        if (ee[0] == 2) { *type = 3; return 2 * jj[0]; }
        return -3;
    }
    if (nz == 2 && ee[0] == 1) {
        if (ee[1] == 1) { *type = 4; return 2 * jj[1]; }
        if (ee[1] == -1) { *type = 5; return 2 * jj[1] + 1; }
    }
    return -3;
}

static int walk_get(walk_t *w, int *x, cplx *g, cplx *t)
{
    const uint64_t code = encode(w, x);
    slot_t *s = tab_find(w, code + 1);
    if (s) { *g = s->g; *t = s->t; return OR_OK; }
    for (int i = 0; i < w->D; ++i)
        if (x[i] < 0 || x[i] >= w->dims[i]) return OR_ERULE;
    if (code == 0) {
        *g = w->c;
        *t = w->dc;
        w->type_count[0]++;
        return tab_insert(w, 1, *g, *t);
    }
    int type = -1;
    const int wi = parent_index(w, x, &type);
    if (wi < 0) return OR_ERULE;
    if (type >= 0) w->type_count[type]++;

    x[wi] -= 1;                                   /* x now holds the pivot P */
    if (ks_insert(&w->pivots, encode(w, x) + 1) < 0) { x[wi] += 1; return OR_ENOMEM; }
    cplx acc = 0, tacc = 0;
    int rc = OR_OK;
    if (w->has_b) {
        cplx gp, tp;
        rc = walk_get(w, x, &gp, &tp);
        if (rc) { x[wi] += 1; return rc; }
        acc += w->b[wi] * gp;
        if (w->has_t) tacc += w->db[wi] * gp + w->b[wi] * tp;
    }
    for (int l = 0; l < w->D; ++l) {
        const int Pl = x[l];
        if (Pl <= 0) continue;
        cplx gr, tr;
        x[l] -= 1;
        rc = walk_get(w, x, &gr, &tr);
        x[l] += 1;
        if (rc) { x[wi] += 1; return rc; }
        const double sq = sqrt((double)Pl);
        acc += sq * w->As[wi * w->D + l] * gr;
        if (w->has_t) tacc += sq * (w->dAs[wi * w->D + l] * gr + w->As[wi * w->D + l] * tr);
    }
    const double den = sqrt((double)(x[wi] + 1));
    x[wi] += 1;
    *g = acc / den;
    *t = w->has_t ? tacc / den : 0;
    return tab_insert(w, code + 1, *g, *t);
}

void or_walk_free(walk_t *w)
{
    if (!w) return;
    free(w->tab);
    free(w->pivots.keys);
    free(w->As); free(w->dAs); free(w->b); free(w->db);
    free(w);
}

/*
 * detected: M flags (NULL = all detected).  dA/db/dc may be NULL (no
 * tangent).  Returns NULL on bad arguments or allocation failure.
 */
walk_t *or_walk_new(int M, const int *cutoffs, const unsigned char *detected,
                    const cplx *A, const cplx *b, const cplx *c,
                    const cplx *dA, const cplx *db, const cplx *dc)
{
    if (M < 1 || 2 * M > OR_MAXD) return NULL;
    walk_t *w = calloc(1, sizeof(walk_t));
    if (!w) return NULL;
    w->M = M;
    w->D = 2 * M;
    const int D = w->D;
    uint64_t r = 1;
    for (int i = D - 1; i >= 0; --i) {
        const int C = cutoffs[i / 2];
        if (C < 1) { free(w); return NULL; }
        w->dims[i] = C;
        w->radix[i] = r;
        r *= (uint64_t)C;
    }
    for (int j = 0; j < M; ++j) w->detected[j] = detected ? (detected[j] != 0) : 1;
    w->As = malloc(sizeof(cplx) * D * D);
    w->dAs = malloc(sizeof(cplx) * D * D);
    w->b = malloc(sizeof(cplx) * D);
    w->db = malloc(sizeof(cplx) * D);
    if (!w->As || !w->dAs || !w->b || !w->db) { or_walk_free(w); return NULL; }
    symmetrise(D, A, w->As);
    memcpy(w->b, b, sizeof(cplx) * D);
    w->c = *c;
    w->has_b = !all_zero(D, b);
    w->has_t = (dA != NULL);
    if (w->has_t) {
        symmetrise(D, dA, w->dAs);
        memcpy(w->db, db, sizeof(cplx) * D);
        w->dc = *dc;
        /* a b-tangent switches the b-term on even where b itself is zero */
        if (!all_zero(D, db)) w->has_b = 1;
    } else {
        memset(w->dAs, 0, sizeof(cplx) * D * D);
        memset(w->db, 0, sizeof(cplx) * D);
        w->dc = 0;
    }
    return w;
}

/* Amplitude at one full lattice index x[D]. */
int or_walk_amplitude(walk_t *w, const int *x_in, cplx *g, cplx *t)
{
    int x[OR_MAXD];
    memcpy(x, x_in, sizeof(int) * w->D);
    cplx tt;
    return walk_get(w, x, g, t ? t : &tt);
}

/* Probability p(n) = G_{n1 n1 n2 n2 ...} (Sec. 3.1) for one pattern n[M]. */
int or_walk_prob(walk_t *w, const int *n, cplx *p, cplx *pdot)
{
    int x[OR_MAXD];
    for (int j = 0; j < w->M; ++j) x[2 * j] = x[2 * j + 1] = n[j];
    cplx tt;
    return walk_get(w, x, p, pdot ? pdot : &tt);
}

/*
 * Every probability of the all-detected case, row-major over modes
 * (mode 0 slowest).  out/out_dot hold prod C complex values.
 */
int or_walk_all_probs(walk_t *w, cplx *out, cplx *out_dot)
{
    int n[OR_MAXD / 2];
    memset(n, 0, sizeof(n));
    int64_t N = 1;
    for (int j = 0; j < w->M; ++j) N *= w->dims[2 * j];
    for (int64_t f = 0; f < N; ++f) {
        cplx p, pd;
        int rc = or_walk_prob(w, n, &p, &pd);
        if (rc) return rc;
        out[f] = p;
        if (out_dot) out_dot[f] = pd;
        for (int j = w->M - 1; j >= 0; --j) {
            if (++n[j] < w->dims[2 * j]) break;
            n[j] = 0;
        }
    }
    return OR_OK;
}

/*
 * Conditional states (Algorithm 2, any number of undetected modes).
 * out[pattern][ket][bra]: detected patterns row-major over the detected modes
 * in mode order; ket and bra multi-indices row-major over the undetected
 * modes in mode order; element = G at x with x_{2j} = x_{2j+1} = n_j for
 * detected j and (x_{2j}, x_{2j+1}) = (ket_j, bra_j) for undetected j.
 */
int or_walk_all_conditional(walk_t *w, cplx *out, cplx *out_dot)
{
    int det[OR_MAXD / 2], und[OR_MAXD / 2], nd = 0, nu = 0;
    for (int j = 0; j < w->M; ++j) {
        if (w->detected[j]) det[nd++] = j; else und[nu++] = j;
    }
    int64_t NP = 1, NU = 1;
    for (int a = 0; a < nd; ++a) NP *= w->dims[2 * det[a]];
    for (int a = 0; a < nu; ++a) NU *= w->dims[2 * und[a]];
    int x[OR_MAXD];
    int64_t f = 0;
    for (int64_t p = 0; p < NP; ++p) {
        int64_t rem = p;
        for (int a = nd - 1; a >= 0; --a) {
            const int C = w->dims[2 * det[a]];
            x[2 * det[a]] = x[2 * det[a] + 1] = (int)(rem % C);
            rem /= C;
        }
        for (int64_t kk = 0; kk < NU; ++kk) {
            int64_t rk = kk;
            for (int a = nu - 1; a >= 0; --a) {
                const int C = w->dims[2 * und[a]];
                x[2 * und[a]] = (int)(rk % C);
                rk /= C;
            }
            for (int64_t bb = 0; bb < NU; ++bb) {
                int64_t rb = bb;
                for (int a = nu - 1; a >= 0; --a) {
                    const int C = w->dims[2 * und[a]];
                    x[2 * und[a] + 1] = (int)(rb % C);
                    rb /= C;
                }
                cplx g, t;
                int rc = or_walk_amplitude(w, x, &g, &t);
                if (rc) return rc;
                out[f] = g;
                if (out_dot) out_dot[f] = t;
                ++f;
            }
        }
    }
    return OR_OK;
}

/*
 * Walk statistics: stats[0..5] = amplitudes written per detected-part type
 * (diag, offset_1 ket, offset_1 bra, offset_2, offset_1010, offset_1001 of
 * App. B.2; the vacuum counts as diagonal), stats[6] = distinct pivots,
 * stats[7] = amplitudes stored, stats[8] = amplitudes whose detected part is
 * zero (Algorithm 2, step 1; the vacuum excluded).
 */
void or_walk_stats(const walk_t *w, int64_t *stats)
{
    int64_t s = 0;
    for (int i = 0; i < 6; ++i) { stats[i] = w->type_count[i]; s += w->type_count[i]; }
    stats[6] = (int64_t)w->pivots.used;
    stats[7] = (int64_t)w->used;
    stats[8] = (int64_t)w->used - s;
}

/*
 * Per-level histogram of the stored amplitudes: hist[6*s + t] counts the
 * amplitudes of detected-part type t (as in or_walk_stats) whose total
 * weight is 2s (even types) or 2s+1 (offset_1 types); nlev rows.
 */
void or_walk_level_hist(const walk_t *w, int64_t *hist, int nlev)
{
    memset(hist, 0, sizeof(int64_t) * 6 * nlev);
    int x[OR_MAXD];
    for (uint64_t i = 0; i < w->cap; ++i) {
        if (!w->tab[i].key) continue;
        uint64_t code = w->tab[i].key - 1;
        int wsum = 0;
        for (int d = 0; d < w->D; ++d) {
            x[d] = (int)((code / w->radix[d]) % (uint64_t)w->dims[d]);
            wsum += x[d];
        }
        int type = 0;
        if (code != 0 && parent_index((walk_t *)w, x, &type) < 0) continue;
        if (code == 0) type = 0;
        if (type < 0) continue;
        const int s = wsum / 2;
        if (s < nlev) hist[6 * s + type]++;
    }
}
