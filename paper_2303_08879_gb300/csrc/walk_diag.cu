// walk_diag.cu -- host side of the all-detected walk (Algorithm 1 of arXiv
// 2303.08879, Sec. 3.1) and its adjoint: tuning, grid sizing and the
// launchers of the persistent kernels of walk_diag_impl.cuh (instantiated
// in walk_diag_fp64.cu and walk_diag_tc*.cu), plus the small helper
// kernels (vacuum problems, the input scan, the bounded-wait self-test).
#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>

#include "walk_diag_impl.cuh"

namespace fk {

namespace {

__global__ void copy_c_kernel(const double2 *c, double2 *probs, int B, int64_t stride)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B) probs[(size_t)i * stride] = c[i];
}

__global__ void vacuum_vjp_kernel(const double2 *gprobs, double2 *gA, double2 *gb, double2 *gc,
                                  int B, int Do)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B * Do * Do) gA[i] = make_double2(0, 0);
    if (i < B * Do) gb[i] = make_double2(0, 0);
    if (i < B) gc[i] = gprobs[i];
}

__global__ void fill_int_kernel(int *p, int n, int v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// NaN or Inf in any of the complex inputs: exponent field all ones.
__global__ void check_finite_kernel(const unsigned long long *A, int64_t nA, const unsigned long long *b,
                                    int64_t nb, const unsigned long long *c, int64_t nc, Control *ctl)
{
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    constexpr unsigned long long kExp = 0x7ff0000000000000ull;
    int bad = 0;
    for (int64_t i = gtid; i < 2 * nA; i += gsz) bad |= (A[i] & kExp) == kExp;
    for (int64_t i = gtid; i < 2 * nb; i += gsz) bad |= (b[i] & kExp) == kExp;
    for (int64_t i = gtid; i < 2 * nc; i += gsz) bad |= (c[i] & kExp) == kExp;
    if (__syncthreads_or(bad) && threadIdx.x == 0) {
        atomicCAS(&ctl->status, 0, (int)FK_ENONFINITE);
        atomicExch(&ctl->skip, 1);
    }
}

__global__ void wait_selftest_kernel(Control *ctl, unsigned long long timeout_ns)
{
    if (threadIdx.x != 0) return;
    const unsigned long long t0 = gtimer();
    while (ld_acquire(&ctl->wait_flag) == 0u) {
        if (gtimer() - t0 > timeout_ns) {
            atomicCAS(&ctl->status, 0, (int)FK_ETIMEOUT);
            return;
        }
        __nanosleep(256);
    }
}

// ---------------------------------------------------------- host plumbing
struct GridCache {
    std::mutex mu;
    int dev = -1, sms = 0;
};
GridCache g_cache;

int device_sms(int *sms)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FK_ECUDA;
    std::lock_guard<std::mutex> lk(g_cache.mu);
    if (g_cache.dev != dev) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FK_ECUDA;
        g_cache.dev = dev;
        g_cache.sms = n;
    }
    *sms = g_cache.sms;
    return FK_OK;
}

// Compiled tile shapes (pivots per tile, output rows per register chunk) of
// the FP64 engine and the tensor-core kernels by KS = ceil(M / 4) (M <= 12;
// 128 pivots per tile; the VJP is two launches: the reverse walk, then the
// partial pass).
using Variant = WalkKernels;
struct VariantTable {
    Variant v[kNumFp64Shapes];
    const Variant *tc[3] = {nullptr, nullptr, nullptr};
    VariantTable()
    {
        v[0] = *fp64_walk_kernels_128_8();
        v[1] = *fp64_walk_kernels_128_4();
        v[2] = *fp64_walk_kernels_64_8();
        v[3] = *fp64_walk_kernels_64_4();
        v[4] = *fp64_walk_kernels_256_8();
        tc[0] = tc1_walk_kernels();
        tc[1] = tc2_walk_kernels();
        tc[2] = tc3_walk_kernels();
    }
};
const VariantTable &tables()
{
    static const VariantTable t;
    return t;
}
constexpr int kTcMaxModes = 12;

// Process-wide defaults (fk_diag_set_tuning, fk_diag_set_engine), read once
// per call under the lock; per-call flag bits override them.
std::mutex g_tune_mu;
int g_tpb = 128, g_ch = 8, g_bps = 0, g_engine = FK_ENGINE_AUTO;

// The tuning one call runs with.
struct Tune {
    int tpb, ch, bps, engine;
};

constexpr int kNumVariants = kNumFp64Shapes;

Tune resolve_tune(unsigned flags)
{
    Tune t;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        t = Tune{g_tpb, g_ch, g_bps, g_engine};
    }
    if (flags & FK_FLAG_ENGINE_FP64) t.engine = FK_ENGINE_FP64;
    if (flags & FK_FLAG_ENGINE_TENSOR) t.engine = FK_ENGINE_TENSOR;
    const int v = (int)((flags >> 8) & 15u);
    if (v >= 1 && v <= kNumVariants) {
        t.tpb = tables().v[v - 1].tpb;
        t.ch = tables().v[v - 1].ch;
        t.bps = (int)((flags >> 12) & 63u);
    }
    return t;
}

const Variant &variant_of(const Tune &t)
{
    for (int i = 0; i < kNumVariants; ++i)
        if (tables().v[i].tpb == t.tpb && tables().v[i].ch == t.ch) return tables().v[i];
    return tables().v[0];
}

bool tc_engine_for(const DiagShape &sh, const Tune &t)
{
    return t.engine != FK_ENGINE_FP64 && sh.M <= kTcMaxModes;
}

// Kernel, block size, shared memory and partial-sum slots per block for
// shape sh under tuning t: the forward (vjp false) or the VJP launch that
// owns the partial-sum slots (vjp true: the FP64 engine's reverse walk, the
// tensor engine's partial pass).  tc_walk: the tensor engine's reverse walk
// instead.
void walk_kernel(const DiagShape &sh, const Tune &t, bool vjp, const void **fn, int *tpb, size_t *smem,
                 int *bps, int *slots_per_block, bool tc_walk = false)
{
    const Variant &v = variant_of(t);
    *bps = t.bps;
    if (tc_engine_for(sh, t)) {
        const Variant &tc = *tables().tc[(sh.M + 3) / 4 - 1];
        const int mode = tc_walk ? kVjp : (vjp ? kPart : kFwd);
        *fn = tc_walk ? tc.vjp : (vjp ? tc.part : tc.fwd);
        *tpb = 128;
        *smem = tc.smem(sh.M, sh.L, mode, sh.has_b != 0);
        *slots_per_block = 128 / 32;
        return;
    }
    *fn = vjp ? v.vjp : v.fwd;
    *tpb = v.tpb;
    *smem = v.smem(sh.M, sh.L, vjp ? kVjp : kFwd, sh.has_b != 0);
    *slots_per_block = 1;
}

}  // namespace

namespace {
std::mutex g_split_mu;
void *g_split_event = nullptr;   // cudaEvent_t recorded between the two VJP launches
// debug-checks build: caller-registered buffer of per-level timestamps
std::mutex g_trace_mu;
unsigned long long *g_trace = nullptr;
int g_trace_cap = 0;

void attach_trace(DiagArgs &a)
{
    std::lock_guard<std::mutex> lk(g_trace_mu);
    a.trace = g_trace;
    a.trace_cap = g_trace_cap;
}
}  // namespace

int set_debug_trace(void *buf, int capacity)
{
#ifdef FK_DEBUG_CHECKS
    if (capacity < 0 || (buf == nullptr && capacity != 0)) return FK_EINVAL;
    std::lock_guard<std::mutex> lk(g_trace_mu);
    g_trace = (unsigned long long *)buf;
    g_trace_cap = buf ? capacity : 0;
    return FK_OK;
#else
    (void)buf;
    (void)capacity;
    return FK_EUNSUPPORTED;
#endif
}

int set_vjp_split_event(void *event)
{
    std::lock_guard<std::mutex> lk(g_split_mu);
    g_split_event = event;
    return FK_OK;
}

int set_diag_engine(int engine)
{
    if (engine != FK_ENGINE_FP64 && engine != FK_ENGINE_TENSOR && engine != FK_ENGINE_AUTO) return FK_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_engine = engine;
    return FK_OK;
}

int set_diag_tuning(int tpb, int ch, int bps)
{
    if (tpb == 0 && ch == 0) {
        tpb = 128;
        ch = 8;
    }
    bool ok = false;
    for (int i = 0; i < kNumVariants; ++i) ok |= (tables().v[i].tpb == tpb && tables().v[i].ch == ch);
    if (!ok || bps < 0 || bps > 32) return FK_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tpb = tpb;
    g_ch = ch;
    g_bps = bps;
    return FK_OK;
}

int diag_tuning_flags(int engine, int tpb, int ch, int bps, unsigned *flags)
{
    if (!flags) return FK_EINVAL;
    unsigned f = 0;
    if (engine == FK_ENGINE_FP64) f |= FK_FLAG_ENGINE_FP64;
    else if (engine == FK_ENGINE_TENSOR) f |= FK_FLAG_ENGINE_TENSOR;
    else if (engine != FK_ENGINE_AUTO) return FK_EINVAL;
    if (bps < 0 || bps > 32) return FK_EINVAL;
    if (tpb != 0 || ch != 0) {
        int idx = 0;
        for (int i = 0; i < kNumVariants; ++i)
            if (tables().v[i].tpb == tpb && tables().v[i].ch == ch) idx = i + 1;
        if (idx == 0) return FK_EINVAL;
        f |= (unsigned)idx << 8 | (unsigned)bps << 12;
    } else if (bps != 0) {
        return FK_EINVAL;
    }
    *flags = f;
    return FK_OK;
}

int check_diag_flags(unsigned flags)
{
    if ((flags & FK_FLAG_ENGINE_FP64) && (flags & FK_FLAG_ENGINE_TENSOR)) return FK_EINVAL;
    const int v = (int)((flags >> 8) & 15u);
    if (v > kNumVariants || (v == 0 && ((flags >> 12) & 63u) != 0) || ((flags >> 12) & 63u) > 32)
        return FK_EINVAL;
    return FK_OK;
}

// Blocks a launch of shape sh and `batch` circuits can keep busy: the tiles
// of its largest phase, or of all phases for the tensor engine's partial pass.
static int64_t useful_blocks(const DiagShape &sh, int batch, int tpb, bool all_phases)
{
    const int i = tpb <= 64 ? 0 : (tpb <= 128 ? 1 : 2);
    const int64_t t = all_phases ? sh.all_tiles128 : sh.max_phase_tiles[i];
    return t < 1 ? 1 : (int64_t)batch * t;
}

int diag_grid_size(const DiagShape &sh, bool vjp, unsigned flags, int batch, int *grid, int *slots)
{
    int sms = 0;
    int rc = device_sms(&sms);
    if (rc) return rc;
    int bps = 0, tpb = 0, spb = 1;
    size_t smem = 0;
    const void *fn = nullptr;
    const Tune tn = resolve_tune(flags);
    walk_kernel(sh, tn, vjp, &fn, &tpb, &smem, &bps, &spb);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return FK_ECUDA;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, tpb, smem) != cudaSuccess) return FK_ECUDA;
    if (per < 1) return FK_EUNSUPPORTED;
    if (bps > 0 && bps < per) per = bps;
    int64_t g = (int64_t)per * sms;
    const int64_t useful = useful_blocks(sh, batch, tpb, vjp && tc_engine_for(sh, tn));
    if (useful < g) g = useful;
    *grid = (int)g;
    if (slots) *slots = (int)g * spb;
    return FK_OK;
}

// A batch with at least two circuits per block walks circuit by circuit in
// each block (block barriers between phases) rather than level by level over
// the grid: small circuits then stop paying a grid barrier per level.
static int circuit_per_block(int grid, int batch)
{
    return 2 * (int64_t)grid <= batch ? 1 : 0;
}

static int launch_coop(const void *fn, int grid, int tpb, size_t smem, DiagArgs *args, cudaStream_t st)
{
    void *params[] = {args};
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(tpb), params, smem, st);
    return e == cudaSuccess ? FK_OK : FK_ECUDA;
}

// Key of the pivot geometry table: FNV-1a over the shape (a struct without
// padding, zero-filled before it is built) and the table's address.
static unsigned long long geometry_key(const DiagShape &sh, const int *geo)
{
    static_assert(sizeof(DiagShape) % 8 == 0, "DiagShape has no tail padding");
    unsigned long long h = 0xcbf29ce484222325ull;
    const unsigned char *p = (const unsigned char *)&sh;
    for (size_t i = 0; i < sizeof(DiagShape); ++i) h = (h ^ p[i]) * 0x100000001b3ull;
    const unsigned long long g = (unsigned long long)(uintptr_t)geo;
    for (int i = 0; i < 8; ++i) h = (h ^ ((g >> (8 * i)) & 0xffu)) * 0x100000001b3ull;
    return h | 1ull;   // never 0, the cleared value
}

static DiagArgs make_args(const DiagShape &sh, int batch, unsigned flags, const void *A,
                          const void *b, const void *c, void *ws, const DiagLayout &lay)
{
    DiagArgs a{};
    a.sh = sh;
    a.B = batch;
    a.flags = flags;
    a.A = (const double2 *)A;
    a.b = (const double2 *)b;
    a.c = (const double2 *)c;
    char *w = (char *)ws;
    a.ctl = (Control *)(w + lay.ctl);
    a.As = (double2 *)(w + lay.As);
    a.bs = (double2 *)(w + lay.bs);
    a.dig = (unsigned char *)(w + lay.dig);
    a.ctr = (int *)(w + lay.ctr);
    a.geo = lay.geo != lay.F ? (int *)(w + lay.geo) : nullptr;
    a.geo_key = a.geo != nullptr ? geometry_key(sh, a.geo) : 0ull;
    a.F = (double2 *)(w + lay.F);
    a.lvl = (unsigned long long *)(w + lay.lvl);
    a.timeout_ns = kBarrierTimeoutNs;
    attach_trace(a);
    return a;
}

static unsigned long long stop_threshold(double eps)
{
    return (unsigned long long)((1.0 - eps) * 0x1p56);
}

static int launch_check_finite(const DiagShape &sh, int batch, const void *A, const void *b,
                               const void *c, Control *ctl, cudaStream_t st)
{
    const int64_t Do = sh.D_orig;
    return launch_check_finite(A, (int64_t)batch * Do * Do, b, (int64_t)batch * Do, c, batch, ctl, st);
}

int launch_diag_forward(const DiagShape &sh, int batch, unsigned flags, const void *A,
                        const void *b, const void *c, void *probs, void *ws,
                        const DiagLayout &lay, void *stream, const EarlyStop *es)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync((char *)ws + lay.ctl, 0, sizeof(Control), st) != cudaSuccess) return FK_ECUDA;
    if (sh.M == 0) {
        if ((flags & FK_FLAG_CHECK_FINITE) &&
            launch_check_finite(sh, batch, A, b, c, (Control *)((char *)ws + lay.ctl), st) != 0)
            return FK_ECUDA;
        copy_c_kernel<<<(batch + 127) / 128, 128, 0, st>>>((const double2 *)c, (double2 *)probs, batch, 1);
        if (es && es->levels)
            fill_int_kernel<<<(batch + 127) / 128, 128, 0, st>>>(es->levels, batch, 1);
        return cudaGetLastError() == cudaSuccess ? FK_OK : FK_ECUDA;
    }
    DiagArgs a = make_args(sh, batch, flags, A, b, c, ws, lay);
    a.probs = (double2 *)probs;
    int rc0 = 0;
    if (es) {
        // unstarted photon numbers stay zero; the per-level sums start from zero
        if (cudaMemsetAsync(probs, 0, (size_t)batch * sh.n_diag * 16, st) != cudaSuccess) return FK_ECUDA;
        if (cudaMemsetAsync((char *)ws + lay.lvl, 0, (size_t)batch * (sh.L + 2) * 8, st) != cudaSuccess)
            return FK_ECUDA;
        a.early = 1;
        a.thr = stop_threshold(es->eps);
        a.levels = es->levels;
    }
    if ((flags & FK_FLAG_CHECK_FINITE) && (rc0 = launch_check_finite(sh, batch, A, b, c, a.ctl, st)) != 0)
        return rc0;
    const Tune tn = resolve_tune(flags);
    int grid = 0;
    int rc = diag_grid_size(sh, false, flags, batch, &grid);
    if (rc) return rc;
    a.grid = grid;
    a.pc = circuit_per_block(grid, batch);
    int bps = 0, tpb = 0, spb = 1;
    size_t smem = 0;
    const void *fn = nullptr;
    walk_kernel(sh, tn, false, &fn, &tpb, &smem, &bps, &spb);
    return launch_coop(fn, grid, tpb, smem, &a, st);
}

int launch_diag_vjp(const DiagShape &sh, int batch, unsigned flags, const void *A, const void *b,
                    const void *c, const void *gprobs, void *gA, void *gb, void *gc, void *ws,
                    const DiagLayout &lay, void *stream, const EarlyStop *es)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (sh.M == 0) {
        const int n = batch * sh.D_orig * sh.D_orig + batch;
        vacuum_vjp_kernel<<<(n + 127) / 128, 128, 0, st>>>((const double2 *)gprobs, (double2 *)gA,
                                                         (double2 *)gb, (double2 *)gc, batch, sh.D_orig);
        return cudaGetLastError() == cudaSuccess ? FK_OK : FK_ECUDA;
    }
    char *w = (char *)ws;
    // the words before geo_key: the key the forward left says whether its
    // pivot geometry table is still the one this walk needs
    if (cudaMemsetAsync(w + lay.ctl, 0, offsetof(Control, geo_key), st) != cudaSuccess) return FK_ECUDA;
    // With b = 0 every adjoint the walk reads is stored before it is read (or
    // read as zero), so Fbar needs clearing only for the b != 0 sums.
    if (sh.has_b && cudaMemsetAsync(w + lay.Fbar, 0, lay.scratch - lay.Fbar, st) != cudaSuccess) return FK_ECUDA;
    if (cudaMemsetAsync(w + lay.partA, 0, lay.total - lay.partA, st) != cudaSuccess) return FK_ECUDA;
    DiagArgs a = make_args(sh, batch, flags, A, b, c, ws, lay);
    a.gprobs = (const double2 *)gprobs;
    a.Fbar = (double2 *)(w + lay.Fbar);
    a.scratch = (double2 *)(w + lay.scratch);
    a.partA = (double2 *)(w + lay.partA);
    a.partb = (double2 *)(w + lay.partb);
    a.gA = (double2 *)gA;
    a.gb = (double2 *)gb;
    a.gc = (double2 *)gc;
    a.grid = lay.grid_vjp;
    a.slots = lay.slots_vjp;
    a.geo_reuse = 1;
    if (es) {
        a.early = 1;
        a.thr = stop_threshold(es->eps);
    }
    int rc = 0;
    if ((flags & FK_FLAG_CHECK_FINITE) && (rc = launch_check_finite(sh, batch, A, b, c, a.ctl, st)) != 0)
        return rc;
    const Tune tn = resolve_tune(flags);
    int bps = 0, tpb = 0, spb = 1;
    size_t smem = 0;
    const void *fn = nullptr;
    walk_kernel(sh, tn, true, &fn, &tpb, &smem, &bps, &spb);
    int grid = 0, slots = 0;
    rc = diag_grid_size(sh, true, flags, batch, &grid, &slots);
    if (rc) return rc;
    // tuning or engine changed since the layout was sized
    if (grid != lay.grid_vjp || slots != lay.slots_vjp) return FK_EWORKSPACE;
    if (tc_engine_for(sh, tn)) {
        // the reverse walk (its own grid), then the partial pass that owns the slots
        const void *wfn = nullptr;
        int wtpb = 0, wbps = 0, wspb = 1;
        size_t wsmem = 0;
        walk_kernel(sh, tn, true, &wfn, &wtpb, &wsmem, &wbps, &wspb, true);
        if (cudaFuncSetAttribute(wfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem) != cudaSuccess)
            return FK_ECUDA;
        int per = 0, sms = 0;
        if ((rc = device_sms(&sms)) != 0) return rc;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, wfn, wtpb, wsmem) != cudaSuccess) return FK_ECUDA;
        if (per < 1) return FK_EUNSUPPORTED;
        DiagArgs w = a;
        const int64_t useful = useful_blocks(sh, batch, wtpb, false);
        w.grid = (int)((int64_t)per * sms < useful ? (int64_t)per * sms : useful);
        w.pc = circuit_per_block(w.grid, batch);
        if ((rc = launch_coop(wfn, w.grid, wtpb, wsmem, &w, st)) != 0) return rc;
        void *ev = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_split_mu);
            ev = g_split_event;
        }
        if (ev && cudaEventRecord((cudaEvent_t)ev, st) != cudaSuccess) return FK_ECUDA;
    }
    a.pc = tc_engine_for(sh, tn) ? 0 : circuit_per_block(lay.grid_vjp, batch);   // the partial pass has no levels
    return launch_coop(fn, lay.grid_vjp, tpb, smem, &a, st);
}

void tuning_key(unsigned flags, int out[4])
{
    const Tune t = resolve_tune(flags);
    out[0] = t.engine;
    out[1] = t.tpb;
    out[2] = t.ch;
    out[3] = t.bps;
}

int multi_geometry(const DiagShape &env, unsigned flags, bool vjp, const int64_t useful[4], int *grid,
                   int *slots_pb, int *tpb_out)
{
    int sms = 0;
    int rc = device_sms(&sms);
    if (rc) return rc;
    const Tune tn = resolve_tune(flags);
    int bps = 0, tpb = 0, spb = 1;
    size_t smem = 0;
    const void *fn = nullptr;
    walk_kernel(env, tn, vjp, &fn, &tpb, &smem, &bps, &spb);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return FK_ECUDA;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, tpb, smem) != cudaSuccess) return FK_ECUDA;
    if (per < 1) return FK_EUNSUPPORTED;
    if (bps > 0 && bps < per) per = bps;
    int64_t g = (int64_t)per * sms;
    const int i = tpb <= 64 ? 0 : (tpb <= 128 ? 1 : 2);
    int64_t u = (vjp && tc_engine_for(env, tn)) ? useful[3] : useful[i];
    if (u < 1) u = 1;
    if (u < g) g = u;
    *grid = (int)g;
    *slots_pb = spb;
    *tpb_out = tpb;
    return FK_OK;
}

static DiagArgs multi_args(const MultiPlan &p, unsigned flags, const void *A, const void *b, const void *c,
                           void *ws)
{
    static_assert(sizeof(DiagArgs) <= 4096, "a group view must fit its 4 KB slot");
    DiagArgs a{};
    char *w = (char *)ws;
    a.sh = p.env;
    a.B = p.B;
    a.flags = flags;
    a.A = (const double2 *)A;
    a.b = (const double2 *)b;
    a.c = (const double2 *)c;
    a.ctl = (Control *)w;
    a.ctr = (int *)(w + p.off_ctr);
    a.timeout_ns = kBarrierTimeoutNs;
    attach_trace(a);
    a.G = p.G;
    const unsigned char *img = (const unsigned char *)(w + p.off_plan);
    a.grp = (const DiagGroup *)img;
    const size_t o_cidx = align_up(sizeof(DiagGroup) * p.G);
    const size_t o_oidx = align_up(o_cidx + sizeof(int) * p.B);
    const size_t o_tiles = align_up(o_oidx + sizeof(int64_t) * p.B);
    a.cidx = (const int *)(img + o_cidx);
    a.oidx = (const int64_t *)(img + o_oidx);
    a.gtiles = (const int *)(img + o_tiles);
    a.gargs = (DiagArgs *)(w + p.off_views);
    a.wsbase = w;
    return a;
}

static int multi_prepare(const MultiPlan &p, unsigned flags, const void *A, const void *b, const void *c,
                         void *ws, cudaStream_t st)
{
    const void *hp = nullptr;
    int rc = multi_pinned_plan(p, &hp);
    if (rc) return rc;
    if (cudaMemsetAsync(ws, 0, sizeof(Control), st) != cudaSuccess) return FK_ECUDA;
    if (cudaMemcpyAsync((char *)ws + p.off_plan, hp, p.plan_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FK_ECUDA;
    if (flags & FK_FLAG_CHECK_FINITE) {
        const int64_t Do = 2 * (int64_t)p.M;
        rc = launch_check_finite(A, p.B * Do * Do, b, p.B * Do, c, p.B, (Control *)ws, st);
        if (rc) return rc;
    }
    return FK_OK;
}

int launch_multi_forward(const MultiPlan &p, unsigned flags, const void *A, const void *b, const void *c,
                         void *probs, void *ws, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = multi_prepare(p, flags, A, b, c, ws, st);
    if (rc) return rc;
    if (p.env.M == 0) {   // every circuit is the vacuum: p = c, one output each
        copy_c_kernel<<<(p.B + 127) / 128, 128, 0, st>>>((const double2 *)c, (double2 *)probs, p.B, 1);
        return cudaGetLastError() == cudaSuccess ? FK_OK : FK_ECUDA;
    }
    DiagArgs a = multi_args(p, flags, A, b, c, ws);
    a.probs = (double2 *)probs;
    a.grid = p.grid_fwd;
    const Tune tn = resolve_tune(flags);
    int bps = 0, tpb = 0, spb = 1;
    size_t smem = 0;
    const void *fn = nullptr;
    walk_kernel(p.env, tn, false, &fn, &tpb, &smem, &bps, &spb);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return FK_ECUDA;
    return launch_coop(fn, p.grid_fwd, tpb, smem, &a, st);
}

int launch_multi_vjp(const MultiPlan &p, unsigned flags, const void *A, const void *b, const void *c,
                     const void *gprobs, void *gA, void *gb, void *gc, void *ws, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = multi_prepare(p, flags, A, b, c, ws, st);
    if (rc) return rc;
    if (p.env.M == 0) {
        const int n = p.B * (2 * p.M) * (2 * p.M) + p.B;
        vacuum_vjp_kernel<<<(n + 127) / 128, 128, 0, st>>>((const double2 *)gprobs, (double2 *)gA, (double2 *)gb,
                                                         (double2 *)gc, p.B, 2 * p.M);
        return cudaGetLastError() == cudaSuccess ? FK_OK : FK_ECUDA;
    }
    char *w = (char *)ws;
    // adjoints need clearing only for the b != 0 sums (as for one shape)
    if (p.env.has_b && cudaMemsetAsync(w + p.off_vjp, 0, p.off_scratch - p.off_vjp, st) != cudaSuccess)
        return FK_ECUDA;
    if (cudaMemsetAsync(w + p.off_part, 0, p.total_vjp - p.off_part, st) != cudaSuccess) return FK_ECUDA;
    DiagArgs a = multi_args(p, flags, A, b, c, ws);
    a.gprobs = (const double2 *)gprobs;
    a.gA = (double2 *)gA;
    a.gb = (double2 *)gb;
    a.gc = (double2 *)gc;
    a.grid = p.grid;
    a.slots = p.grid * p.slots_pb;
    const Tune tn = resolve_tune(flags);
    int bps = 0, tpb = 0, spb = 1;
    size_t smem = 0;
    const void *fn = nullptr;
    walk_kernel(p.env, tn, true, &fn, &tpb, &smem, &bps, &spb);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return FK_ECUDA;
    if (tc_engine_for(p.env, tn)) {
        // the reverse walk on the forward's grid, then the partial pass that owns the slots
        const void *wfn = nullptr;
        int wtpb = 0, wbps = 0, wspb = 1;
        size_t wsmem = 0;
        walk_kernel(p.env, tn, true, &wfn, &wtpb, &wsmem, &wbps, &wspb, true);
        if (cudaFuncSetAttribute(wfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem) != cudaSuccess)
            return FK_ECUDA;
        int per = 0, sms = 0;
        if ((rc = device_sms(&sms)) != 0) return rc;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, wfn, wtpb, wsmem) != cudaSuccess) return FK_ECUDA;
        if (per < 1) return FK_EUNSUPPORTED;
        DiagArgs r = a;
        r.grid = (int)((int64_t)per * sms < p.grid_fwd ? (int64_t)per * sms : p.grid_fwd);
        if ((rc = launch_coop(wfn, r.grid, wtpb, wsmem, &r, st)) != 0) return rc;
        void *ev = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_split_mu);
            ev = g_split_event;
        }
        if (ev && cudaEventRecord((cudaEvent_t)ev, st) != cudaSuccess) return FK_ECUDA;
    }
    return launch_coop(fn, p.grid, tpb, smem, &a, st);
}

int launch_wait_selftest(void *ws, unsigned long long timeout_ns, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(ws, 0, sizeof(Control), st) != cudaSuccess) return FK_ECUDA;
    wait_selftest_kernel<<<1, 32, 0, st>>>((Control *)ws, timeout_ns);
    return cudaGetLastError() == cudaSuccess ? FK_OK : FK_ECUDA;
}

int launch_check_finite(const void *A, int64_t n_A, const void *b, int64_t n_b, const void *c,
                        int64_t n_c, Control *ctl, void *stream)
{
    const int64_t n = 2 * (n_A > n_b ? (n_A > n_c ? n_A : n_c) : (n_b > n_c ? n_b : n_c));
    const int grid = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    check_finite_kernel<<<grid < 1 ? 1 : grid, 256, 0, (cudaStream_t)stream>>>(
        (const unsigned long long *)A, n_A, (const unsigned long long *)b, n_b,
        (const unsigned long long *)c, n_c, ctl);
    return cudaGetLastError() == cudaSuccess ? FK_OK : FK_ECUDA;
}

int read_status(const void *ws, void *stream, int *status)
{
    cudaStream_t st = (cudaStream_t)stream;
    int v = 0;
    if (cudaMemcpyAsync(&v, ws, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return FK_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FK_ECUDA;
    *status = v;
    return FK_OK;
}

int read_debug(const void *ws, void *stream, long long *out)
{
    cudaStream_t st = (cudaStream_t)stream;
    Control c;
    if (cudaMemcpyAsync(&c, ws, sizeof(Control), cudaMemcpyDeviceToHost, st) != cudaSuccess) return FK_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FK_ECUDA;
    out[0] = c.dbg_count;
    out[1] = c.dbg_site;
    out[2] = c.dbg_index;
    out[3] = c.dbg_lo;
    out[4] = c.dbg_hi;
    return FK_OK;
}

}  // namespace fk
