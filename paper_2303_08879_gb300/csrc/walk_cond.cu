// walk_cond.cu -- host side of the conditional-state walk (Algorithm 2 of
// arXiv 2303.08879, Sec. 3.2): per-batch plans (cached, copied from pinned
// memory so calls can be graph-captured), workspace layout, engine choice
// and the cooperative launches of the kernels in walk_cond_impl.cuh.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "walk_cond_impl.cuh"

namespace fk {

namespace {

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
    a.dig = lay.ks > 0 ? (unsigned char *)(w + lay.dig) : nullptr;
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

const CondKernels *cond_kernels_k0();
const CondKernels *cond_kernels_k1();
const CondKernels *cond_kernels_k2();
const CondKernels *cond_kernels_k3();

namespace {
// The launch's kernel: engine KS (0 = FP64) x (forward, VJP).
const void *cond_kernel(int ks, bool vjp)
{
    const CondKernels *k = ks == 0 ? cond_kernels_k0() : ks == 1 ? cond_kernels_k1()
                         : ks == 2 ? cond_kernels_k2() : cond_kernels_k3();
    return vjp ? k->vjp : k->forward;
}
}  // namespace

// Product engine of a conditional call: FK_FLAG_ENGINE_FP64 -> FP64 (0);
// otherwise the tensor engine with KS = ceil(2 (Dmax + 1) / 16) K steps when
// KS <= 3 (up to 11 modes), FP64 beyond (FK_FLAG_ENGINE_TENSOR there:
// FK_EUNSUPPORTED).
int cond_engine_ks(const CondPlan &plan, unsigned flags, int *ks)
{
    if ((flags & FK_FLAG_ENGINE_FP64) && (flags & FK_FLAG_ENGINE_TENSOR)) return FK_EINVAL;
    if (flags & FK_FLAG_ENGINE_FP64) {
        *ks = 0;
        return FK_OK;
    }
    const int k = cond_ks(plan.Dmax);
    if (k > 3) {
        if (flags & FK_FLAG_ENGINE_TENSOR) return FK_EUNSUPPORTED;
        *ks = 0;
        return FK_OK;
    }
    *ks = k;
    return FK_OK;
}

int cond_grid_size(const CondPlan &plan, bool vjp, int ks, int *grid)
{
    int sms = 0;
    int rc = device_sms(&sms);
    if (rc) return rc;
    const size_t smem = cond_smem_bytes(plan.Dmax, vjp, ks);
    const void *fn = cond_kernel(ks, vjp);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return FK_ECUDA;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, TPB, smem) != cudaSuccess) return FK_ECUDA;
    if (per < 1) return FK_EUNSUPPORTED;
    *grid = per * sms;
    return FK_OK;
}

int cond_layout(const CondPlan &plan, bool vjp, unsigned flags, CondLayout *lay)
{
    const size_t B = (size_t)plan.B, D = (size_t)plan.Dmax, c16 = 16;
    int rc = cond_engine_ks(plan, flags, &lay->ks);
    if (rc) return rc;
    size_t o = 0;
    lay->ctl = o; o = align_up(o + sizeof(Control));
    lay->plan = o; o = align_up(o + plan.plan_bytes);
    lay->Ar = o; o = align_up(o + B * D * D * c16);
    lay->br = o; o = align_up(o + B * D * c16);
    lay->geo = o; o = align_up(o + (size_t)plan.geo_total * sizeof(PGeom));
    lay->dig = o; o = align_up(o + (lay->ks > 0 ? B * kDigBytes : 0));
    lay->F = o; o = align_up(o + (size_t)plan.F_total * c16);
    lay->grid_vjp = 0;
    if (vjp) {
        int grid = 0;
        rc = cond_grid_size(plan, true, lay->ks, &grid);
        if (rc) return rc;
        lay->grid_vjp = grid;
        // partial-sum slots: one per block (FP64) or per warp (tensor engine)
        const size_t slots = (size_t)grid * (lay->ks > 0 ? TPB / 32 : 1);
        lay->Fbar = o; o = align_up(o + (size_t)plan.F_total * c16);
        lay->scratch = o; o = align_up(o + (size_t)plan.scratch_total * c16);
        lay->partA = o; o = align_up(o + B * slots * D * D * c16);
        lay->partb = o; o = align_up(o + B * slots * D * c16);
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
    rc = cond_grid_size(plan, false, lay.ks, &grid);
    if (rc) return rc;
    a.grid = grid;
    a.spb = 1;
    a.slots = grid;
    return launch(cond_kernel(lay.ks, false), grid, cond_smem_bytes(plan.Dmax, false, lay.ks), &a, st);
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
    a.spb = lay.ks > 0 ? TPB / 32 : 1;
    a.slots = a.grid * a.spb;
    return launch(cond_kernel(lay.ks, true), lay.grid_vjp, cond_smem_bytes(plan.Dmax, true, lay.ks), &a, st);
}

}  // namespace fk

