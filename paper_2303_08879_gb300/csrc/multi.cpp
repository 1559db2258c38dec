// multi.cpp -- host plan of the all-detected walk for a batch whose circuits
// have different cutoffs (and so different kept modes): one launch walks
// them all (Algorithm 1, Sec. 3.1.3; the batching of many circuits per
// launch).
//
// Circuits are grouped by shape (the kept cutoffs and which caller modes
// they are).  Each group keeps the storage of a one-shape launch (A_s, b,
// digit fragments, pivot geometry, amplitudes, adjoints, partial sums) in
// its own region of the workspace; the device image of the plan lists the
// groups, the caller index and output offset of every circuit (outputs are
// packed in the caller's order, each circuit row-major over its own
// cutoffs), and per level and phase kind the prefix sums over the groups of
// their tiles, which is how the kernels hand out the tiles of all groups
// through one counter per phase.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "fk_internal.h"
#include "../../include/fockdiag.h"

namespace fk {

namespace {

// Number of digit vectors with extents ext summing to each s <= L.
std::vector<int64_t> hist(const std::vector<int> &ext, int L)
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

struct Entry {
    MultiPlan plan;
    std::vector<unsigned char> bytes;
    void *pinned = nullptr;
};

std::mutex g_mu;
std::map<std::string, std::unique_ptr<Entry>> g_plans;

int build(int B, int M, const int *cut, unsigned flags, Entry *e)
{
    const bool has_b = !(flags & FK_FLAG_B_ZERO);
    MultiPlan &p = e->plan;
    p.B = B;
    p.M = M;
    // group circuits by shape
    std::vector<DiagShape> shapes;
    std::vector<std::vector<int>> members;
    std::map<std::vector<int>, int> index;
    p.out_offsets.assign((size_t)B + 1, 0);
    for (int i = 0; i < B; ++i) {
        DiagShape sh;
        int rc = build_diag_shape(M, cut + (size_t)i * M, has_b, &sh);
        if (rc) return rc;
        p.out_offsets[i + 1] = p.out_offsets[i] + sh.n_diag;
        std::vector<int> key;
        key.push_back(sh.M);
        for (int k = 0; k < sh.M; ++k) {
            key.push_back(sh.C[k]);
            key.push_back(sh.mode_map[k]);
        }
        auto it = index.find(key);
        if (it == index.end()) {
            it = index.emplace(key, (int)shapes.size()).first;
            shapes.push_back(sh);
            members.emplace_back();
        }
        members[it->second].push_back(i);
    }
    const int G = (int)shapes.size();
    p.G = G;
    p.n_out = p.out_offsets[B];
    // envelope: largest kept M and L (shared memory, tensor-engine K steps)
    std::memset(&p.env, 0, sizeof(p.env));
    p.env.M_orig = M;
    p.env.D_orig = 2 * M;
    p.env.has_b = has_b ? 1 : 0;
    for (const DiagShape &sh : shapes) {
        p.env.M = std::max(p.env.M, sh.M);
        p.env.L = std::max(p.env.L, sh.L);
    }
    p.L = p.env.L;
    int64_t useful[4] = {0, 0, 0, 0};
    for (int g = 0; g < G; ++g) {
        const int64_t nb = (int64_t)members[g].size();
        for (int i = 0; i < 3; ++i) useful[i] += nb * shapes[g].max_phase_tiles[i];
        useful[3] += nb * shapes[g].all_tiles128;
    }
    int tpb = 0, grid_f = 0, spb_f = 0, grid_v = 0, spb_v = 0;
    if (p.env.M > 0) {
        int rc = multi_geometry(p.env, flags, false, useful, &grid_f, &spb_f, &tpb);
        if (rc) return rc;
        rc = multi_geometry(p.env, flags, true, useful, &grid_v, &spb_v, &tpb);
        if (rc) return rc;
    } else {
        grid_f = grid_v = 1;
        spb_f = spb_v = 1;
        tpb = 128;
    }
    p.grid_fwd = grid_f;
    p.grid = grid_v;
    p.slots_pb = spb_v;
    const int slots = grid_v * spb_v;
    // device image: DiagGroup[G] | int cidx[B] | int64 oidx[B] | int gtiles[L][2][G + 1]
    const size_t n_tiles = (size_t)std::max(p.L, 1) * 2 * (G + 1);
    const size_t o_cidx = align_up(sizeof(DiagGroup) * G);
    const size_t o_oidx = align_up(o_cidx + sizeof(int) * B);
    const size_t o_tiles = align_up(o_oidx + sizeof(int64_t) * B);
    const size_t nbytes = o_tiles + sizeof(int) * n_tiles;
    e->bytes.assign(nbytes, 0);
    DiagGroup *grp = (DiagGroup *)e->bytes.data();
    int *cidx = (int *)(e->bytes.data() + o_cidx);
    int64_t *oidx = (int64_t *)(e->bytes.data() + o_oidx);
    int *gt = (int *)(e->bytes.data() + o_tiles);
    // workspace: control block | plan image | group views | tile counters |
    // forward state of every group | VJP state of every group
    size_t o = 0;
    o = align_up(o + sizeof(Control));
    p.off_plan = o;
    p.plan_bytes = nbytes;
    o = align_up(o + nbytes);
    p.off_views = o;
    o = align_up(o + (size_t)G * 4096);   // one DiagArgs per group (checked by the launcher)
    p.off_ctr = o;
    o = align_up(o + 4 * (size_t)(p.L + 1) * sizeof(int));
    int first = 0;
    for (int g = 0; g < G; ++g) {
        DiagGroup &q = grp[g];
        const DiagShape &sh = shapes[g];
        const size_t nb = members[g].size(), D = 2 * (size_t)sh.M, c16 = 16;
        q.sh = sh;
        q.B = (int)nb;
        q.first = first;
        q.slots = slots;
        for (size_t k = 0; k < nb; ++k) {
            cidx[first + k] = members[g][k];
            oidx[first + k] = p.out_offsets[members[g][k]];
        }
        first += (int)nb;
        q.As = (int64_t)o; o = align_up(o + nb * D * D * c16);
        q.bs = (int64_t)o; o = align_up(o + nb * D * c16);
        q.dig = (int64_t)o; o = align_up(o + nb * diag_digit_bytes(sh.M));
        const size_t gb = diag_geo_bytes(sh);
        q.geo = gb ? (int64_t)o : -1; o = align_up(o + gb);
        q.F = (int64_t)o; o = align_up(o + nb * (size_t)sh.circ_alloc * c16);
    }
    p.total_fwd = o;
    p.off_vjp = o;
    for (int g = 0; g < G; ++g) {
        grp[g].Fbar = (int64_t)o;
        o = align_up(o + (size_t)grp[g].B * (size_t)shapes[g].circ_alloc * 16);
    }
    p.off_scratch = o;
    for (int g = 0; g < G; ++g) {
        grp[g].scratch = (int64_t)o;
        o = align_up(o + (size_t)grp[g].B * (size_t)shapes[g].n_ap * 16);
    }
    p.off_part = o;
    for (int g = 0; g < G; ++g) {
        const size_t D = 2 * (size_t)shapes[g].M;
        grp[g].partA = (int64_t)o;
        o = align_up(o + (size_t)grp[g].B * slots * D * D * 16);
        grp[g].partb = (int64_t)o;
        o = align_up(o + (size_t)grp[g].B * slots * D * 16);
    }
    p.total_vjp = o;
    // tiles per phase: AP (kind 0) sum over K of ceil(count_K(s) / tpb), DP
    // (kind 1) ceil(count_0(s) / tpb); zero at the levels a group does not have
    for (int s = 0; s < p.L; ++s)
        for (int kind = 0; kind < 2; ++kind) {
            int *pre = gt + (size_t)(2 * s + kind) * (G + 1);
            int64_t acc = 0;
            for (int g = 0; g < G; ++g) {
                pre[g] = (int)acc;
                const DiagShape &sh = shapes[g];
                int64_t t = 0;
                if (s < sh.L && sh.M > 0) {
                    for (int K = 0; K < (kind == 0 ? sh.M : 1); ++K) {
                        std::vector<int> ext;
                        ext.push_back(sh.C[K] - 1);
                        for (int i = K + 1; i < sh.M; ++i) ext.push_back(sh.C[i]);
                        const int64_t cnt = hist(ext, s)[s];
                        t += (cnt + tpb - 1) / tpb;
                    }
                }
                acc += (int64_t)grp[g].B * t;
                if (acc >= (int64_t(1) << 30)) return FK_EUNSUPPORTED;
            }
            pre[G] = (int)acc;
        }
    p.host_plan = e->bytes.data();
    return FK_OK;
}

}  // namespace

int get_multi_plan(int batch, int M, const int *cutoffs, unsigned flags, const MultiPlan **plan)
{
    if (batch < 1 || M < 1 || !cutoffs || !plan) return FK_EINVAL;
    if (int rc = check_diag_flags(flags)) return rc;
    int tk[4];
    tuning_key(flags, tk);
    const unsigned bz = flags & FK_FLAG_B_ZERO;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FK_ECUDA;
    std::string key((const char *)&batch, sizeof(int));
    key.append((const char *)&M, sizeof(int));
    key.append((const char *)&bz, sizeof(bz));
    key.append((const char *)tk, sizeof(tk));
    key.append((const char *)&dev, sizeof(dev));
    key.append((const char *)cutoffs, sizeof(int) * (size_t)batch * M);
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find(key);
    if (it == g_plans.end()) {
        std::unique_ptr<Entry> e(new Entry());
        int rc = build(batch, M, cutoffs, flags, e.get());
        if (rc) return rc;
        it = g_plans.emplace(key, std::move(e)).first;
    }
    *plan = &it->second->plan;
    return FK_OK;
}

int multi_pinned_plan(const MultiPlan &plan, const void **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &kv : g_plans) {
        Entry &e = *kv.second;
        if (&e.plan != &plan) continue;
        if (!e.pinned) {
            if (cudaHostAlloc(&e.pinned, e.bytes.size(), cudaHostAllocDefault) != cudaSuccess) {
                e.pinned = nullptr;
                return FK_ECUDA;
            }
            std::memcpy(e.pinned, e.bytes.data(), e.bytes.size());
        }
        *out = e.pinned;
        return FK_OK;
    }
    return FK_EINVAL;
}

}  // namespace fk
