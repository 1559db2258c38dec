// fk_internal.h -- declarations shared by the host code and the CUDA
// translation units of the library (not part of the public ABI).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "fk_shape.h"

namespace fk {

// Device-side control block at offset 0 of every workspace.
struct Control {
    int status;          // first error recorded by a kernel (fk_status)
    int has_b;           // OR over circuits of (b != 0), set by the prologue
    unsigned bar_count;  // grid barrier arrivals
    unsigned bar_gen;    // grid barrier generation
    unsigned wait_flag;  // self-test flag that nothing sets
    int skip;            // set by the input scan (FK_FLAG_CHECK_FINITE) before the walk:
                         // every walk kernel of the call returns at once
    // debug-checks build (FK_DEBUG_CHECKS): accesses outside their storage box
    int dbg_count;       // how many
    int dbg_site;        // source line of the first one
    long long dbg_index; // its index and the box [dbg_lo, dbg_hi) it had to lie in
    long long dbg_lo, dbg_hi;
    int pad[48];
    // Key of the all-detected walk's pivot geometry table in this workspace,
    // written by the forward after it built the table.  The forward clears
    // the whole block before its launch; the VJP launch clears only the words
    // before this one, so the reverse walk can tell that the table its
    // workspace holds was built for its shape and reuse it.
    unsigned long long geo_key;
};
static_assert(sizeof(Control) == 256, "control block is 256 bytes");

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Build the storage geometry of the all-detected walk (modes with C_j = 1
// dropped).  Returns 0 or an fk_status.
int build_diag_shape(int M, const int *cutoffs, bool has_b, DiagShape *sh);
// Global photon cutoff n_max (Sec. 2.3, applied to Algorithm 1 as Sec. 3.1.3
// describes): every pattern with n_1 + ... + n_M < n_max, no per-mode cutoff.
int build_global_shape(int M, int n_max, bool has_b, DiagShape *sh);

// Per-circuit digit fragments of A for the tensor-core engine (M <= 12): the
// 2D row exponent fields (padded to 256 bytes), then the fp16 digit fragments
// of the real form of A (up to 3 x 3 tiles x 7 digits x 32 lanes x 16 bytes).
constexpr size_t kDigFragBytes = 3 * 3 * 7 * 32 * 16;
constexpr size_t kDigBytes = 256 + kDigFragBytes;
inline size_t diag_digit_bytes(int M) { return M <= 12 ? kDigBytes : 0; }

// Geometry of every AP(K) pivot (M <= 8), shared by all circuits of a launch:
// 12 ints per pivot, indexed like the VJP scratch (off_ap[K] + level offset
// + rank): the digits (two words), the ranks of e - 1_m for m = K+1..K+7,
// the T2 read offset and the DIAG write offset relative to their levels.
constexpr int kGeoInts = 12;
inline size_t diag_geo_bytes(const DiagShape &sh)
{
    return sh.M >= 1 && sh.M <= 8 ? (size_t)sh.n_ap * kGeoInts * sizeof(int) : 0;
}

// One group of a launch of several all-detected shapes (circuits with
// different cutoffs in one launch): the circuits that share a shape (the same
// kept cutoffs and kept modes), where their state lives in the workspace
// (byte offsets), and where their caller indices and output offsets start in
// the launch's tables.
struct DiagGroup {
    DiagShape sh;
    int B;                    // circuits of the group
    int first;                // first entry in the launch's cidx / oidx tables
    int slots;                // partial-sum slots per circuit (VJP)
    int pad;
    int64_t As, bs, dig, geo, F, Fbar, scratch, partA, partb;
};

// Workspace layout of the all-detected walk for `batch` circuits.
struct DiagLayout {
    size_t ctl, lvl, ctr, As, bs, dig, geo, F, Fbar, scratch, partA, partb, total;
    int grid_vjp, slots_vjp;
};
int diag_layout(const DiagShape &sh, int batch, bool vjp, unsigned flags, DiagLayout *lay);

// ------------------------------------------------------- conditional walk
// Algorithm 2 (Sec. 3.2): undetected modes keep their full (ket, bra) index
// pairs, the detected modes follow the Algorithm-1 structure (with the
// offset_1 types, which the undetected reads need even when b = 0).  The
// amplitude at (u, y) -- u a point of the undetected sub-lattice, y a
// position of the detected structure -- is stored at F[y * U2 + u].
constexpr int FK_MAXU = 4;            // undetected modes with cutoff > 1
constexpr int kCondTPB = 128;

struct CondCirc {
    DiagShape dsh;                    // detected sub-problem (kept modes, offset_1 boxes)
    int nU;                           // undetected modes with C > 1
    int CU[FK_MAXU];                  // their cutoffs
    int U2;                           // prod CU^2 (u-block size)
    int ustride[2 * FK_MAXU];         // u-block strides of the undetected lattice indices
    int Lu;                           // sum 2 (CU - 1): levels of the undetected sub-lattice
    int nchunk;                       // ceil(U2 / kCondTPB)
    int NUo;                          // prod CU: ket (= bra) extent of the output
    int Dred;                         // 2 (dsh.M + nU): detected indices first, then undetected
    int red_to_orig[2 * FK_MAXM + 2 * FK_MAXU];
    int W_off;                        // this circuit's level table in the plan (unsigned words)
    int Wn;                           // its row length (dsh.L + 2)
    int64_t off_F;                    // amplitudes of this circuit in F (elements)
    int64_t off_rho;                  // its block of the output (elements)
    int64_t off_scratch;              // its VJP scratch (elements): dsh.n_ap * U2
    int64_t n_patterns;               // detected patterns (= dsh.n_diag)
    int64_t geo_off;                  // first record of this circuit's pivot geometry table
    int gp_off;                       // its pivot prefix per (kind, level) in the plan's tables:
                                      // [2][dsh.L + 1] unsigned, off-diagonal pivots of every
                                      // level first, then the diagonal pivots
    int pad_geo;
};

struct CondPlan {
    int B, M, Md;                     // circuits, caller's modes, detected modes in the mask
    int Dmax;                         // 2 M
    int Lmax;                         // max detected levels over circuits
    int64_t F_total, scratch_total, rho_total;
    int64_t geo_total;                // pivot geometry records of every circuit
    size_t plan_bytes;                // CondCirc[B] followed by the level tables
    const void *host_plan;            // pinned host copy (kept for the life of the process)
};

struct CondLayout {
    size_t ctl, plan, Ar, br, geo, dig, F, Fbar, scratch, partA, partb, total;
    int grid_vjp;
    int ks;            // product engine: 0 = FP64, 1..3 = tensor engine with KS K steps
};

// Returns the cached plan of (batch, M, cutoffs[batch][M], mask); the pinned
// host copy stays valid for the life of the process (graph replays copy it).
int get_cond_plan(int batch, int M, const int *cutoffs, const unsigned char *mask,
                  const CondPlan **plan);
// Workspace layout of a conditional call; flags select the product engine
// (FK_FLAG_ENGINE_FP64 / FK_FLAG_ENGINE_TENSOR, default the tensor engine).
int cond_layout(const CondPlan &plan, bool vjp, unsigned flags, CondLayout *lay);
int cond_engine_ks(const CondPlan &plan, unsigned flags, int *ks);
int cond_grid_size(const CondPlan &plan, bool vjp, int ks, int *grid);
int launch_cond_forward(const CondPlan &plan, unsigned flags, const void *A, const void *b,
                        const void *c, void *rho, void *ws, const CondLayout &lay, void *stream);
int launch_cond_vjp(const CondPlan &plan, unsigned flags, const void *A, const void *b,
                    const void *c, const void *grho, void *gA, void *gb, void *gc, void *ws,
                    const CondLayout &lay, void *stream);

// Compiled kernels of the all-detected walk (walk_diag_fp64.cu,
// walk_diag_tc1.cu, walk_diag_tc2.cu): pivots per tile, output rows per
// register chunk (FP64) or K steps (tensor engine), the kernels and their
// shared-memory size function (M, L, mode, has_b).
struct WalkKernels {
    int tpb, ch, ks;
    const void *fwd, *vjp, *part;
    size_t (*smem)(int, int, int, bool);
};
constexpr int kNumFp64Shapes = 5;         // 128/8, 128/4, 64/8, 64/4, 256/8
const WalkKernels *fp64_walk_kernels_128_8();
const WalkKernels *fp64_walk_kernels_128_4();
const WalkKernels *fp64_walk_kernels_64_8();
const WalkKernels *fp64_walk_kernels_64_4();
const WalkKernels *fp64_walk_kernels_256_8();
const WalkKernels *tc1_walk_kernels();    // M <= 4
const WalkKernels *tc2_walk_kernels();    // M <= 8
const WalkKernels *tc3_walk_kernels();    // M <= 12

// Tile shape of the all-detected walk (pivots per tile, output rows per
// register chunk, blocks per SM; 0 = as many as fit).  Process-wide default;
// the flag bits of a call override it.
int set_diag_tuning(int tpb, int ch, int blocks_per_sm);
// Product engine of the all-detected forward walk (FK_ENGINE_*).  Process-wide.
int set_diag_engine(int engine);
int set_vjp_split_event(void *event);

// Launchers (walk_diag.cu).  All pointers are device pointers.
// Grid of a walk launch: as many blocks as fit on the GPU, but no more than
// the batch has tiles in its largest phase (all phases for the tensor
// engine's barrier-free partial pass), so small problems wait at grid
// barriers of few blocks.
int diag_grid_size(const DiagShape &sh, bool vjp, unsigned flags, int batch, int *grid,
                   int *slots = nullptr);
// Early stop on the probability sum (Sec. 2.3): the pivots of a circuit stop
// once its probabilities with at most `level` photons sum to >= 1 - eps.
struct EarlyStop {
    double eps;
    int *levels;    // [B] device: photon numbers completed per circuit, or null
};
int launch_diag_forward(const DiagShape &sh, int batch, unsigned flags, const void *A,
                        const void *b, const void *c, void *probs, void *ws,
                        const DiagLayout &lay, void *stream, const EarlyStop *es = nullptr);
int launch_diag_vjp(const DiagShape &sh, int batch, unsigned flags, const void *A,
                    const void *b, const void *c, const void *gprobs, void *gA, void *gb,
                    void *gc, void *ws, const DiagLayout &lay, void *stream,
                    const EarlyStop *es = nullptr);
// Several shapes in one launch: the plan (host-side, cached per batch shape
// and grid) and its launchers.  The plan's device image, copied into the
// workspace by every call, is DiagGroup[G] | int cidx[B] | int64 oidx[B] |
// int gtiles[L][2][G + 1] (per level and phase kind (AP 0, DP 1), prefix sums
// over the groups of their tiles).
struct MultiPlan {
    int B, M, G, L;           // circuits, caller's modes, groups, levels (largest group)
    DiagShape env;            // largest kept M and L over the groups, has_b (kernel choice, smem)
    int grid_fwd;             // forward grid
    int grid, slots_pb;       // VJP grid (the partial-sum pass for the tensor engine) and
                              // partial-sum slots per block it was laid out for
    int64_t n_out;            // packed outputs (sum over circuits of prod C)
    size_t off_plan, plan_bytes, off_views, off_ctr, total_fwd;
    size_t off_vjp, off_scratch, off_part, total_vjp;   // VJP regions: Fbar | scratch | partials
    const void *host_plan;    // the device image (host copy)
    std::vector<int64_t> out_offsets;   // [B + 1]
};
int get_multi_plan(int batch, int M, const int *cutoffs, unsigned flags, const MultiPlan **plan);
int multi_pinned_plan(const MultiPlan &plan, const void **out);
// The process-default tuning resolved with the flag bits of a call (engine,
// tpb, ch, blocks-per-SM cap): part of the key of cached launch plans.
void tuning_key(unsigned flags, int out[4]);
// Kernel variant and grid of a several-shape launch (the envelope selects the
// variant): the grid is capped at useful[0..2] blocks (tiles of the largest
// phases at 64/128/256 pivots, summed over the circuits) or, for the tensor
// engine's partial pass, useful[3] (all its tiles).  *tpb = pivots per tile.
int multi_geometry(const DiagShape &env, unsigned flags, bool vjp, const int64_t useful[4], int *grid,
                   int *slots_pb, int *tpb);
int launch_multi_forward(const MultiPlan &p, unsigned flags, const void *A, const void *b, const void *c,
                         void *probs, void *ws, void *stream);
int launch_multi_vjp(const MultiPlan &p, unsigned flags, const void *A, const void *b, const void *c,
                     const void *gprobs, void *gA, void *gb, void *gc, void *ws, void *stream);
int launch_wait_selftest(void *ws, unsigned long long timeout_ns, void *stream);
// FK_FLAG_CHECK_FINITE: scan n_A, n_b, n_c complex values of A, b, c (device)
// for NaN or Inf; on one, ctl->status = FK_ENONFINITE and ctl->skip = 1.
int launch_check_finite(const void *A, int64_t n_A, const void *b, int64_t n_b, const void *c,
                        int64_t n_c, Control *ctl, void *stream);
// Validation of the per-call engine and tile bits of flags, and their encoding.
int check_diag_flags(unsigned flags);
int diag_tuning_flags(int engine, int tpb, int ch, int bps, unsigned *flags);
int read_status(const void *ws, void *stream, int *status);
// Debug-checks build: the control block's access-violation record
// (count, source line, index, box start, box end) and the trace buffer.
int read_debug(const void *ws, void *stream, long long *out);
int set_debug_trace(void *buf, int capacity);

// Default time limit of one grid-barrier wait.
constexpr unsigned long long kBarrierTimeoutNs = 20ull * 1000ull * 1000ull * 1000ull;

}  // namespace fk
