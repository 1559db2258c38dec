// fk_internal.h -- declarations shared by the host code and the CUDA
// translation units of the library (not part of the public ABI).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "fk_shape.h"

namespace fk {

// Device-side control block at offset 0 of every workspace.
struct Control {
    int status;          // first error recorded by a kernel (fk_status)
    int has_b;           // OR over circuits of (b != 0), set by the prologue
    unsigned bar_count;  // grid barrier arrivals
    unsigned bar_gen;    // grid barrier generation
    unsigned wait_flag;  // self-test flag that nothing sets
    int pad[59];
};
static_assert(sizeof(Control) == 256, "control block is 256 bytes");

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Build the storage geometry of the all-detected walk (modes with C_j = 1
// dropped).  Returns 0 or an fk_status.
int build_diag_shape(int M, const int *cutoffs, bool has_b, DiagShape *sh);

// Workspace layout of the all-detected walk for `batch` circuits.
struct DiagLayout {
    size_t ctl, As, bs, F, Fbar, scratch, partA, partb, total;
    int grid_vjp;
};
int diag_layout(const DiagShape &sh, int batch, bool vjp, DiagLayout *lay);

// Launchers (walk_diag.cu).  All pointers are device pointers.
int diag_grid_size(const DiagShape &sh, bool vjp, int *grid);
int launch_diag_forward(const DiagShape &sh, int batch, unsigned flags, const void *A,
                        const void *b, const void *c, void *probs, void *ws,
                        const DiagLayout &lay, void *stream);
int launch_diag_vjp(const DiagShape &sh, int batch, unsigned flags, const void *A,
                    const void *b, const void *c, const void *gprobs, void *gA, void *gb,
                    void *gc, void *ws, const DiagLayout &lay, void *stream);
int launch_wait_selftest(void *ws, unsigned long long timeout_ns, void *stream);
int read_status(const void *ws, void *stream, int *status);

// Default time limit of one grid-barrier wait.
constexpr unsigned long long kBarrierTimeoutNs = 20ull * 1000ull * 1000ull * 1000ull;

}  // namespace fk
