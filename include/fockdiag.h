/*
 * fockdiag.h -- C ABI of the GB300 (sm_103a) Fock-amplitude library.
 *
 * The library computes photon-number probabilities and conditional density
 * matrices of a noisy M-mode Gaussian state from its Bargmann triple
 * (A, b, c), by the recurrence of arXiv 2303.08879 eq. (recrel) walked as in
 * Algorithm 1 (all modes detected, Sec. 3.1) and Algorithm 2 (conditional
 * states, Sec. 3.2), plus vector-Jacobian products with respect to A, b and
 * c (Sec. 2.5, eqs. dL_dB and dL_dA).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Complex numbers are fk_c128 = {re, im} (same layout as C99 double
 *    complex, cuDoubleComplex and torch.complex128).
 *  - A is D x D row-major and b has D entries, D = 2M.  Lattice index 2j is
 *    the row m and 2j+1 the column n of <m|rho|n> for mode j (the Fock-index
 *    pairing of Sec. 2.1).  A is used through its symmetric part
 *    (A + A^T)/2; amplitudes are the Taylor coefficients of
 *    c exp(z^T A z / 2 + b^T z) scaled by sqrt(k!).
 *  - cutoffs[j] = C_j >= 1: photon numbers 0 <= k < C_j (eq.
 *    local_boundary_conditions, Sec. 2.2).
 *  - Pointers named d_* are DEVICE pointers owned by the caller; host_*
 *    are host pointers.  Compute calls are stream-ordered: they enqueue work
 *    on `stream` (a cudaStream_t; NULL = legacy default stream), never
 *    synchronise it and never allocate device memory.  The caller supplies
 *    a device workspace of at least fk_workspace_size() bytes, 256-byte
 *    aligned, used by one call at a time.
 *  - Errors are returned as fk_status; no exception crosses the ABI.  A
 *    failure detected on the device after launch (a barrier wait that ran
 *    out of time, inconsistent flags) is recorded in the workspace status
 *    word and read back with fk_workspace_status().
 *  - Gradients follow PyTorch's convention for a real loss L:
 *    grad z = dL/dRe z + i dL/dIm z.  For holomorphic amplitudes this is
 *    grad xi = sum_k gbar_k conj(dG_k / dxi), the chain rule of Sec. 2.5.
 *    grad_A is symmetric (A enters only through its symmetric part).
 */
#ifndef FOCKDIAG_H
#define FOCKDIAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } fk_c128;

typedef enum {
    FK_OK = 0,
    FK_EINVAL = 1,         /* bad argument: M < 1, cutoff < 1, NULL pointer, no detected mode ... */
    FK_EUNSUPPORTED = 2,   /* beyond compiled limits (see FK_MAX_*) */
    FK_EWORKSPACE = 3,     /* workspace smaller than fk_workspace_size() or misaligned */
    FK_ENOMEM = 4,         /* host allocation failed */
    FK_ECUDA = 5,          /* a CUDA runtime call or launch failed */
    FK_ETIMEOUT = 6,       /* a device-side barrier wait exceeded its time limit */
    FK_ENONFINITE = 7,     /* FK_FLAG_CHECK_FINITE found a NaN or Inf in A, b or c */
    FK_EBZERO = 8          /* FK_FLAG_B_ZERO was given but b has a nonzero entry */
} fk_status;

/* Compiled limits. */
#define FK_MAX_MODES 12        /* M after dropping modes with C_j = 1 */
#define FK_MAX_CUTOFF 64       /* any single C_j */
#define FK_MAX_LEVELS 512      /* sum_j (C_j - 1) */

/* Operation codes for fk_workspace_size(). */
#define FK_OP_DIAG      1      /* fock_diag_probs[_batched]                  */
#define FK_OP_DIAG_VJP  2      /* fock_diag_probs then fock_diag_probs_vjp   */
#define FK_OP_COND      3      /* fock_conditional_dm[_batched]              */
#define FK_OP_COND_VJP  4      /* fock_conditional_dm then its VJP           */

/* Flags. */
#define FK_FLAG_B_ZERO    1u   /* caller guarantees b == 0 for every circuit:
                                  the odd-weight amplitudes vanish (eq.
                                  recrel_noB, Sec. 2.4), their storage is
                                  omitted and the diagonal pivots of
                                  Algorithm 1 are skipped.  Checked on the
                                  device (FK_EBZERO). */
#define FK_FLAG_RECOMPUTE 2u   /* VJP: run the forward walk first instead of
                                  reusing the state left in the workspace */
#define FK_FLAG_ENGINE_FP64   0x10u   /* this call: FP64 product engine of the
                                         all-detected walk (see fk_diag_set_engine) */
#define FK_FLAG_ENGINE_TENSOR 0x20u   /* this call: tensor-core product engine
                                         (M <= 12 after dropping C_j = 1 modes) */
#define FK_FLAG_CHECK_FINITE  0x40u   /* scan A, b and c on the device before the
                                         walk; on a NaN or Inf the workspace
                                         status word becomes FK_ENONFINITE, the
                                         walk kernels return at once and the
                                         outputs are left unwritten.  The call
                                         itself returns FK_OK (the scan is
                                         stream-ordered); read the status with
                                         fk_workspace_status. */
/* Bits 8..17 of flags: a per-call tile shape of the all-detected walk made by
 * fk_diag_tuning_flags (0 = the process default of fk_diag_set_tuning). */
#define FK_FLAG_TILE_MASK 0x3ff00u

/* Human-readable text for a status code (static storage). */
const char *fk_status_string(int status);

/* Library version, major*10000 + minor*100 + patch. */
int fk_version(void);

/*
 * Bargmann triple of a Gaussian state (host computation).
 * Sec. 2.1, eqs. (A_rho), (b_rho) and Sec. 2.2 (vacuum amplitude):
 *   A = P_M sigma_- sigma_+^{-1},  b = P_M sigma_+^{-1} mu,
 *   c = exp(-mu^dagger sigma_+^{-1} mu / 2) / sqrt(det sigma_+),
 *   sigma_pm = sigma +- I/2, sigma and mu the complex covariance and mean in
 *   the (a_1..a_M, a^dag_1..a^dag_M) basis, hbar = 1.
 * host_V: 2M x 2M real quadrature covariance, ordering (x_1..x_M, p_1..p_M),
 * row-major; host_mean: 2M real quadrature means.  Outputs (host): A (D x D),
 * b (D), c (1) in the library's interleaved lattice order.
 * Returns FK_EINVAL for M < 1 or M > 64 or a singular sigma_+.
 */
int fk_gaussian_to_triple(int M, const double *host_V, const double *host_mean,
                          fk_c128 *host_A, fk_c128 *host_b, fk_c128 *host_c);

/*
 * Parameterised noisy circuit -> Bargmann triple and its Jacobian (host).
 * M squeezed vacua (squeezing r_j of the x quadrature), real displacements
 * x_j, a triangle of M(M-1)/2 beam splitters on neighbouring modes (k, k+1)
 * for k = 0..M-2-i, i = 0..M-2, each [[cos t, -e^{-i p} sin t],
 * [e^{i p} sin t, cos t]], then output phases e^{i psi_j}, then pure loss
 * eta on every mode.  host_theta has M^2 + 2M entries
 *   [r_0..r_{M-1}, x_0..x_{M-1}, (t_1, p_1)..(t_nbs, p_nbs), psi_0..psi_{M-1}].
 * Outputs (A, b, c) as fk_gaussian_to_triple (Sec. 2.1 eqs. A_rho, b_rho;
 * Sec. 2.2 vacuum amplitude) and, if the pointers are not NULL, the
 * derivatives with respect to every parameter: dA [P][D][D], db [P][D],
 * dc [P] (P = M^2 + 2M), from A = P_M (I - sigma_+^{-1}):
 * dA = P_M sigma_+^{-1} dsigma sigma_+^{-1}, and so on.  The paper leaves the
 * circuit ansatz open (Sec. 1); this one serves the gradient-based circuit
 * optimisation of Sec. 2.5 (the chain rule through (A, b, c)).
 */
int fk_circuit_triple(int M, const double *host_theta, double eta, fk_c128 *host_A,
                      fk_c128 *host_b, fk_c128 *host_c, fk_c128 *host_dA, fk_c128 *host_db,
                      fk_c128 *host_dc);

/* The same for n parameter rows host_theta[n][M^2 + 2M] (outputs stacked
 * along a leading n axis), on `threads` host threads (0 = all cores). */
int fk_circuit_triple_batched(int n, int M, const double *host_theta, double eta,
                              fk_c128 *host_A, fk_c128 *host_b, fk_c128 *host_c, fk_c128 *host_dA,
                              fk_c128 *host_db, fk_c128 *host_dc, int threads);

/*
 * Workspace bytes for `op` on `batch` circuits of one shape (M cutoffs,
 * detected_mask; the mask is ignored by the DIAG ops and required by the COND
 * ops; circuits with differing cutoffs use fk_conditional_workspace_size).
 * Depends on the current CUDA device (its SM count sizes per-block partial
 * sums).  Writes *bytes; no device work.
 */
int fk_workspace_size(int M, const int *host_cutoffs, const unsigned char *host_detected_mask,
                      int batch, int op, unsigned flags, size_t *bytes);

/*
 * Detection probabilities, all modes detected (Algorithm 1, Sec. 3.1):
 * p(n) = G_{n1 n1 n2 n2 ...} for every 0 <= n < cutoffs.
 *   d_A [batch][D][D], d_b [batch][D], d_c [batch]   inputs (read only)
 *   d_probs [batch][prod C_j]   output, row-major over modes (mode 0
 *                               slowest); the imaginary part is round-off.
 * The walk's amplitudes stay in the workspace for a following
 * fock_diag_probs_vjp() on the same inputs.
 */
int fock_diag_probs(const fk_c128 *d_A, const fk_c128 *d_b, const fk_c128 *d_c, int M,
                    const int *host_cutoffs, fk_c128 *d_probs, void *d_ws, size_t ws_bytes,
                    void *stream);
int fock_diag_probs_batched(int batch, const fk_c128 *d_A, const fk_c128 *d_b, const fk_c128 *d_c,
                            int M, const int *host_cutoffs, fk_c128 *d_probs, unsigned flags,
                            void *d_ws, size_t ws_bytes, void *stream);

/*
 * Vector-Jacobian product of fock_diag_probs (Sec. 2.5) by a reverse walk.
 *   d_grad_probs [batch][prod C_j]   upstream gradient (PyTorch convention)
 *   d_grad_A [batch][D][D], d_grad_b [batch][D], d_grad_c [batch]  outputs
 * Unless FK_FLAG_RECOMPUTE is set, d_ws must hold the state of a
 * fock_diag_probs[_batched] call with the same inputs, shape and flags: its
 * amplitudes, and the pivot-geometry table (up to 8 kept modes), which the
 * reverse walk takes as built when the key that forward left in the
 * workspace's control block matches this shape and address (it rebuilds the
 * table otherwise, e.g. in a copy of the workspace).
 */
int fock_diag_probs_vjp(const fk_c128 *d_A, const fk_c128 *d_b, const fk_c128 *d_c, int M,
                        const int *host_cutoffs, const fk_c128 *d_grad_probs, fk_c128 *d_grad_A,
                        fk_c128 *d_grad_b, fk_c128 *d_grad_c, void *d_ws, size_t ws_bytes,
                        void *stream);
int fock_diag_probs_vjp_batched(int batch, const fk_c128 *d_A, const fk_c128 *d_b,
                                const fk_c128 *d_c, int M, const int *host_cutoffs,
                                const fk_c128 *d_grad_probs, fk_c128 *d_grad_A,
                                fk_c128 *d_grad_b, fk_c128 *d_grad_c, unsigned flags,
                                void *d_ws, size_t ws_bytes, void *stream);

/*
 * Conditional states (Algorithm 2, Sec. 3.2): for every detection pattern n
 * of the detected modes (host_mask[j] != 0), the unnormalised density matrix
 * of the undetected modes, rho(n) = the diagonal block G_{..n_j n_j..} of the
 * state (Sec. 3.2: "each detection outcome corresponds with one such block").
 * Undetected modes keep both Fock indices; detected modes are walked only
 * along the diagonal, for O(M^2 prod_U C^2 prod_D C) work.
 *   host_cutoffs [batch][M]   each circuit's cutoffs (they may differ)
 *   host_mask [M]             1 = detected, shared by the batch
 *   d_rho                     output, circuits packed back to back; circuit i
 *                             starts at element offset rho_offsets[i] and holds
 *                             [pattern][ket][bra]: patterns row-major over the
 *                             detected modes, ket and bra row-major over the
 *                             undetected modes (mode order)
 * At most 1024 circuits per call, FK_MAX_MODES detected and 4 undetected
 * modes with cutoff > 1.  The walk stays in the workspace for the VJP.
 * Product engine (flags, here and in the VJP): the tensor-core digits by
 * default up to M = 11 caller modes (the real form of [[A, b], [b^T, 0]]
 * fits three 16-row K steps), FP64 beyond; FK_FLAG_ENGINE_FP64 selects
 * FP64, FK_FLAG_ENGINE_TENSOR the tensor engine (FK_EUNSUPPORTED above 11
 * modes).  The workspace size depends on the
 * engine: query fk_conditional_workspace_size with the same flags.
 */
int fk_conditional_workspace_size(int batch, int M, const int *host_cutoffs,
                                  const unsigned char *host_mask, int op, unsigned flags,
                                  size_t *bytes, int64_t *rho_offsets /* [batch + 1] or NULL */);
int fock_conditional_dm(const fk_c128 *d_A, const fk_c128 *d_b, const fk_c128 *d_c, int M,
                        const int *host_cutoffs, const unsigned char *host_mask, fk_c128 *d_rho,
                        void *d_ws, size_t ws_bytes, void *stream);
int fock_conditional_dm_batched(int batch, const fk_c128 *d_A, const fk_c128 *d_b,
                                const fk_c128 *d_c, int M, const int *host_cutoffs,
                                const unsigned char *host_mask, fk_c128 *d_rho, unsigned flags,
                                void *d_ws, size_t ws_bytes, void *stream);

/*
 * Vector-Jacobian product of fock_conditional_dm (Sec. 2.5 by a reverse
 * walk); d_grad_rho has the layout of d_rho.  Unless FK_FLAG_RECOMPUTE is
 * set, d_ws must hold the state of the forward call with the same inputs.
 */
int fock_conditional_dm_vjp(const fk_c128 *d_A, const fk_c128 *d_b, const fk_c128 *d_c, int M,
                            const int *host_cutoffs, const unsigned char *host_mask,
                            const fk_c128 *d_grad_rho, fk_c128 *d_grad_A, fk_c128 *d_grad_b,
                            fk_c128 *d_grad_c, void *d_ws, size_t ws_bytes, void *stream);
int fock_conditional_dm_vjp_batched(int batch, const fk_c128 *d_A, const fk_c128 *d_b,
                                    const fk_c128 *d_c, int M, const int *host_cutoffs,
                                    const unsigned char *host_mask, const fk_c128 *d_grad_rho,
                                    fk_c128 *d_grad_A, fk_c128 *d_grad_b, fk_c128 *d_grad_c,
                                    unsigned flags, void *d_ws, size_t ws_bytes, void *stream);

/*
 * Allocation-free variant of fock_diag_probs_batched.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory themselves -- for example code running where the CUDA
 * allocator is unavailable or forbidden (a plugin host that owns all device
 * memory, a real-time loop that must not allocate, a binding without access
 * to cudaMalloc).  The walk's scratch then lives in one device array of
 * FK_STATIC_WORKSPACE_BYTES that the library reserves on every GPU it is
 * loaded on and keeps until the process exits.  The caller still passes the
 * inputs and the probabilities output (device pointers, as above).
 *   - Calls whose workspace would exceed FK_STATIC_WORKSPACE_BYTES return
 *     FK_EWORKSPACE (fk_workspace_size with FK_OP_DIAG gives the need).
 *   - Every call looks up the array's device address in the current GPU's
 *     context (cudaGetSymbolAddress, which allocates nothing); the first call
 *     on a GPU may load the library's kernels onto it, so make that first
 *     call before any stream capture.
 *   - Every call on a GPU shares the one array: calls that overlap on the
 *     GPU (different streams or threads without ordering) race and corrupt
 *     each other.  Calls are otherwise stream-ordered like the others.
 *   - The call clears what must start at zero (the status word and barrier
 *     counters); the array keeps the previous call's amplitudes otherwise.
 *   - host_status may be NULL.  If not, the call waits for the walk to
 *     finish (synchronising `stream`) and stores the device-side status
 *     there (FK_OK, FK_ETIMEOUT, FK_EBZERO).
 * No cudaMalloc, cudaFree or other allocating routine is called.
 */
#define FK_STATIC_WORKSPACE_BYTES (16u << 20)   /* 16 MiB per GPU */
int fock_diag_probs_static(int batch, const fk_c128 *d_A, const fk_c128 *d_b, const fk_c128 *d_c,
                           int M, const int *host_cutoffs, fk_c128 *d_probs, unsigned flags,
                           void *stream, int *host_status);

/*
 * State-vector walk (Sec. 2.2, "State vector simulations") of a pure
 * Gaussian state: psi_k for every k < cutoffs over M modes from the pure
 * triple (A_psi [M][M], b_psi [M], psi_0) by eq. recrel, pivots in order of
 * weight, each amplitude from its canonical parent (first nonzero index).
 * fk_gaussian_to_pure_triple builds the triple on the host from a pure
 * state's quadrature covariance V [2M][2M] and mean [2M] (hbar = 1, as
 * fk_gaussian_to_triple); it returns FK_EINVAL for a mixed state.  psi_0 is
 * taken real and positive (the global phase is free).
 *
 * fock_pure_amplitudes_batched: A [B][M][M] (symmetrised internally), b [B][M],
 * c [B], psi [B][prod C] row-major (mode 0 slowest), all device pointers.
 * FK_FLAG_B_ZERO promises b = 0: odd weights are zero and skipped (Sec. 2.4).
 * fock_pure_amplitudes_vjp_batched: grad_psi [B][prod C] -> grad_A (symmetric),
 * grad_b, grad_c in the PyTorch convention, all weights included; needs the
 * forward's workspace or FK_FLAG_RECOMPUTE.  Workspace from
 * fk_pure_workspace_size (op FK_OP_DIAG / FK_OP_DIAG_VJP), M <= 16,
 * prod C < 2^31, C_j <= FK_MAX_CUTOFF.  Errors as for the density-matrix walk.
 */
int fk_gaussian_to_pure_triple(int M, const double *host_V, const double *host_mean,
                               fk_c128 *host_A, fk_c128 *host_b, fk_c128 *host_c);
int fk_pure_workspace_size(int batch, int M, const int *host_cutoffs, int op, unsigned flags,
                           size_t *bytes);
int fock_pure_amplitudes_batched(int batch, const fk_c128 *d_A, const fk_c128 *d_b,
                                 const fk_c128 *d_c, int M, const int *host_cutoffs,
                                 fk_c128 *d_psi, unsigned flags, void *d_ws, size_t ws_bytes,
                                 void *stream);
int fock_pure_amplitudes_vjp_batched(int batch, const fk_c128 *d_A, const fk_c128 *d_b,
                                     const fk_c128 *d_c, int M, const int *host_cutoffs,
                                     const fk_c128 *d_grad_psi, fk_c128 *d_grad_A,
                                     fk_c128 *d_grad_b, fk_c128 *d_grad_c, unsigned flags,
                                     void *d_ws, size_t ws_bytes, void *stream);

/*
 * Early stop on the probability sum (Sec. 2.3, last paragraph): after the
 * pivots of each level (photon number) are applied, a circuit stops once its
 * probabilities with at most that many photons sum to >= 1 - eps; the
 * probabilities of higher photon numbers are returned as 0.  Decisions are
 * per circuit and deterministic (the sums are kept in 2^-56 fixed point).
 * d_levels [B] (device, or NULL) receives the number of photon numbers
 * completed per circuit (0 .. levels-1 are exact).  eps in [0, 1]; eps = 0
 * runs the full walk.  The VJP differentiates the stopped walk (its zero
 * outputs are constants) and needs the workspace of the stopped forward with
 * the same eps (or FK_FLAG_RECOMPUTE).  Shapes, workspace (fk_workspace_size
 * with FK_OP_DIAG / FK_OP_DIAG_VJP), flags, stream and errors as for
 * fock_diag_probs_batched / fock_diag_probs_vjp_batched.
 */
int fock_diag_probs_stop_batched(int batch, const fk_c128 *d_A, const fk_c128 *d_b,
                                 const fk_c128 *d_c, int M, const int *host_cutoffs, double eps,
                                 fk_c128 *d_probs, int *d_levels, unsigned flags, void *d_ws,
                                 size_t ws_bytes, void *stream);
int fock_diag_probs_stop_vjp_batched(int batch, const fk_c128 *d_A, const fk_c128 *d_b,
                                     const fk_c128 *d_c, int M, const int *host_cutoffs,
                                     double eps, const fk_c128 *d_grad_probs, fk_c128 *d_grad_A,
                                     fk_c128 *d_grad_b, fk_c128 *d_grad_c, unsigned flags,
                                     void *d_ws, size_t ws_bytes, void *stream);

/*
 * Global photon-number cutoff (Sec. 2.3, eq. global_boundary_conditions, with
 * Algorithm 1 changed as Sec. 3.1.3 describes: the level loop runs to n_max,
 * the per-mode cutoff tests drop out): the probabilities of every detection
 * pattern n with n_1 + ... + n_M < n_max.  Storage and work grow like
 * binomial(n_max + M, M) (App. B.1) instead of n_max^M.
 *
 * Outputs (and upstream gradients) are packed level-major: by total photon
 * number, then lexicographically with mode 0 slowest; fk_global_size gives
 * the count per circuit (binomial(n_max - 1 + M, M)) and
 * fk_global_pattern_index the position of a pattern (-1 if n_1 + ... + n_M
 * >= n_max or a count is negative).  The batched forward / VJP take
 * A [B][2M][2M], b [B][2M], c [B] (device) like fock_diag_probs_batched;
 * probs and grad_probs are [B][count]; flags, workspace, stream and errors as
 * for fock_diag_probs_batched / fock_diag_probs_vjp_batched (workspace from
 * fk_global_workspace_size with op FK_OP_DIAG or FK_OP_DIAG_VJP).  n_max in
 * [1, FK_MAX_CUTOFF], M <= 12.
 */
int fk_global_size(int M, int n_max, int64_t *count);
int fk_global_pattern_index(int M, int n_max, const int *host_pattern, int64_t *index);
int fk_global_workspace_size(int batch, int M, int n_max, int op, unsigned flags, size_t *bytes);
int fock_diag_probs_global_batched(int batch, const fk_c128 *d_A, const fk_c128 *d_b,
                                   const fk_c128 *d_c, int M, int n_max, fk_c128 *d_probs,
                                   unsigned flags, void *d_ws, size_t ws_bytes, void *stream);
int fock_diag_probs_global_vjp_batched(int batch, const fk_c128 *d_A, const fk_c128 *d_b,
                                       const fk_c128 *d_c, int M, int n_max,
                                       const fk_c128 *d_grad_probs, fk_c128 *d_grad_A,
                                       fk_c128 *d_grad_b, fk_c128 *d_grad_c, unsigned flags,
                                       void *d_ws, size_t ws_bytes, void *stream);
/* Storage of the global-cutoff walk: out[0] = amplitudes allocated per
 * circuit, out[1] = pivots applied (App. B.1 count), out[2] = outputs per
 * circuit.  out_len >= 3. */
int fk_describe_global_schedule(int M, int n_max, unsigned flags, int64_t *out, int out_len);

/*
 * Per-circuit cutoffs in one launch (Algorithm 1, Sec. 3.1.3, for a batch of
 * circuits of different shapes, e.g. a sweep over GBS circuits whose modes
 * are cut at different photon numbers).  host_cutoffs is [batch][M] (C >= 1;
 * a circuit with fewer modes gives its unused modes cutoff 1 and they are
 * dropped from its walk, rule R1 of the walk: their indices stay 0).  All
 * circuits share M and the input layout of fock_diag_probs_batched: A
 * [batch][2M][2M], b [batch][2M], c [batch] (device).  Outputs are packed in
 * the caller's order: circuit i's probabilities, row-major over its own
 * cutoffs (mode 0 slowest, prod_j C_ij values), start at out_offsets[i]
 * (fk_multi_workspace_size writes out_offsets[0..batch], the total last).
 * Circuits that share a shape form a group with its own storage; every
 * phase of the walk hands out the tiles of all groups through one counter,
 * so all shapes advance level by level in the same cooperative launch.
 * flags: FK_FLAG_B_ZERO (all circuits), FK_FLAG_ENGINE_*, tile bits,
 * FK_FLAG_CHECK_FINITE; the VJP also FK_FLAG_RECOMPUTE.  The VJP takes
 * d_grad_probs in the packed layout and writes grad_A, grad_b, grad_c as the
 * one-shape VJP.  The launch plan (grouping, offsets, tile tables) is built
 * on the host once per (batch, M, cutoffs, flags, tuning) and kept for the
 * life of the process in pinned memory, so the calls can be captured in a
 * CUDA graph; each call copies it into the workspace.  Errors as for
 * fock_diag_probs_batched; FK_EUNSUPPORTED when a phase holds 2^30 tiles or
 * more.
 */
int fk_multi_workspace_size(int batch, int M, const int *host_cutoffs, int op, unsigned flags,
                            size_t *bytes, int64_t *host_out_offsets);
int fock_diag_probs_multi_batched(int batch, const fk_c128 *d_A, const fk_c128 *d_b, const fk_c128 *d_c,
                                  int M, const int *host_cutoffs, fk_c128 *d_probs, unsigned flags,
                                  void *d_ws, size_t ws_bytes, void *stream);
int fock_diag_probs_multi_vjp_batched(int batch, const fk_c128 *d_A, const fk_c128 *d_b,
                                      const fk_c128 *d_c, int M, const int *host_cutoffs,
                                      const fk_c128 *d_grad_probs, fk_c128 *d_grad_A, fk_c128 *d_grad_b,
                                      fk_c128 *d_grad_c, unsigned flags, void *d_ws, size_t ws_bytes,
                                      void *stream);

/*
 * Tile shape of the all-detected walk kernels, process-wide default (the
 * paper has no counterpart: the autotuner in paper_2303_08879_gb300/
 * autotune.py times the shapes on the caller's workload and sets the
 * fastest).  tpb = pivots per tile (64, 128 or 256), ch = output rows per
 * register chunk (4 or 8; compiled pairs: 128/8, 128/4, 64/8, 64/4, 256/8),
 * blocks_per_sm = cap on resident blocks per SM (0 = as many as fit).
 * tpb = ch = 0 restores the default 128/8.  The shape applies to the FP64
 * engine (the tensor engine has one shape).  Workspaces must be sized
 * (fk_workspace_size) with the setting and flags they run with; a VJP
 * launched with a different setting returns FK_EWORKSPACE.
 *
 * The process-wide defaults (this call and fk_diag_set_engine) are guarded
 * by a lock and read once per call.  Callers that share a process and want
 * different settings pass them per call in `flags` instead: the engine bits
 * FK_FLAG_ENGINE_* and the tile bits from fk_diag_tuning_flags, which take
 * precedence over the defaults and involve no shared state.
 */
int fk_diag_set_tuning(int tpb, int ch, int blocks_per_sm);

/*
 * Per-call form of fk_diag_set_tuning / fk_diag_set_engine: *flags_out gets
 * the bits (engine FK_ENGINE_*, tile shape tpb/ch, blocks_per_sm cap) to OR
 * into the flags of fock_diag_probs*_batched, their VJPs and
 * fk_workspace_size.  tpb = ch = 0 keeps the process-default shape.
 * FK_EINVAL for a shape that is not compiled or a cap outside 0..32.
 */
int fk_diag_tuning_flags(int engine, int tpb, int ch, int blocks_per_sm, unsigned *flags_out);

/*
 * Product engine of the all-detected walk, process-wide default.  Each write
 * of Algorithm 1 is a row of A (restricted to the pivot's modes) times the
 * pivot's reads (eq. recrel with F = G / sqrt(k!)).
 *   FK_ENGINE_FP64:   complex128 DFMA (three real products per term).
 *   FK_ENGINE_TENSOR: the same sums on the fp16 tensor cores: every value is
 *     cut to a 56-bit fixed-point integer relative to a power of two shared
 *     by a row of A or by one pivot's reads, split into seven balanced
 *     base-256 digits (exact in fp16), and the digit products with digit
 *     index sum <= 6 are accumulated exactly (integer partial sums below
 *     2^23 in fp32), recombined in int64 and scaled back with one rounding.
 *     The error is of the order of 2^-53 times the largest term of a sum,
 *     like FP64; values below 2^-997 count as zero.  The VJP runs the
 *     adjoint products conj(A) Y the same way and forms each warp's
 *     partial dL/dA = sum_t Y(t) X(t)^H from digits too, after moving each
 *     pivot's power of two from its reads to its adjoints (products
 *     unchanged), so each term is exact relative to the largest product of
 *     its row.  With this engine the VJP is two launches on the stream:
 *     the reverse walk, then the pass that forms the partial sums.  Kept
 *     modes: up to 12 (one, two or three 16-row K steps); shapes with
 *     M > 12 use FP64.
 *   FK_ENGINE_AUTO:   the tensor engine where it applies (M <= 12 kept
 *     modes), else FP64.  The default: on GB300 the tensor engine runs the
 *     8-mode forward + VJP about 3 times faster than the best FP64 shape
 *     and the 12-mode one about 3.9 times faster.
 * Returns FK_EINVAL for another value.  Per call, FK_FLAG_ENGINE_FP64 and
 * FK_FLAG_ENGINE_TENSOR override this default.
 */
#define FK_ENGINE_FP64 0
#define FK_ENGINE_TENSOR 1
#define FK_ENGINE_AUTO 2
int fk_diag_set_engine(int engine);

/*
 * Measurement hook (no counterpart in the paper): when `event` is a CUDA
 * event (cudaEvent_t passed as a pointer), every following tensor-engine
 * all-detected VJP records it on its stream between its two launches, so a
 * caller can time the reverse walk and the partial-sum pass apart.  NULL
 * switches the hook off (the default).  The caller keeps the event alive
 * while the hook is set.  Process-wide; returns FK_OK.
 */
int fk_diag_set_vjp_split_event(void *event);

/*
 * Reads the device-side status word of a workspace after the calls queued
 * on `stream` (synchronises the stream).  *status = FK_OK or the first error
 * a kernel recorded; the word is cleared by the next compute call.
 */
int fk_workspace_status(const void *d_ws, void *stream, int *status);

/*
 * Self-test of the bounded device-side wait: launches one block that waits
 * for a flag in the workspace that nothing sets, giving up after
 * timeout_ns; the status word then reads FK_ETIMEOUT.  Needs 256 bytes of
 * workspace.  Used by the failure-detection tests; no GPU fault involved.
 */
int fk_selftest_wait_timeout(void *d_ws, size_t ws_bytes, unsigned long long timeout_ns,
                             void *stream);

/*
 * Debug-checks build (the paper has no counterpart; these stand in for a
 * memory checker).  The library built with -DFK_DEBUG_CHECKS
 * (libfockdiag_debug.so) checks the index of every amplitude, adjoint,
 * scratch, output and pivot-geometry access of the all-detected walk
 * (Algorithm 1 and its reverse walk) against the storage box of its
 * type (DIAG, T2(K), the P1010/P1001 pairs of anchor K, the T1 pairs,
 * AP(K) scratch; the App. B.2 types), and those of the conditional walk
 * (Algorithm 2) against its circuit's amplitude, scratch and output
 * arrays.  A violation is counted in the
 * workspace's control block, the first one with its source line, index and
 * box; the access is redirected to the first entry of that box, so nothing
 * outside the buffers is touched.  The normal build compiles the checks
 * out.
 *
 * fk_debug_checks: 1 in the debug-checks build, 0 otherwise.
 * fk_workspace_debug: out[5] = {violations, source line of the first,
 *   its index, box start, box end} of the last walk call on d_ws
 *   (host array; synchronises `stream`).  Always zeros in the normal build.
 * fk_debug_set_trace: registers a device buffer of 1 + 2 capacity 64-bit
 *   words (process-wide; NULL and 0 unregister it) for per-level device
 *   timestamps: after each grid barrier of the walk kernels, word 0 is
 *   incremented and a record (tag, %globaltimer ns) appended while room is
 *   left; tag = kernel << 24 | level << 8 | phase, kernel 1 = forward,
 *   2 = reverse walk, 3 = final gradient reduction, phase 0 = off-diagonal
 *   pivots, 1 = diagonal pivots.  The caller zeroes word 0.  Returns
 *   FK_EUNSUPPORTED in the normal build.
 */
int fk_debug_checks(void);
int fk_workspace_debug(const void *d_ws, void *stream, long long *out);
int fk_debug_set_trace(unsigned long long *d_buf, int capacity);

/*
 * Schedule description (host only, no device work): for the all-detected
 * walk of one circuit writes
 *   out[0] = amplitudes stored, out[1] = pivots applied, out[2] = levels,
 *   out[3 + 6*s .. 3 + 6*s + 5] for level s = number of
 *   {diagonal, offset_1, offset_2, offset_1010, offset_1001, pivots}:
 *   amplitudes of total weight 2s (diagonal, 2, 1010, 1001) or 2s + 1
 *   (offset_1) and the pivots applied at level s (digit sum s),
 * for at most out_len entries.  flags as in fock_diag_probs_batched.
 */
int fk_describe_diag_schedule(int M, const int *host_cutoffs, unsigned flags, int64_t *out,
                              int out_len);

#ifdef __cplusplus
}
#endif

#endif /* FOCKDIAG_H */
