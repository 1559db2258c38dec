// fk_shape.h -- geometry of the compact amplitude storage of the
// all-detected walk (Algorithm 1, Sec. 3.1.3-3.1.4 and App. B.2).
//
// Every amplitude written by Algorithm 1 is diag + offset with offset one of
// the App. B.2 types.  With modes j = 0..M-1 (lattice indices 2j, 2j+1) and
// all C_j >= 2 (modes with C_j = 1 are removed beforehand: their indices are
// always zero, so no read or write ever touches them):
//
//   DIAG          d                   digits d_j in [0, C_j)
//   T2(K)         e + 2*1_{2K}        modes < K zero, e_K in [0, C_K-3]
//   P1010(K,m)    e + 1_{2K} + 1_{2m}    modes < K zero, e_K in [0, C_K-2],
//   P1001(K,m)    e + 1_{2K} + 1_{2m+1}  e_m in [0, C_m-2]          (K < m)
//   T1K(j)        d + 1_{2j}          d_0 in [0, C_0-2], and for j >= 1
//   T1B(j)        d + 1_{2j+1}        d_j in [0, C_j-2]; T1B(0): d_0 <= C_0-3
//
// T1K/T1B (offset_1) are needed only when b != 0 (their weight is odd,
// eq. recrel_noB).  Two layouts of the boxes exist:
//  * mixed radix (off_* fields, used by the conditional walk): each box is
//    a dense row-major array over its digits (mode M-1 fastest);
//  * level-major (lm_* fields, used by the all-detected walk): the vectors of
//    "family K" -- digits over modes K..M-1, e_K <= C_K-2 -- are ordered by
//    digit sum, then lexicographically (mode K slowest).  DIAG uses the
//    family of all modes without the restriction; T2(K) and every
//    P1010/P1001(K,m) pair use family K; the T1K/T1B(j) pairs use family 0.
//    A box whose own digit ranges are narrower leaves those entries unused.
//    Within a level, a vector's position is its rank, computed from
//    prefix sums of the level counts; a pivot's writes sit at its own rank
//    and consecutive pivots touch consecutive entries.
//
// Pivots (Algorithm 1):
//   AP(K) off-diagonal pivot e + 1_{2K}, modes < K zero, e_K in [0, C_K-2]
//         (the off-diagonal pivots of Algorithm 1).  Reads e (DIAG), T2(K)[e-1_K], P1001(K,n)[e-1_n],
//         P1010(K,n)[e-1_n] (n > K) and, if b != 0, its own value T1K(K)[e];
//         writes T2(K)[e], DIAG[e+1_K], P1010(K,m)[e], P1001(K,m)[e].
//   DP    diagonal pivot d with d_0 in [0, C_0-2] (the diagonal pivots of
//         Algorithm 1), b != 0 only.
//         Reads T1B(j)[d-1_j], T1K(j)[d-1_j] and its value DIAG[d]; writes
//         T1K(j)[d], T1B(j)[d].
// The level of a pivot is its digit sum s = |e| (|d|); level s reads
// amplitudes of total weight 2s (and 2s+1 for the pivot value) and writes
// weight 2s+1 (DP) or 2s+2 (AP), so all pivots of one level (DP first, then
// AP) are independent.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define FK_HD __host__ __device__ __forceinline__
#else
#define FK_HD inline
#endif

#define FK_MAXM 12

namespace fk {

struct DiagShape {
    int M;                    // modes kept (all C_j >= 2)
    int M_orig;               // modes of the caller's problem
    int D_orig;               // 2 * M_orig
    int L;                    // levels: pivots have digit sums s = 0..L-1
    int has_b;                // storage for offset_1 types present
    int global;               // global photon cutoff (C_j = n_max, levels < n_max - 1): the
                              // families hold only digit sums <= L, outputs are level-major
    int C[FK_MAXM];           // cutoffs of the kept modes
    int mode_map[FK_MAXM];    // kept mode -> caller's mode
    int64_t n_diag;           // prod C_j
    int64_t circ_size;        // amplitudes stored per circuit
    int64_t off_t2[FK_MAXM];
    int64_t off_t1k[FK_MAXM];
    int64_t off_t1b[FK_MAXM];
    int64_t off_1010[FK_MAXM][FK_MAXM];   // P1010(K,m) element i at off_1010 + 2 i
    int64_t off_1001[FK_MAXM][FK_MAXM];   // P1001(K,m) element i at off_1001 + 2 i (interleaved)
    int64_t off_ap[FK_MAXM];  // AP(K) pivot boxes inside the VJP scratch array
    int64_t n_ap;             // sum_K |AP(K)|
    int64_t fam[FK_MAXM];     // |family K| = (C_K - 1) prod_{i>K} C_i
    int64_t lm_t2[FK_MAXM];   // level-major T2(K)
    int64_t lm_p[FK_MAXM];    // level-major P pairs of anchor K: pair (K,m) at lm_p[K] + 2 (m-K-1) fam[K],
                              // P1010 at even, P1001 at odd positions
    int64_t lm_t1[FK_MAXM];   // level-major T1 pair of mode j (b != 0): T1B at even, T1K at odd
    int64_t circ_alloc;       // level-major amplitudes allocated per circuit (>= circ_size)
    int64_t stride[FK_MAXM];  // DIAG strides S_j = prod_{i>j} C_i
    // Work bounds per circuit for sizing the grid of small problems: the
    // largest number of pivot tiles in one phase (any level, AP or DP) for
    // 64-, 128- and 256-pivot tiles, and the tiles of every AP and DP phase
    // together at 128 pivots (the barrier-free partial pass).
    int64_t max_phase_tiles[3];
    int64_t all_tiles128;
};

// Dense index of digits `dig` in the box over modes k0..M-1 whose extents are
// C_i except C_a - da at mode a and C_m - dm at mode m (a, m may be -1).
// Digits of modes < k0 are ignored (they are zero in every such box).
template <class Digits>
FK_HD int64_t box_index(const DiagShape &sh, const Digits &dig, int k0, int a, int da, int m,
                        int dm)
{
    int64_t idx = 0, st = 1;
    for (int i = sh.M - 1; i >= k0; --i) {
        idx += (int64_t)dig(i) * st;
        st *= (int64_t)(sh.C[i] - (i == a ? da : 0) - (i == m ? dm : 0));
    }
    return idx;
}

FK_HD int64_t box_size(const DiagShape &sh, int k0, int a, int da, int m, int dm)
{
    int64_t st = 1;
    for (int i = sh.M - 1; i >= k0; --i) {
        const int e = sh.C[i] - (i == a ? da : 0) - (i == m ? dm : 0);
        st *= (int64_t)(e > 0 ? e : 0);
    }
    return st;
}

}  // namespace fk
