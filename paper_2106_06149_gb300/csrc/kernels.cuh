// Device-side data structures shared by the host planner (api.cu) and the kernels (osv_kernels.cu,
// residual.cu, adjoint.cu).
#pragma once
#include "common.cuh"

namespace osv {

// A copy (optionally transposed) of a rows x cols block: dst[r * ldd + c] = src(r, c),
// src(r, c) = trans ? src[c * lds + r] : src[r * lds + c].  scale multiplies the copied values.
struct BlockCopy {
    double *dst;
    const double *src;
    int rows, cols, trans, accumulate;   // accumulate = 1: dst += scale * src (atomicAdd)
    long long ldd, lds;
    double scale;
};

// One stored pair p = (i, j), i <= j, with domain (Q_i Q_j) (or Q_i when i == j) of padded order np.
struct PairInfo {
    int i, j, np;
    long long off;        // offset (doubles) of this pair's np x np matrices in the per-pair arrays
    long long e_off;      // offset of its np-vectors (eigenvalues)
};

// One coupling term of the residual of cluster slot `dst`:
//   R~_dst -= f[fx * n_occ + fy] * S~ T~'_src S~^T,  S~ = S~_(dst pair, src pair),
// S~ stored at sblk (rows = pair with the smaller id); s_trans = 1 when dst's pair has the larger id.
// t_trans = 1 uses the transpose of the source amplitudes (amplitude t_ik with i > k).
struct Term {
    int dst, src;           // cluster-slot indices (global slot numbering)
    int fx, fy;             // occupied Fock entry multiplying the term
    int s_trans, t_trans;
    long long sblk;         // offset (doubles) of the stored coupling block
    int coupling;           // coupling id (for the adjoint accumulators)
};

// One pair inside one cluster.
struct Slot {
    int pair;               // stored pair id
    int cluster;
    long long t_off;        // offset of this slot's np x np amplitude / residual matrices
    int mult;               // 2 for i != j (ordered pairs ij and ji), 1 for ii
};

struct ClusterInfo {
    int slot0, slot1;       // [slot0, slot1) in the slot list
    int term0, term1;       // [term0, term1) in the term list
    int weight;             // MBE weight w_c
    int size;               // number of LMOs
};

// One weak pair ij (one-block scheme, Sec. 2.2.2): its n_max x n_max blocks (row-major, leading dimension n_max)
// and a 7 n_max^2 workspace.  S = Q_i Q_j^T, F = Q_i diag(eps) Q_j^T (rows of Q = OSVs), K_ur = Q_i (ia|jb) Q_j^T,
// K_ll = Q_j (ia|jb) Q_i^T; V, e, r: the pseudo-canonical bases of the pairs ii and jj; Ti, Tj: the 1b cluster
// amplitudes of ii and jj in those bases.
struct WeakPair {
    int i, j;
    const double *Kur, *Kll, *S, *F;
    const double *Vi, *Vj, *ei, *ej, *Ti, *Tj;
    const int *ri, *rj;
    double *work;
};

// Everything the residual / adjoint kernels read.
struct SolveArgs {
    const ClusterInfo *clusters;
    const int *order;       // cluster processing order (largest first)
    const Slot *slots;
    const Term *terms;
    const PairInfo *pairs;
    const int *rdim;        // per pair: pseudo-canonical dimension r_p
    const double *e;        // per pair: pseudo-canonical orbital energies (pair e_off)
    const double *Kt;       // per pair: K~ = V^T K V (np x np, pair off)
    const double *sblk;     // coupling blocks S~
    const double *focc;     // n_occ x n_occ
    int n_occ;
    double *T;              // per slot amplitudes (slot t_off)
    double *R;              // per slot residuals
    double *G1;             // per cluster scratch, gstride doubles each
    long long gstride;
    double *E_cluster;      // per cluster Hylleraas energy
    int *iters;             // per cluster iterations (-1: not converged)
    double tol;
    int max_iter;
    // mixed mode (FP32 iterations + FP64 refinement): FP32 copies of e, K~ and S~, per-slot FP32 work arrays
    const float *e32, *Kt32, *sblk32;
    float *T32, *R32, *H32;   // FP32 amplitudes / corrections, residuals, right-hand sides (per slot)
    float *G1_32;
    int *evals64;             // per cluster: FP64 residual evaluations used
    int *evals32;             // per cluster: FP32 residual evaluations (mixed solve)
    int np_max;               // largest padded pair order (shared-memory staging of the FP32 terms)
    int *next;                // work counter of the persistent cluster solve (zeroed per launch)
    int ncl;                  // clusters in the order list
};

}  // namespace osv
