/*
 * osvmbe.h -- C ABI of libosvmbe: MBE(3)-OSV-MP2 energies and OSV-space analytical gradients on one GPU
 * (GB300, sm_103a).  Method: Q. Liang and J. Yang, "Third-order many-body expansion of OSV-MP2 wavefunction
 * for low-order scaling analytical gradient computation" (arXiv 2106.06149).
 *
 * Conventions for every entry point
 *   - Every call returns an osv_status; none aborts, traps or exits.  osv_last_error() gives a message.
 *   - "DEVICE" pointers are CUDA device pointers owned by the caller; "HOST" pointers are ordinary memory.
 *     Inputs are read, never written; outputs are written only where stated.
 *   - Work is enqueued on the stream given to osv_create (NULL = the legacy default stream).  Calls that
 *     return host values (energy, osv_build with n_osv_out, cluster_residual_solve with n_iter_out) wait
 *     for the stream; the others only enqueue.
 *   - Input buffers named in osv_problem must stay valid and unchanged from osv_build until the last
 *     gradient_backward of that problem has completed on the stream.
 *   - Matrices are row-major; "n x m" means n rows of m contiguous elements.
 *   - The context owns all intermediates (OSVs, pair bases, cluster amplitudes, densities) until the next
 *     clusters_build/osv_build on it or osv_destroy.  One context is used by one host thread at a time.
 */
#ifndef OSVMBE_H
#define OSVMBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct osv_ctx osv_ctx;

typedef enum {
    OSV_OK = 0,
    OSV_ERR_INVALID = -1,  /* bad argument, size or call order; nothing was enqueued                     */
    OSV_ERR_NOCONV = -2,   /* some cluster's residual iterations hit max_iter; results are still written  */
    OSV_ERR_OOM = -3,      /* a device allocation failed                                                   */
    OSV_ERR_CUDA = -4,     /* a CUDA runtime call failed                                                   */
    OSV_ERR_TIMEOUT = -5,  /* a bounded device loop gave up (eigensolver iteration cap)                    */
    OSV_ERR_NUMERIC = -6   /* non-finite value met (input, energy or gradient)                             */
} osv_status;

typedef enum {
    OSV_FP64 = 0,          /* every step in FP64 on the CUDA cores                                         */
    OSV_MIXED_TF32X3 = 1,  /* reserved, rejected with OSV_ERR_INVALID: split TF32 (hi*hi + hi*lo + lo*hi)
                              with FP32 accumulation over the full K is biased (E error ~1e-5 relative) and
                              misses the 1e-6 Eh bar                                                         */
    OSV_MIXED_BF16X4 = 2   /* dense DF contractions (T_kk Gram, half transforms, K blocks and the adjoint's
                              dense products) on tcgen05 tensor cores: each FP64 operand row gets a
                              power-of-two scale, is rounded to 32 bits and cut into four signed 8-bit digits
                              (exact BF16); the 13 digit products of order i + j <= 4 are accumulated in tensor
                              memory per 256-K chunk (orders 0-2 exactly, orders 3-4 rounded below 2^-40 of the
                              result) and drained into double-float sums: unbiased, ~31 significant bits of the
                              row scales.  OSV and pair-basis eigensolves run in FP32 and are refined to FP64
                              accuracy (Rayleigh-Ritz, double-float Jacobi polish); the residual iterates in
                              FP32 with FP64-accurate (double-float) evaluations and corrections; norms, energy
                              and gradient accumulation are FP64-accurate                                    */
} osv_precision;

/* Method parameters.  l_osv: OSV cut on the eigenvalues of T_kk (Sec. 2.1, Eq. 6).  r2b/r3b: distance
 * cutoffs (Angstrom) that select 2b and 3b clusters (Sec. 2.2.1; they replace the OSV-overlap metric of
 * Eqs. 26-27): a pair is kept iff |r_i - r_j| <= r2b, a triple iff its three pairs are kept and all three
 * distances are <= r3b.  mbe_order: 1, 2 or 3; 0 = one cluster holding every LMO (plain OSV-MP2). */
typedef struct {
    double l_osv;      /* keep eigenvalues > l_osv ...                                                   */
    int n_osv_max;     /* ... capped at n_osv_max (> 0; at least one OSV is always kept)                 */
    int n_osv_fixed;   /* > 0: keep exactly this many OSVs per LMO, l_osv ignored                        */
    double r2b, r3b;
    int mbe_order;
    double tau_red;    /* pair-overlap eigenvalues below tau_red are dropped (redundant pair space)      */
    double tol;        /* converged when max over the cluster's pairs of ||R~_ij||_F <= tol              */
    int max_iter;      /* residual iteration cap (>= 1)                                                  */
    int precision;     /* osv_precision                                                                  */
} osv_params;

/* One problem: n_occ localized occupied orbitals (LMOs), n_vir canonical virtuals, n_aux fitting functions.
 * B holds, for every LMO i, the DF block B_i^{aP} = (ia|P) restricted to i's local fitting domain A_i
 * (sorted aux indices aux_idx[aux_ptr[i] .. aux_ptr[i+1]-1]); B_ia^P is zero for P outside A_i
 * (orbital-specific fitting domains, Sec. 2.3, Eq. 35).  Block i starts at element aux_ptr[i] * n_vir and is
 * n_vir x a_i row-major, a_i = aux_ptr[i+1] - aux_ptr[i].  (ia|jb) = sum_P B_ia^P B_jb^P. */
typedef struct {
    int n_occ, n_vir, n_aux;
    const double *centres;   /* HOST n_occ x 3, Angstrom (cluster selection only)                         */
    const int64_t *aux_ptr;  /* HOST n_occ + 1, non-decreasing, aux_ptr[0] = 0                             */
    const int32_t *aux_idx;  /* HOST aux_ptr[n_occ] entries, each list strictly increasing, in [0, n_aux)  */
    const double *f_occ;     /* DEVICE n_occ x n_occ occupied Fock matrix in the LMO basis (Eh); must be
                                symmetric; entries are used as Eq. 4 writes them                          */
    const double *eps_vir;   /* DEVICE n_vir canonical virtual energies f_aa (Eh)                          */
    const void *B;           /* DEVICE, B_dtype elements, layout above                                     */
    int B_dtype;             /* 0 = float64, 1 = float32                                                   */
} osv_problem;

/* Create a context bound to a CUDA stream (cudaStream_t passed as void*; NULL = legacy default stream).
 * The current CUDA device at this call is the context's device; later calls switch to it. */
osv_status osv_create(osv_ctx **ctx, void *cuda_stream);
osv_status osv_destroy(osv_ctx *ctx);
/* Message describing the last error on ctx (static storage owned by ctx; "" if none; ctx may be NULL). */
const char *osv_last_error(const osv_ctx *ctx);

/* Select the 1b/2b/3b clusters and their MBE weights on the host (Sec. 2.2.1).  The weight of cluster c is
 * w_c = sum over selected supersets c' of c of (-1)^(|c'|-|c|); with it sum_c w_c X^c is the MBE(3)
 * expansion of Eqs. 28-34.  n_clusters[0..2] (HOST, may be NULL) receive the numbers of 1b, 2b, 3b clusters
 * (mbe_order 0: n_clusters[0] = 1 full cluster, others 0).  Must precede osv_build. */
osv_status clusters_build(osv_ctx *ctx, const osv_problem *prob, const osv_params *params, int *n_clusters);

/* OSV-overlap screening (Sec. 2.2.1; the paper's cluster selection, in place of the distance cutoffs):
 *   osv_overlap_metric builds the OSVs of every LMO with `params` (as osv_build does; mbe_order is ignored) and
 *   writes the metric of Eq. 2bscreen for every pair of LMOs, s2b_ij = sum_{mu in i, nu in j} <mu|nu>^2 /
 *   sqrt(n_i n_j), <mu|nu> the entries of Q_i^T Q_j, into s2b_out (HOST n_occ x n_occ, row-major; 0 <= s2b <= 1,
 *   s2b_ii = 1).  The Gram of the OSVs runs on the precision mode's dense back end (exact BF16 slices on the
 *   tensor cores in OSV_MIXED_BF16X4).  Synchronises.  It replaces any earlier plan on ctx: call
 *   clusters_build_osv next.
 *   clusters_build_osv is clusters_build with the selection rule of Eqs. 2bscreen and 3bscreen: pair ij (i < j)
 *   is a 2b cluster iff s2b[i][j] > l2b; triple ijk is a 3b cluster iff its three pairs are 2b clusters and
 *   (s2b_ij + s2b_ik + s2b_jk) / 3 > l3b (entries read at i < j); r2b and r3b of params are not used.  MBE
 *   weights, mbe_order and the rest of the plan as in clusters_build.  OSV_ERR_INVALID for a NULL or non-finite
 *   s2b. */
osv_status osv_overlap_metric(osv_ctx *ctx, const osv_problem *prob, const osv_params *params, double *s2b_out);
osv_status clusters_build_osv(osv_ctx *ctx, const osv_problem *prob, const osv_params *params, const double *s2b,
                              double l2b, double l3b, int *n_clusters);

/* Build orbital-specific virtuals and all pair quantities for the selected clusters (steps on the device):
 *   T_kk = (ka|kb) / (eps_a + eps_b - 2 f_kk), eigenpairs to FP64 accuracy (FP64 tridiagonal route, or FP32
 *   with FP64 Rayleigh-Ritz refinement in OSV_MIXED_BF16X4), Q_k = eigenvectors of the n_k largest eigenvalues
 *   (Sec. 2.1, Eqs. 5-6; the discarded space enters the OSV relaxation of Eq. 8 only through the resolvent of
 *   T_kk restricted to it, so its eigenvectors are never formed);
 *   S, F and K blocks A_(ij,kl) = (Q_i Q_j)^T A (Q_k Q_l) (Eq. 7) with K over the common fitting domain;
 *   per pair an orthonormal pseudo-canonical basis of (Q_i Q_j).
 * n_osv_out: HOST n_occ ints receiving n_k (may be NULL; non-NULL synchronises the stream). */
osv_status osv_build(osv_ctx *ctx, const osv_problem *prob, const osv_params *params, int *n_osv_out);

/* Solve the cluster residual equations (Eq. 4, sum over k restricted to the cluster, Sec. 2.2.1) for every
 * cluster to max_ij ||R~_ij||_F <= tol, and the cluster Hylleraas energies (Eq. 3).
 * n_iter_out: HOST int receiving the largest iteration count over clusters (may be NULL; non-NULL
 * synchronises).  cluster_status: DEVICE int32 per cluster (may be NULL): iterations used, or -1 where the
 * cluster did not converge.  Returns OSV_ERR_NOCONV (after a synchronisation) if any cluster did not
 * converge and n_iter_out is non-NULL; otherwise the failure is reported by the next energy() call. */
osv_status cluster_residual_solve(osv_ctx *ctx, int *n_iter_out, int32_t *cluster_status);

/* Collective pair amplitudes T_(ij,ij) = sum over clusters c containing i, j of w_c T^c_(ij,ij)
 * (MBE(3), Eqs. 28-32). */
osv_status mbe3_combine(osv_ctx *ctx);

/* Weak 2b clusters by the one-block scheme (Sec. 2.2.2), after cluster_residual_solve: every pair ij (i < j) with
 * l_discard <= s2b[i][j] <= l2b that belongs to no selected cluster is a weak pair.  Its amplitudes are the upper-
 * right block X of T_(ij,ij) (rows: the OSVs of i, columns: those of j), solving the upper-right block of the 2b
 * cluster's Eq. 4 with the pairs ii and jj held at their 1b cluster amplitudes (directly, in the pseudo-canonical
 * bases of ii and jj); its energy is the Hylleraas functional (Eq. 3) of the ordered pairs ij and ji.
 * *E_weak (HOST) = the sum over weak pairs, to be added to energy()'s E (the strong clusters); *n_weak (HOST, may
 * be NULL) = their number.  Pairs with s2b below l_discard are dropped.  No weak pairs below mbe_order 2.  The
 * cross half transforms Q_j B_i, Q_i B_j run on the dense back end, the per-pair blocks in FP64.  Synchronises. */
osv_status weak_pairs_energy(osv_ctx *ctx, const double *s2b, double l2b, double l_discard, double *E_weak,
                             int *n_weak);

/* One-step posterior correction over the collective amplitudes (Sec. 3, the estimate beyond MBE(3)), after
 * mbe3_combine.  For every pair ij of a selected cluster, Eq. 4 is evaluated at the collective amplitudes T with
 * k running over the LMOs of every selected cluster that holds both i and j, and one step of the cluster
 * solver's preconditioned update is taken, T' = T - R~ / (e_a + e_b - f_ii - f_jj) in the pair's
 * pseudo-canonical basis.  HOST outputs: *E_global = sum over ordered pairs of <K + R(T), 2T - T^T>, *E_corrected
 * the same functional at T', *dR_max (may be NULL) = max over pairs of ||R~(T)||_F.  FP64 evaluations (double-
 * float in OSV_MIXED_BF16X4).  Synchronises; OSV_ERR_NUMERIC for a non-finite result. */
osv_status posterior_correction(osv_ctx *ctx, double *E_global, double *E_corrected, double *dR_max);

/* E = sum_c w_c E^c_Hylleraas (Eq. 3 per cluster, MBE-combined) into *E_out (HOST);
 * E_linear_out (HOST, may be NULL) = sum_ij <K_(ij,ij), 2T - T^T> with the collective amplitudes.
 * Synchronises the stream.  Returns OSV_ERR_NOCONV if any cluster of the last cluster_residual_solve hit
 * max_iter (E and E_linear are still written), OSV_ERR_NUMERIC if E is not finite. */
osv_status energy(osv_ctx *ctx, double *E_out, double *E_linear_out);

/* Adjoint of the energy (amplitudes are variational, Sec. 2.1): accumulate dE_scale * dE/dB into dE_dB
 * (DEVICE, same layout and dtype as prob->B) and dE_scale * dE/df_occ into dE_dFocc (DEVICE n_occ x n_occ
 * float64, entrywise derivative with F used as given).  Includes the OSV relaxation through the discarded
 * eigenvectors of T_kk (Sec. 2.1, Eq. 8) and the MBE(3) combination of the pair densities (Eqs. 33-34).
 * The buffers are added to (+=), not overwritten; either may be NULL to skip it.  Half-transformed
 * integrals are recomputed, not stored.  Synchronises the stream and returns OSV_ERR_TIMEOUT or
 * OSV_ERR_NUMERIC if a device step of the build, the solve or the adjoint reported one. */
osv_status gradient_backward(osv_ctx *ctx, double dE_scale, void *dE_dB, double *dE_dFocc);

/* One whole step recorded as a CUDA graph (no counterpart in the paper; the per-geometry loop of an energy and
 * gradient calculation).  osv_graph_capture first runs one eager step (osv_build -> cluster_residual_solve ->
 * mbe3_combine -> energy, and gradient_backward when dE_dB or dE_dFocc is non-NULL), which plans and tunes a new
 * shape and reports any failure of the step itself; it then records the same step, from the T_kk Gram to the
 * gradient outputs, as one graph: every launch, the zeroing of dE_dB and dE_dFocc (DEVICE, as in
 * gradient_backward, but OVERWRITTEN by the step rather than added to) and the copies of E, E_linear, the error
 * word and the per-cluster iteration counts into a pinned host block.  clusters_build must precede it.  The graph
 * holds the device addresses of prob (B, f_occ, eps_vir), of dE_dB and of dE_dFocc and the parameters as given:
 * change their VALUES in place between launches (a new geometry), never their addresses, sizes or the parameters
 * (capture again instead).  osv_graph_launch replays the step on the context's stream, synchronises and returns E
 * and E_linear (HOST, either may be NULL) with energy()'s and gradient_backward()'s error rules (OSV_ERR_NOCONV,
 * OSV_ERR_NUMERIC, OSV_ERR_TIMEOUT).  Any call that re-plans (clusters_build, osv_build of another shape or
 * precision, osv_overlap_metric) drops the graph; osv_graph_launch then returns OSV_ERR_INVALID.
 * osv_graph_kernels: the kernels one replay launches (0 without a graph); the launch counter of
 * osv_kernel_launches grows by that much per replay and not at all while recording. */
osv_status osv_graph_capture(osv_ctx *ctx, const osv_problem *prob, const osv_params *params, double dE_scale,
                             void *dE_dB, double *dE_dFocc);
osv_status osv_graph_launch(osv_ctx *ctx, double *E_out, double *E_linear_out);
osv_status osv_graph_kernels(osv_ctx *ctx, long long *count);

/* Autotuner of the launch shapes (no counterpart in the paper).  When a context plans a problem in the mixed
 * precision (the first osv_build of a new shape), it times on the device, with CUDA events, the candidate launch
 * shapes of its tunable kernels and keeps the fastest: the FP32 Householder tridiagonalisation (a pair of CTAs per
 * matrix, one CTA per matrix and two per SM, a cluster of 4, 8 or 16 CTAs per matrix, or one CTA per matrix with
 * delayed updates) and the tile shape of every double-float GEMM batch whose problems
 * all overwrite their outputs.  Results do not depend on the choice beyond rounding order.  osv_autotune(ctx, 0)
 * turns it off for later plans (the fixed rules then apply); it is on by default.  osv_autotune_report writes the
 * last plan's choices as a NUL-terminated JSON object into buf (HOST, len bytes, may be NULL), with the fixed
 * rule's choice, the tuned one and the timings per item, and *needed (HOST, may be NULL) = the bytes the whole
 * report takes; "" when nothing was tuned. */
osv_status osv_autotune(osv_ctx *ctx, int on);
osv_status osv_autotune_report(osv_ctx *ctx, char *buf, int len, int *needed);
/* Fix the launch shape of the FP32 tridiagonalisation for this context's later plans instead of tuning it:
 * 0 = a pair of CTAs per matrix, 1 = one CTA per matrix and two per SM, 2 / 3 / 4 = a cluster of 4 / 8 / 16 CTAs
 * per matrix (one per SM; fewer matrices in flight, so their trailing matrices stay in L2), 5 / 6 / 7 = one CTA per
 * matrix that writes the rank-2 updates of 2 / 2 / 4 steps into the trailing matrix together (6: two CTAs per SM;
 * fewer bytes written), 8 / 9 = variants 6 / 5 with the row chunks staged through shared memory, 10 / 11 = variant
 * 9 with two / three chunks in flight ahead, 12 = variant 9 with eight rows per warp group; -1 = tuned again (the
 * default).  The results differ only in rounding order.  OSV_ERR_INVALID out of range; a later osv_build reports
 * OSV_ERR_CUDA if the GPU cannot hold one cluster of the chosen size. */
osv_status osv_set_tridiag_variant(osv_ctx *ctx, int variant);

/* Failure detection (no counterpart in the paper): every wait of the tensor-core kernels on their pipeline
 * barriers is bounded; when a wait runs out the kernel raises OSV_ERR_TIMEOUT in the context's error word, lets
 * the work it already committed finish, frees its tensor memory and returns.  osv_set_wait_budget sets the bound
 * of those waits for this context's later calls, in SM clock cycles (cycles <= 0 restores the default of 2^32,
 * about two seconds).  A tiny budget makes the waits run out on purpose, which is how the timeout path is tested;
 * results computed under an expired wait are meaningless and the call that reads the error word reports it. */
osv_status osv_set_wait_budget(osv_ctx *ctx, long long cycles);

/* Diagnostics (all synchronise; HOST outputs):
 *   osv_cluster_count: number of clusters (all orders).
 *   osv_cluster_info: members[3*c..3*c+2] (-1 padded; mbe_order 0 reports the first 3 members only),
 *     weight[c], energy[c] (cluster Hylleraas energy E^c), iters[c] (-1 = not converged); any may be NULL.
 *   osv_eigenvalues: the n_vir eigenvalues of T_kk of LMO k, decreasing. */
osv_status osv_cluster_count(osv_ctx *ctx, int *n_clusters);
osv_status osv_cluster_info(osv_ctx *ctx, int32_t *members, int32_t *weight, double *energy, int32_t *iters);
osv_status osv_eigenvalues(osv_ctx *ctx, int k, double *w_out);
/* Collective amplitudes of the ordered pair (i, j) after mbe3_combine (Eqs. 28-32), in the canonical virtual
 * space: t_out (HOST n_vir x n_vir) = (Q_i Q_j) T_(ij,ij) (Q_i Q_j)^T, rows indexed by the virtuals of i's
 * side; t_ji = t_ij^T.  The pair must lie in a selected cluster (OSV_ERR_INVALID otherwise).  Formed on the
 * host from the device's OSVs, pair basis and amplitudes (a diagnostic, not part of the hot path). */
osv_status osv_pair_amplitudes(osv_ctx *ctx, int i, int j, double *t_out);

/* Per-stage timing: osv_profile_enable(ctx, 1) clears previous records and makes every later call record a
 * pair of CUDA events around each of its stages on the context's stream; (ctx, 0) stops and clears.  A recorded
 * step (osv_graph_capture) carries its own stage events, and each osv_graph_launch made while profiling is on adds
 * their times.
 * osv_profile_read (synchronises) returns the stages in first-seen order: names[32*q] (NUL-terminated, up to
 * 31 chars), summed milliseconds ms[q] and number of records calls[q] for q < min(max_stages, *n_stages);
 * names, ms, calls may be NULL.  Profiling adds event records; leave it off when capturing a CUDA graph. */
osv_status osv_profile_enable(osv_ctx *ctx, int on);
osv_status osv_profile_read(osv_ctx *ctx, int max_stages, char *names, double *ms, int *calls, int *n_stages);

/* Algorithmic FLOPs of the last cluster_residual_solve (synchronises): for every cluster, the number of
 * residual evaluations (iterations + 1) times the sum over its coupling terms of Eq. 4 of
 * 2 (r_p r_q^2 + r_p^2 r_q), r the pseudo-canonical pair dimensions; the O(r^2) diagonal terms are not
 * counted.  HOST *flops. */
osv_status osv_residual_flops(osv_ctx *ctx, double *flops);

/* Algorithmic FLOPs of the per-cluster partials of gradient_backward (the densities of Eqs. 14-16, 33-34 in
 * the pseudo-canonical pair bases), for the clusters of the last solve with a non-zero MBE weight: per pair of
 * order r, 8 r^3 (Tb L T^T + T^T L Tb and Tb T^T + T^T Tb); per coupling term (r_p, r_q),
 * 4 r_p^2 r_q + 4 r_p r_q^2 (Tb S~, Tb^T S~, then those times T~' and T~'^T).  Synchronises.  HOST *flops. */
osv_status osv_adjoint_flops(osv_ctx *ctx, double *flops);

/* Iteration statistics of the last cluster_residual_solve (synchronises), summed over clusters:
 * *updates32 = FP32 Jacobi updates (mixed modes: first solve and correction solves; 0 in FP64 mode),
 * *evals64 = FP64-accurate residual evaluations (FP64 mode: iterations + 1 per cluster), *unconverged =
 * clusters that hit max_iter (their FP32 updates are not counted).  HOST outputs. */
osv_status osv_solve_counts(osv_ctx *ctx, long long *updates32, long long *evals64, int *unconverged);

/* Coupling-term FLOPs of the last cluster_residual_solve split by arithmetic (synchronises): per cluster the
 * per-evaluation count of osv_residual_flops times its FP32 evaluations (*flops32; 0 in FP64 mode) and times its
 * FP64-accurate evaluations (*flops64: FP64 units in FP64 mode, double-float on the FP32 pipe in the mixed
 * modes).  HOST outputs. */
osv_status osv_residual_work(osv_ctx *ctx, double *flops32, double *flops64);

/* Process-wide number of CUDA kernel launches issued by this library so far (HOST *count). */
osv_status osv_kernel_launches(long long *count);

/* Batched symmetric eigensolver used for Eq. 6 (utility entry point): for b = 0..batch-1, the n x n
 * symmetric matrix A + b*n*n (DEVICE, read only) gets eigenvalues w + b*n (DEVICE, decreasing) and
 * eigenvectors as rows of Zt + b*n*n (DEVICE; row mu is the eigenvector of w[mu]).  Householder
 * tridiagonalisation and implicit QL in FP64.  Allocates 2*batch*n*n doubles of scratch with cudaMalloc per
 * call and frees it before returning; synchronises the stream.  1 <= n <= 4096. */
osv_status osv_syev_batched(const double *A, int n, int batch, double *w, double *Zt, void *cuda_stream);

/* Allocation-free variant of osv_syev_batched (the paper has no counterpart: this is a service for callers).
 * For callers that cannot call cudaMalloc: code running under an external memory manager that owns the whole
 * device memory, where a stray cudaMalloc fails or fragments its pool, and latency-sensitive callers that
 * cannot take the device-wide synchronisation of cudaFree.  Same arguments, results and error codes as
 * osv_syev_batched, except:
 *   - no cudaMalloc / cudaFree: scratch is a static device array of 2^20 doubles (8 MiB) plus 1024 matrix
 *     descriptors, held by every GPU that loads the library until the process exits;
 *   - limits: batch <= 1024 and batch*n*n + 3*batch*n <= 1048576; larger requests return OSV_ERR_INVALID with
 *     the numbers in osv_last_error(NULL);
 *   - Zt doubles as the working matrix (A may equal Zt for an in-place call);
 *   - every call looks up the static array's device address (cudaGetSymbolAddress with the calling thread's
 *     current device); the first call on each device also loads the library's device code there, so make that
 *     first call before any stream capture;
 *   - every call shares the one static array (the error word is cleared on each call): calls that overlap on
 *     the GPU, from several host threads or streams, race and must be serialised by the caller.
 * Synchronises the stream. */
osv_status osv_syev_batched_noalloc(const double *A, int n, int batch, double *w, double *Zt, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* OSVMBE_H */
