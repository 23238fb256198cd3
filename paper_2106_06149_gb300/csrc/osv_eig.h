// OSV eigenproblem (Eq. 6) via tridiagonalisation, multisection and inverse iteration, the OSV-relaxation solves
// (Eq. 8), and the small parallel-Jacobi eigensolver.  The tridiagonal route is templated on the working
// precision R (double for the FP64 path; float for the first stage of the mixed path, whose results are then
// refined in FP64 by osv_refine.cu).
#pragma once
#include "kernels.cuh"

namespace osv {

// One symmetric matrix reduced in place: A (n x n, lda) -> reflectors (row k, columns k+1..), tridiagonal
// d (diagonal), e (sub-diagonal e[k] couples k and k+1), tau (reflector scalars); w: eigenvalues, decreasing.
template <class R>
struct TriDescT {
    R *A;
    long long lda;
    int n;
    R *d, *e, *tau, *w;
};
using TriDesc = TriDescT<double>;
using TriDesc32 = TriDescT<float>;

// variant (FP32 only): 0 = a pair of CTAs per matrix (thread-block cluster), 1 = one CTA per matrix, two per SM,
// 2 / 3 / 4 = a cluster of 4 / 8 / 16 CTAs per matrix (cudaErrorNotSupported when the GPU cannot hold one),
// 5 / 6 / 7 = one CTA per matrix with the updates of 2 / 2 / 4 steps written together (6: two CTAs per SM),
// 8 / 9 = variants 6 / 5 with the row chunks staged through shared memory (a second set of loads in flight),
// 10 / 11 = variant 9 with two / three chunks in flight ahead (cudaErrorNotSupported where the ring does not fit),
// 12 = variant 9 with eight rows per warp group instead of four
constexpr int kTriVariants = 13;
template <class R>
cudaError_t osv_tridiag(const TriDescT<R> *d, int batch, int n, cudaStream_t s, int variant = 0);
// The cnt largest eigenvalues of every tridiagonal (decreasing, into w[0..cnt)), by 32-point multisection in
// FP64 arithmetic (one warp per eigenvalue).
template <class R>
cudaError_t osv_tri_eigvals(const TriDescT<R> *d, int batch, int n, int cnt, cudaStream_t s);
// Kept eigenvectors (rows mu < nkeep[b] of Y, tridiagonal basis), orthonormalised.  work: 4 n nmax per matrix.
template <class R>
cudaError_t osv_tri_kept_vectors(const TriDescT<R> *d, int batch, int n, int nmax, const int *nkeep, R *Y,
                                 R *work, cudaStream_t s);
// rows mu < nrow[b] of V (nmax x n per matrix) <- H V (forward = 0) or H^T V (forward = 1)
template <class R>
cudaError_t osv_reflect(const TriDescT<R> *d, int batch, int n, int nmax, const int *nrow, R *V, int forward,
                        cudaStream_t s);
// rows mu < nkeep[b] of X -= their projection on the orthonormal rows mu < nkeep[b] of Y
template <class R>
cudaError_t osv_project_out(const int *nkeep, const R *Y, R *X, int batch, int n, int nmax, cudaStream_t s);
// X row mu = (Tri - s_mu)^{-1} (-R row mu) for mu < nkeep[b], zero rows otherwise.  Shift s_mu =
// shift[b * shift_ld + mu] (FP64) or, with shift == nullptr, the tridiagonal's own w[mu].
template <class R>
cudaError_t osv_tri_shift_solve(const TriDescT<R> *d, int batch, int n, int nmax, const int *nkeep, const R *Rin,
                                R *X, R *work, const double *shift, int shift_ld, cudaStream_t s);
// Parallel Jacobi eigensolver for symmetric matrices of order <= kJacobiMax (same descriptors and outputs as
// eigh_batched: w decreasing, eigenvectors as rows of Zt).
constexpr int kJacobiMax = 112;
cudaError_t eigh_small_jacobi(const EighDesc *d, int batch, int n_max, int *err, cudaStream_t s);
// Same contract, mixed precisions (FP32 sweeps, FP64 re-orthonormalisation and polishing sweeps) for orders
// <= kJacobiMixedMax; results to FP64 accuracy.  A descriptor's zwork (>= ne^2 / 2 doubles, ne = n rounded up
// to even) carries the FP32 stage's vectors between its two kernels; with zwork null one kernel does both.
constexpr int kJacobiMixedMax = 82;
cudaError_t eigh_small_jacobi_mixed(const EighDesc *d, int batch, int n_max, int *err, cudaStream_t s);

}  // namespace osv
