// OSV eigenproblem (Eq. 6) via tridiagonalisation, bisection and inverse iteration, the OSV-relaxation solves
// (Eq. 8), and the small parallel-Jacobi eigensolver.
#pragma once
#include "kernels.cuh"

namespace osv {

// One symmetric matrix reduced in place: A (n x n, lda) -> reflectors (row k, columns k+1..), tridiagonal
// d (diagonal), e (sub-diagonal e[k] couples k and k+1), tau (reflector scalars); w: eigenvalues, decreasing.
struct TriDesc {
    double *A;
    long long lda;
    int n;
    double *d, *e, *tau, *w;
};

cudaError_t osv_tridiag(const TriDesc *d, int batch, int n, cudaStream_t s);
cudaError_t osv_tri_eigvals(const TriDesc *d, int batch, int n, cudaStream_t s);
// Kept eigenvectors (rows mu < nkeep[b] of Y, tridiagonal basis), orthonormalised.  work: 4 n nmax per matrix.
cudaError_t osv_tri_kept_vectors(const TriDesc *d, int batch, int n, int nmax, const int *nkeep, double *Y,
                                 double *work, cudaStream_t s);
// rows mu < nrow[b] of V (nmax x n per matrix) <- H V (forward = 0) or H^T V (forward = 1)
cudaError_t osv_reflect(const TriDesc *d, int batch, int n, int nmax, const int *nrow, double *V, int forward,
                        cudaStream_t s);
// rows mu < nkeep[b] of X -= their projection on the orthonormal rows mu < nkeep[b] of Y
cudaError_t osv_project_out(const int *nkeep, const double *Y, double *X, int batch, int n, int nmax, cudaStream_t s);
// X row mu = (Tri - w_mu)^{-1} (-R row mu) for mu < nkeep[b], zero rows otherwise
cudaError_t osv_tri_shift_solve(const TriDesc *d, int batch, int n, int nmax, const int *nkeep, const double *R,
                                double *X, double *work, cudaStream_t s);
// Parallel Jacobi eigensolver for symmetric matrices of order <= kJacobiMax (same descriptors and outputs as
// eigh_batched: w decreasing, eigenvectors as rows of Zt).
constexpr int kJacobiMax = 112;
cudaError_t eigh_small_jacobi(const EighDesc *d, int batch, int n_max, int *err, cudaStream_t s);

}  // namespace osv
