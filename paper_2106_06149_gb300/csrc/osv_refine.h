// Mixed-precision OSV eigenproblem (Eq. 6) and OSV-relaxation solves (Eq. 8): an FP32 tridiagonal route
// gives starting vectors and a preconditioner, FP64 Rayleigh-Ritz refinement gives the eigenpairs.
#pragma once
#include <vector>

#include "osv_eig.h"

namespace osv {

// Largest n_max (kept OSVs per LMO) the refinement handles (its Rayleigh-Ritz step lives in shared memory).
constexpr int kRefineMaxN = 64;
// FP64 correction steps of the eigenvector refinement and of the relaxation solve.
constexpr int kOsvRefineSteps = 2;
constexpr int kRelaxRefineSteps = 1;

struct OsvRefine {
    // FP32 copy of T_kk reduced in place (reflectors), its tridiagonal, the FP32 kept vectors (tridiagonal
    // basis), inverse-iteration work, and two FP32 row blocks for the preconditioner
    float *A32 = nullptr, *d32 = nullptr, *e32 = nullptr, *tau32 = nullptr, *w32 = nullptr, *Y32 = nullptr,
          *work32 = nullptr, *X32 = nullptr, *Z32 = nullptr;
    std::vector<TriDesc32> tri_h;
    TriDesc32 *tri_d = nullptr;
    // per LMO: QW = [Q; W] (2 nm x n_vir, W = Q T), [G; H] = QW Q^T (2 nm x nm), Rayleigh-Ritz rotation Ct
    // (nm x nm), Ritz values lam (nm)
    double *QW[2] = {nullptr, nullptr}, *GH = nullptr, *Ct = nullptr, *lam = nullptr;
    double *AT = nullptr, *RS = nullptr;   // relaxation: a T and the FP64 residual (nm x n_vir per LMO)
    int *nm_all = nullptr;                 // n_max for every LMO (rows refined)
    float *Twy = nullptr;                  // compact-WY T factors of the FP32 reflectors (osv_wy_floats)
    int tri_variant = 0;                   // FP32 tridiagonalisation launch shape (osv_tridiag), set by the autotuner
    GemmBatch gb_w[2], gb_gh[2], gb_rot[2], gb_fin[2];
};

// Q (nm x n_vir per LMO, rows >= n_k zero), omega[b * n_vir + mu] (mu < nm) and nosv from T_kk, whose FP32
// copy r.A32 has been written.  err receives kDevNonFinite if a Gram matrix is not positive definite and
// kDevEighNoConv if a Rayleigh-Ritz Jacobi solve hits its sweep cap.
cudaError_t osv_mixed_eigh(const OsvRefine &r, int n_occ, int nv, int nm, double *Q, double *omega, int *nosv,
                           double l_osv, int n_fixed, int *err, cudaStream_t s, int steps = kOsvRefineSteps);
// a = (omega_mu - T)^{-1} g_mu on the discarded space of each LMO (g: rows mu < nosv, already projected),
// to FP64 accuracy: FP32 preconditioner plus kRelaxRefineSteps FP64 residual corrections; gb_at computes
// r.AT = a T.  Rows >= nosv of a are zero.
cudaError_t osv_mixed_relax(const OsvRefine &r, const GemmBatch &gb_at, int n_occ, int nv, int nm, const double *Q,
                            const int *nosv, const double *g, double *a, cudaStream_t s);

// Blocked FP32 reflector products: T factors of every block of kNB reflectors (osv_wy_floats(batch, n) floats),
// then rows mu < nrow[b] of V <- H V (forward = 0) or H^T V (forward = 1), same contract as osv_reflect<float>.
size_t osv_wy_floats(int batch, int n);
cudaError_t osv_wy_prepare(const TriDesc32 *d, int batch, int n, float *T, cudaStream_t s);
cudaError_t osv_reflect_wy(const TriDesc32 *d, const float *T, int batch, int n, int nmax, const int *nrow, float *V,
                           int forward, cudaStream_t s);
// Same contract as osv_project_out, for nmax <= 64: FP32 arithmetic for float, double-float for double.
bool osv_project_rows_fits(int n, int nmax);
template <class R>
cudaError_t osv_project_rows(const int *nkeep, const R *Y, R *X, int batch, int n, int nmax, cudaStream_t s);

}  // namespace osv
