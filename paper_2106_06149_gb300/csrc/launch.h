// Host-side launchers of the device kernels (each returns the launch status; none synchronises).
#pragma once
#include <algorithm>

#include "kernels.cuh"

namespace osv {

cudaError_t launch_f32_to_f64(const float *in, double *out, long long n, cudaStream_t s);
// T_kk (FP64, in place over the Gram products) and a working copy in W (double or float) for the eigensolver
template <class W>
cudaError_t launch_tkk_scale(double *T, W *work, const double *eps, const double *focc, int n_occ, int nv, int *err,
                             cudaStream_t s);
cudaError_t launch_osv_count(const double *omega, int ld, int *nosv, int n_occ, int nmax, double l_osv, int n_fixed,
                             cudaStream_t s);
cudaError_t launch_s2b(const double *G, const int *nosv, int n, int nm, double *s, cudaStream_t st);
cudaError_t launch_scale_cols(const double *Q, const double *eps, double *Qe, long long rows, int nv, cudaStream_t s);
cudaError_t launch_block_copy(const BlockCopy *d_bc, int n, cudaStream_t s);
cudaError_t launch_pair_x(const PairInfo *pairs, int npairs, const double *Ut, const double *sv, double *X,
                          int *rdim, double tau_red, cudaStream_t s);
cudaError_t launch_clean_w(const PairInfo *pairs, int npairs, const int *rdim, double *Wt, double *e,
                           cudaStream_t s);
cudaError_t launch_residual(const SolveArgs &a, int nclusters, bool mixed, cudaStream_t s);
// one-block amplitudes and energies of weak pairs (E per pair)
cudaError_t launch_weak_pairs(const WeakPair *wp, int nweak, int nm, const double *focc, int n_occ, double *E,
                              cudaStream_t s);
// one-step posterior correction: R1 = R(Tc), T2 = Tc - R1 / D, R2 = R(T2), per-pair norms (rnorm[0, np) of R1,
// rnorm[np, 2np) of R2) and pair functionals E1 (at Tc), E2 (at T2)
cudaError_t launch_posterior(const SolveArgs &a, int npairs, const double *Tc, double *R1, double *T2, double *R2,
                             double *rnorm, double *E1, double *E2, bool df, cudaStream_t s);
cudaError_t launch_to_f32(const double *in, float *out, long long n, cudaStream_t s);
cudaError_t launch_combine(const PairInfo *pairs, int npairs, const int *ptr, const long long *src, const int *w,
                           const double *T, double *Tc, cudaStream_t s);
cudaError_t launch_energy(const PairInfo *pairs, const int *rdim, const double *Kt, const double *Tc, int npairs,
                          double *lin, const double *Ec, const ClusterInfo *cl, int ncl, double *out,
                          cudaStream_t s);

}  // namespace osv
