// Weak 2b clusters by the one-block scheme (Sec. 2.2.2): the pair amplitudes of a weak pair ij are restricted to
// their upper-right block X (rows: the OSVs of i, columns: those of j), T_(ij,ij) = [[0, X], [0, 0]], and X solves
// the upper-right block of the 2b cluster's residual (Eq. 4) with the diagonal pairs held at their 1b cluster
// amplitudes.  With orthonormal OSVs per LMO that block is the Sylvester equation
//   (F_ii - f_ii) X + X (F_jj - f_jj) = -K_ur + f_ij (T_ii S + S T_jj),
// K_ur = Q_i^T (ia|jb) Q_j, S = Q_i^T Q_j, F_xy = Q_x^T diag(eps) Q_y, which is diagonal in the pseudo-canonical
// bases V_ii, V_jj of the pairs ii and jj (V^T F V = diag(e)): X = V_ii [(V_ii^T RHS V_jj) / (e_a + e_b - f_ii -
// f_jj)] V_jj^T.  The weak pair's energy is the Hylleraas functional (Eq. 3) of the ordered pairs ij and ji, which
// are transposes of one another; with the upper-right residual block zero it reads
//   E_w = 2 (2 <K_ur, X> - <M_ll, X^T>),
//   M_ll = Q_j^T (K + R) Q_i = 2 K_ll + F^T X S^T + S^T X F^T - (f_ii + f_jj) S^T X S^T - f_ij (S^T T_ii + T_jj S^T),
// K_ll = Q_j^T (ia|jb) Q_i, F = F_ij.  One CTA per weak pair, FP64 (the blocks are at most n_max x n_max).
#include "kernels.cuh"
#include "launch.h"

namespace osv {

namespace {

constexpr int kThreads = 256;

// C = alpha op(A) op(B) + beta C, all n x n row-major with leading dimension n (block-cooperative, global memory)
__device__ void mm(int n, const double *__restrict__ A, bool ta, const double *__restrict__ B, bool tb, double *C,
                   double alpha, double beta) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int m = idx / n, c = idx % n;
        double acc = 0.0;
        for (int k = 0; k < n; ++k)
            acc = fma(ta ? A[k * n + m] : A[m * n + k], tb ? B[c * n + k] : B[k * n + c], acc);
        C[idx] = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * C[idx]);
    }
    __syncthreads();
}

__device__ double dot(int n, const double *__restrict__ A, const double *__restrict__ B, bool tb, double *red) {
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int m = idx / n, c = idx % n;
        acc = fma(A[idx], tb ? B[c * n + m] : B[idx], acc);
    }
    return block_sum(acc, red);
}

__global__ void __launch_bounds__(kThreads) k_weak_pair(const WeakPair *__restrict__ wp, int nm, const double *focc,
                                                        int n_occ, double *__restrict__ E) {
    const WeakPair P = wp[blockIdx.x];
    __shared__ double red[kThreads / 32];
    const long long nn = (long long)nm * nm;
    double *Tii = P.work, *Tjj = Tii + nn, *R = Tjj + nn, *X = R + nn, *M = X + nn, *t1 = M + nn, *t2 = t1 + nn;
    const double fii = focc[(long long)P.i * n_occ + P.i], fjj = focc[(long long)P.j * n_occ + P.j];
    const double fij = focc[(long long)P.i * n_occ + P.j];
    const int ri = *P.ri, rj = *P.rj;
    // 1b amplitudes in the OSV basis: T = V T~ V^T
    mm(nm, P.Vi, false, P.Ti, false, t1, 1.0, 0.0);
    mm(nm, t1, false, P.Vi, true, Tii, 1.0, 0.0);
    mm(nm, P.Vj, false, P.Tj, false, t1, 1.0, 0.0);
    mm(nm, t1, false, P.Vj, true, Tjj, 1.0, 0.0);
    // RHS = -K_ur + f_ij (T_ii S + S T_jj)
    mm(nm, Tii, false, P.S, false, t1, 1.0, 0.0);
    mm(nm, P.S, false, Tjj, false, t1, 1.0, 1.0);
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) R[idx] = fij * t1[idx] - P.Kur[idx];
    __syncthreads();
    // X = V_ii [(V_ii^T RHS V_jj) / (e_a + e_b - f_ii - f_jj)] V_jj^T
    mm(nm, P.Vi, true, R, false, t1, 1.0, 0.0);
    mm(nm, t1, false, P.Vj, false, t2, 1.0, 0.0);
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
        const int a = idx / nm, b = idx % nm;
        t2[idx] = (a < ri && b < rj) ? t2[idx] / (P.ei[a] + P.ej[b] - fii - fjj) : 0.0;
    }
    __syncthreads();
    mm(nm, P.Vi, false, t2, false, t1, 1.0, 0.0);
    mm(nm, t1, false, P.Vj, true, X, 1.0, 0.0);
    // M_ll = (F - (f_ii + f_jj) S)^T X S^T + S^T X F^T + 2 K_ll - f_ij (S^T T_ii + T_jj S^T)
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) R[idx] = P.F[idx] - (fii + fjj) * P.S[idx];
    __syncthreads();
    mm(nm, X, false, P.S, true, t1, 1.0, 0.0);          // X S^T
    mm(nm, R, true, t1, false, M, 1.0, 0.0);            // (F - (f_ii + f_jj) S)^T X S^T
    mm(nm, X, false, P.F, true, t1, 1.0, 0.0);          // X F^T
    mm(nm, P.S, true, t1, false, M, 1.0, 1.0);          // + S^T X F^T
    mm(nm, P.S, true, Tii, false, t1, 1.0, 0.0);        // S^T T_ii
    mm(nm, Tjj, false, P.S, true, t1, 1.0, 1.0);        // + T_jj S^T
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) M[idx] += 2.0 * P.Kll[idx] - fij * t1[idx];
    __syncthreads();
    const double a = dot(nm, P.Kur, X, false, red);
    const double b = dot(nm, M, X, true, red);
    if (threadIdx.x == 0) E[blockIdx.x] = 2.0 * (2.0 * a - b);
}

}  // namespace

cudaError_t launch_weak_pairs(const WeakPair *wp, int nweak, int nm, const double *focc, int n_occ, double *E,
                              cudaStream_t s) {
    if (nweak <= 0) return cudaSuccess;
    count_launch();
    k_weak_pair<<<nweak, kThreads, 0, s>>>(wp, nm, focc, n_occ, E);
    return cudaGetLastError();
}

}  // namespace osv
