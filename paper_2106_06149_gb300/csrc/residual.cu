// Cluster residual solver (Eq. 4 per cluster, Sec. 2.2.1), MBE(3) combination (Eqs. 28-32) and the
// Hylleraas energy (Eq. 3), FP64.
//
// Each pair ij of a cluster works in the orthonormal pseudo-canonical basis Phi_ij = (Q_i Q_j) V_ij of its own
// domain (V^T S_(ij,ij) V = 1, V^T F_(ij,ij) V = diag(e)).  Projected on it, Eq. 4 reads
//   R~_ij = K~_ij + (e_a + e_b - f_ii - f_jj) T~_ij - sum_{k != j} f_kj S~ T~_ik S~^T - sum_{k != i} f_ik S~ T~_kj S~^T
// with S~ = Phi_ij^T Phi_(other pair) and k running over the cluster's LMOs; the Jacobi update is
// T~ -= R~ / (e_a + e_b - f_ii - f_jj).  One CTA owns one cluster for all its iterations; the small
// products run as block-cooperative register-tiled FP64 GEMMs.
#include "kernels.cuh"
#include "launch.h"

namespace osv {

namespace {

constexpr int kThreads = 256;

// C (M x N) = alpha * op(A) op(B) (+ C if accumulate).  op(A)(m,k) = ta ? A[k*lda+m] : A[m*lda+k],
// op(B)(k,n) = tb ? B[n*ldb+k] : B[k*ldb+n].  Block-cooperative, 4 x 4 outputs per thread and tile.
__device__ void blk_gemm(int M, int N, int K, const double *__restrict__ A, long long lda, bool ta,
                         const double *__restrict__ B, long long ldb, bool tb, double *C, long long ldc,
                         double alpha, bool accumulate) {
    const int mt = (M + 3) >> 2, nt = (N + 3) >> 2;
    for (int t = threadIdx.x; t < mt * nt; t += blockDim.x) {
        const int bm = (t / nt) << 2, bn = (t % nt) << 2;
        double acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
        for (int k = 0; k < K; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int m = bm + i;
                a[i] = m < M ? (ta ? A[(long long)k * lda + m] : A[(long long)m * lda + k]) : 0.0;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = bn + j;
                b[j] = n < N ? (tb ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n]) : 0.0;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = bm + i;
            if (m >= M) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = bn + j;
                if (n >= N) continue;
                double *c = C + (long long)m * ldc + n;
                *c = accumulate ? *c + alpha * acc[i][j] : alpha * acc[i][j];
            }
        }
    }
}

__device__ __forceinline__ double denom(const double *e, int a, int b, double fii, double fjj) {
    return e[a] + e[b] - fii - fjj;
}

__global__ void __launch_bounds__(kThreads) k_residual(SolveArgs A) {
    const int c = A.order[blockIdx.x];
    const ClusterInfo C = A.clusters[c];
    __shared__ double red[kThreads / 32];
    double *G1 = A.G1 + (long long)blockIdx.x * A.gstride;
    const int tid = threadIdx.x;
    bool conv = false;
    int it = 0;
    for (;; ++it) {
        // R~ = K~ + D o T~
        for (int s = C.slot0; s < C.slot1; ++s) {
            const Slot S = A.slots[s];
            const PairInfo P = A.pairs[S.pair];
            const int r = A.rdim[S.pair], np = P.np;
            const double fii = A.focc[(long long)P.i * A.n_occ + P.i], fjj = A.focc[(long long)P.j * A.n_occ + P.j];
            const double *e = A.e + P.e_off;
            for (int idx = tid; idx < r * r; idx += kThreads) {
                const int a = idx / r, b = idx % r;
                const long long o = (long long)a * np + b;
                A.R[S.t_off + o] = A.Kt[P.off + o] + denom(e, a, b, fii, fjj) * A.T[S.t_off + o];
            }
        }
        __syncthreads();
        // coupling terms
        for (int t = C.term0; t < C.term1; ++t) {
            const Term T = A.terms[t];
            const Slot Sd = A.slots[T.dst], Ss = A.slots[T.src];
            const PairInfo Pd = A.pairs[Sd.pair], Ps = A.pairs[Ss.pair];
            const int rp = A.rdim[Sd.pair], rq = A.rdim[Ss.pair];
            const double f = A.focc[(long long)T.fx * A.n_occ + T.fy];
            const double *Sb = A.sblk + T.sblk;
            // stored block is (smaller pair id) x (larger pair id)
            const long long lds = T.s_trans ? Pd.np : Ps.np;
            // G1 = S~_pq T~'_q   (rp x rq)
            blk_gemm(rp, rq, rq, Sb, lds, T.s_trans, A.T + Ss.t_off, Ps.np, T.t_trans, G1, Ps.np, 1.0, false);
            __syncthreads();
            // R~_p -= f G1 S~_pq^T
            blk_gemm(rp, rp, rq, G1, Ps.np, false, Sb, lds, !T.s_trans, A.R + Sd.t_off, Pd.np, -f, true);
            __syncthreads();
        }
        // max over pairs of ||R~||_F
        double rmax = 0.0;
        for (int s = C.slot0; s < C.slot1; ++s) {
            const Slot S = A.slots[s];
            const PairInfo P = A.pairs[S.pair];
            const int r = A.rdim[S.pair], np = P.np;
            double ss = 0.0;
            for (int idx = tid; idx < r * r; idx += kThreads) {
                const double v = A.R[S.t_off + (long long)(idx / r) * np + idx % r];
                ss += v * v;
            }
            rmax = fmax(rmax, sqrt(block_sum(ss, red)));
        }
        if (!(rmax > A.tol)) {   // converged (a NaN norm also stops here and is caught by energy())
            conv = rmax <= A.tol;
            break;
        }
        if (it >= A.max_iter) break;
        for (int s = C.slot0; s < C.slot1; ++s) {
            const Slot S = A.slots[s];
            const PairInfo P = A.pairs[S.pair];
            const int r = A.rdim[S.pair], np = P.np;
            const double fii = A.focc[(long long)P.i * A.n_occ + P.i], fjj = A.focc[(long long)P.j * A.n_occ + P.j];
            const double *e = A.e + P.e_off;
            for (int idx = tid; idx < r * r; idx += kThreads) {
                const int a = idx / r, b = idx % r;
                const long long o = S.t_off + (long long)a * np + b;
                A.T[o] -= A.R[o] / denom(e, a, b, fii, fjj);
            }
        }
        __syncthreads();
    }
    // cluster Hylleraas energy: sum over ordered pairs of <K~ + R~, 2T~ - T~^T>
    double E = 0.0;
    for (int s = C.slot0; s < C.slot1; ++s) {
        const Slot S = A.slots[s];
        const PairInfo P = A.pairs[S.pair];
        const int r = A.rdim[S.pair], np = P.np;
        double acc = 0.0;
        for (int idx = tid; idx < r * r; idx += kThreads) {
            const int a = idx / r, b = idx % r;
            const long long o = (long long)a * np + b;
            const double tbar = 2.0 * A.T[S.t_off + o] - A.T[S.t_off + (long long)b * np + a];
            acc += (A.Kt[P.off + o] + A.R[S.t_off + o]) * tbar;
        }
        E += S.mult * block_sum(acc, red);
    }
    if (tid == 0) {
        A.E_cluster[c] = E;
        A.iters[c] = conv ? it : -1;
    }
}

// Collective amplitudes: T~coll_p = sum over clusters containing p of w_c T~^c_p (Eqs. 28-32).
__global__ void k_combine(const PairInfo *__restrict__ pairs, const int *__restrict__ ptr,
                          const long long *__restrict__ src, const int *__restrict__ w,
                          const double *__restrict__ T, double *__restrict__ Tc) {
    const int p = blockIdx.x;
    const PairInfo P = pairs[p];
    const long long nn = (long long)P.np * P.np;
    for (long long idx = threadIdx.x; idx < nn; idx += blockDim.x) {
        double acc = 0.0;
        for (int q = ptr[p]; q < ptr[p + 1]; ++q) acc += w[q] * T[src[q] + idx];
        Tc[P.off + idx] = acc;
    }
}

// Per-pair linear energy term mult * <K~, 2T~coll - T~coll^T>.
__global__ void k_pair_linear(const PairInfo *__restrict__ pairs, const int *__restrict__ rdim,
                              const double *__restrict__ Kt, const double *__restrict__ Tc,
                              double *__restrict__ out) {
    const int p = blockIdx.x;
    const PairInfo P = pairs[p];
    const int r = rdim[p], np = P.np;
    __shared__ double red[kThreads / 32];
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
        const int a = idx / r, b = idx % r;
        acc += Kt[P.off + (long long)a * np + b] *
               (2.0 * Tc[P.off + (long long)a * np + b] - Tc[P.off + (long long)b * np + a]);
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[p] = (P.i == P.j ? 1.0 : 2.0) * acc;
}

// E = sum_c w_c E^c and E_lin = sum_p lin_p, deterministic order.
__global__ void k_energy_final(const double *__restrict__ Ec, const ClusterInfo *__restrict__ cl, int ncl,
                               const double *__restrict__ lin, int npairs, double *__restrict__ out) {
    __shared__ double red[kThreads / 32];
    double a = 0.0, b = 0.0;
    for (int c = threadIdx.x; c < ncl; c += blockDim.x) a += cl[c].weight * Ec[c];
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) b += lin[p];
    a = block_sum(a, red);
    b = block_sum(b, red);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

}  // namespace

cudaError_t launch_residual(const SolveArgs &a, int nclusters, cudaStream_t s) {
    if (nclusters <= 0) return cudaSuccess;
    count_launch();
    k_residual<<<nclusters, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_combine(const PairInfo *pairs, int npairs, const int *ptr, const long long *src, const int *w,
                           const double *T, double *Tc, cudaStream_t s) {
    if (npairs <= 0) return cudaSuccess;
    count_launch();
    k_combine<<<npairs, kThreads, 0, s>>>(pairs, ptr, src, w, T, Tc);
    return cudaGetLastError();
}

cudaError_t launch_energy(const PairInfo *pairs, const int *rdim, const double *Kt, const double *Tc, int npairs,
                          double *lin, const double *Ec, const ClusterInfo *cl, int ncl, double *out,
                          cudaStream_t s) {
    if (npairs > 0) { count_launch(); k_pair_linear<<<npairs, kThreads, 0, s>>>(pairs, rdim, Kt, Tc, lin); }
    count_launch();
    k_energy_final<<<1, kThreads, 0, s>>>(Ec, cl, ncl, lin, npairs, out);
    return cudaGetLastError();
}

}  // namespace osv
