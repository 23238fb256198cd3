// Element-wise and bookkeeping kernels of the OSV build (Sec. 2.1, Eqs. 5-7).
#include "kernels.cuh"
#include "launch.h"

namespace osv {

namespace {

__global__ void k_f32_to_f64(const float *__restrict__ in, double *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

// T_kk = (ka|kb) / (eps_a + eps_b - 2 f_kk)  (Eq. 6); the Gram product (ka|kb) is already in T.
// A copy goes to `work` (overwritten by the eigensolver).  Non-finite entries raise the error word.
template <class W>
__global__ void k_tkk_scale(double *__restrict__ T, W *__restrict__ work, const double *__restrict__ eps,
                            const double *__restrict__ focc, int n_occ, int nv, int *err) {
    const int k = blockIdx.y;
    const double fkk = focc[(long long)k * n_occ + k];
    const long long nn = (long long)nv * nv;
    double *Tk = T + (long long)k * nn;
    W *Wk = work + (long long)k * nn;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nn;
         idx += (long long)gridDim.x * blockDim.x) {
        const int a = int(idx / nv), b = int(idx % nv);
        const double v = Tk[idx] / (eps[a] + eps[b] - 2.0 * fkk);
        if (!isfinite(v)) raise_err(err, kDevNonFinite);
        Tk[idx] = v;
        Wk[idx] = (W)v;
    }
}

// n_k from the decreasing eigenvalues: #(omega > l_osv) capped at nmax (or fixed), at least one (Eq. 6).  Only
// the leading nmax eigenvalues (row stride ld) are read.
__global__ void k_osv_count(const double *__restrict__ omega, int ld, int *__restrict__ nosv, int n_occ, int nmax,
                            double l_osv, int n_fixed) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_occ) return;
    const double *w = omega + (long long)k * ld;
    int n;
    if (n_fixed > 0) {
        n = min(n_fixed, nmax);
    } else {
        n = 0;
        while (n < nmax && w[n] > l_osv) ++n;
    }
    nosv[k] = max(n, 1);
}

// Qe[r][a] = Q[r][a] * eps[a] over all rows of all LMOs.
__global__ void k_scale_cols(const double *__restrict__ Q, const double *__restrict__ eps, double *__restrict__ Qe,
                             long long rows, int nv) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < rows * nv;
         idx += (long long)gridDim.x * blockDim.x)
        Qe[idx] = Q[idx] * eps[idx % nv];
}

__global__ void k_block_copy(const BlockCopy *__restrict__ bc) {
    const BlockCopy b = bc[blockIdx.x];
    const long long nel = (long long)b.rows * b.cols;
    for (long long idx = threadIdx.x; idx < nel; idx += blockDim.x) {
        const int r = int(idx / b.cols), c = int(idx % b.cols);
        const double v = b.scale * (b.trans ? b.src[(long long)c * b.lds + r] : b.src[(long long)r * b.lds + c]);
        double *d = b.dst + (long long)r * b.ldd + c;
        if (b.accumulate) atomicAdd(d, v);
        else *d = v;
    }
}

// Orthonormal basis of the pair domain from S_pp = U diag(s) U^T (U in rows of Ut, s decreasing):
// X[:, c] = U[:, c] / sqrt(s_c) for s_c > tau_red, zero columns otherwise; r_p = number kept.
__global__ void k_pair_x(const PairInfo *__restrict__ pairs, const double *__restrict__ Ut,
                         const double *__restrict__ s, double *__restrict__ X, int *__restrict__ rdim,
                         double tau_red) {
    const PairInfo P = pairs[blockIdx.x];
    const int np = P.np;
    __shared__ int s_r;
    if (threadIdx.x == 0) {
        int r = 0;
        while (r < np && s[P.e_off + r] > tau_red) ++r;
        s_r = r;
        rdim[blockIdx.x] = r;
    }
    __syncthreads();
    const int r = s_r;
    for (long long idx = threadIdx.x; idx < (long long)np * np; idx += blockDim.x) {
        const int a = int(idx / np), c = int(idx % np);
        X[P.off + idx] = c < r ? Ut[P.off + (long long)c * np + a] / sqrt(s[P.e_off + c]) : 0.0;
    }
}

// After the r_p x r_p pseudo-canonical eigensolve: zero the eigenvector rows/columns beyond r_p and the
// unused eigenvalue slots, so that V = X W^T has exactly r_p non-zero columns.
__global__ void k_clean_w(const PairInfo *__restrict__ pairs, const int *__restrict__ rdim,
                          double *__restrict__ Wt, double *__restrict__ e) {
    const PairInfo P = pairs[blockIdx.x];
    const int np = P.np, r = rdim[blockIdx.x];
    for (long long idx = threadIdx.x; idx < (long long)np * np; idx += blockDim.x) {
        const int a = int(idx / np), c = int(idx % np);
        if (a >= r || c >= r) Wt[P.off + idx] = 0.0;
    }
    for (int a = r + threadIdx.x; a < np; a += blockDim.x) e[P.e_off + a] = 0.0;
}

// OSV-overlap metric of Sec. 2.2.1, Eq. 2bscreen, from the Gram G of all OSV rows (row i*nm + mu is OSV mu of
// LMO i, zero beyond n_i): s_ij = sum over the n_i x n_j block of G^2 / sqrt(n_i n_j).  One CTA per (i, j).
__global__ void k_s2b(const double *__restrict__ G, const int *__restrict__ nosv, int n, int nm,
                      double *__restrict__ s) {
    const int i = blockIdx.y, j = blockIdx.x;
    const long long ld = (long long)n * nm;
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < nm * nm; idx += blockDim.x) {
        const int mu = idx / nm, nu = idx % nm;
        const double g = G[(long long)(i * nm + mu) * ld + (long long)j * nm + nu];
        acc = fma(g, g, acc);
    }
    __shared__ double red[32];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) s[(long long)i * n + j] = acc / sqrt((double)nosv[i] * (double)nosv[j]);
}

}  // namespace

cudaError_t launch_s2b(const double *G, const int *nosv, int n, int nm, double *s, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    k_s2b<<<dim3(n, n), 128, 0, st>>>(G, nosv, n, nm, s);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float *in, double *out, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    count_launch();
    k_f32_to_f64<<<blocks, 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

template <class W>
cudaError_t launch_tkk_scale(double *T, W *work, const double *eps, const double *focc, int n_occ, int nv, int *err,
                             cudaStream_t s) {
    if (n_occ <= 0) return cudaSuccess;
    const long long nn = (long long)nv * nv;
    const int bx = (int)std::min<long long>((nn + 255) / 256, 64);
    count_launch();
    k_tkk_scale<W><<<dim3(bx, n_occ), 256, 0, s>>>(T, work, eps, focc, n_occ, nv, err);
    return cudaGetLastError();
}
template cudaError_t launch_tkk_scale<double>(double *, double *, const double *, const double *, int, int, int *,
                                              cudaStream_t);
template cudaError_t launch_tkk_scale<float>(double *, float *, const double *, const double *, int, int, int *,
                                             cudaStream_t);

cudaError_t launch_osv_count(const double *omega, int ld, int *nosv, int n_occ, int nmax, double l_osv, int n_fixed,
                             cudaStream_t s) {
    if (n_occ <= 0) return cudaSuccess;
    count_launch();
    k_osv_count<<<(n_occ + 127) / 128, 128, 0, s>>>(omega, ld, nosv, n_occ, nmax, l_osv, n_fixed);
    return cudaGetLastError();
}

cudaError_t launch_scale_cols(const double *Q, const double *eps, double *Qe, long long rows, int nv, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    const int blocks = (int)std::min<long long>((rows * nv + 255) / 256, 152LL * 8);
    count_launch();
    k_scale_cols<<<blocks, 256, 0, s>>>(Q, eps, Qe, rows, nv);
    return cudaGetLastError();
}

cudaError_t launch_block_copy(const BlockCopy *d_bc, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    k_block_copy<<<n, 256, 0, s>>>(d_bc);
    return cudaGetLastError();
}

cudaError_t launch_pair_x(const PairInfo *pairs, int npairs, const double *Ut, const double *sv, double *X,
                          int *rdim, double tau_red, cudaStream_t s) {
    if (npairs <= 0) return cudaSuccess;
    count_launch();
    k_pair_x<<<npairs, 256, 0, s>>>(pairs, Ut, sv, X, rdim, tau_red);
    return cudaGetLastError();
}

cudaError_t launch_clean_w(const PairInfo *pairs, int npairs, const int *rdim, double *Wt, double *e,
                           cudaStream_t s) {
    if (npairs <= 0) return cudaSuccess;
    count_launch();
    k_clean_w<<<npairs, 256, 0, s>>>(pairs, rdim, Wt, e);
    return cudaGetLastError();
}

}  // namespace osv
