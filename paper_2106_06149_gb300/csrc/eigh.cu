// Batched dense symmetric eigensolver in FP64 (OSV eigenproblem of Eq. 6 and the pair-overlap / pseudo-
// canonical problems of the pair bases).  Three launches per batch:
//   1. Householder tridiagonalisation, one CTA per matrix, in place (reflectors stored below the diagonal);
//   2. explicit Q = H_0 H_1 ... H_{n-3}, row-parallel: each thread owns rows of Q, several CTAs per matrix;
//   3. implicit QL with Wilkinson shifts on the tridiagonal matrix (Bowdler, Martin, Reinsch and Wilkinson,
//      Numer. Math. 11 (1968) 293), the plane rotations of each sweep applied to the rows of Z = Q in
//      parallel; then eigenpairs sorted by decreasing eigenvalue.
// Every loop is bounded: a QL iteration cap sets an error word instead of spinning.
#include <cfloat>

#include "common.cuh"

namespace osv {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxQlIter = 60;

__device__ __forceinline__ int order_of(const EighDesc &D) { return D.n_dev ? min(*D.n_dev, D.n) : D.n; }

// ---------------------------------------------------------------------------------- 1. tridiagonalise
__global__ void __launch_bounds__(kThreads) k_tridiag(const EighDesc *__restrict__ descs) {
    const EighDesc D = descs[blockIdx.x];
    const int n = order_of(D);
    extern __shared__ double sh[];
    double *v = sh;                 // reflector, length <= n
    double *p = sh + D.n;           // A v, then w
    __shared__ double red[kThreads / 32];
    __shared__ double s_beta;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = kThreads / 32;
    double *A = D.A;
    const long long lda = D.lda;
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        double ss = 0.0;
        for (int r = tid; r < m; r += kThreads) {
            const double x = A[(long long)(k + 1 + r) * lda + k];
            v[r] = x;
            ss += x * x;
        }
        ss = block_sum(ss, red);
        const double alpha = sqrt(ss);
        if (tid == 0) {
            const double x0 = v[0];   // only thread 0 reads v[0] before rewriting it
            D.d[k] = A[(long long)k * lda + k];
            if (alpha == 0.0) {
                D.e[k] = 0.0;
                D.tau[k] = 0.0;
                s_beta = 0.0;
            } else {
                const double sgn = x0 >= 0.0 ? 1.0 : -1.0;
                v[0] = x0 + sgn * alpha;
                D.e[k] = -sgn * alpha;
                s_beta = 1.0 / (alpha * (alpha + fabs(x0)));
                D.tau[k] = s_beta;
            }
        }
        __syncthreads();
        const double beta = s_beta;
        if (beta == 0.0) continue;   // column already reduced; its (zero) entries double as the reflector
        // p = beta * A' v, one warp per row of the trailing block A' = A[k+1:, k+1:]
        for (int r = wid; r < m; r += nw) {
            const double *row = A + (long long)(k + 1 + r) * lda + (k + 1);
            double s = 0.0;
            for (int c = lane; c < m; c += 32) s += row[c] * v[c];
            s = warp_sum(s);
            if (lane == 0) p[r] = beta * s;
        }
        __syncthreads();
        double pv = 0.0;
        for (int r = tid; r < m; r += kThreads) pv += p[r] * v[r];
        const double kc = 0.5 * beta * block_sum(pv, red);
        for (int r = tid; r < m; r += kThreads) p[r] -= kc * v[r];   // w = p - K v
        __syncthreads();
        // A' <- A' - v w^T - w v^T
        for (long long idx = tid; idx < (long long)m * m; idx += kThreads) {
            const int r = int(idx / m), c = int(idx % m);
            A[(long long)(k + 1 + r) * lda + (k + 1 + c)] -= v[r] * p[c] + p[r] * v[c];
        }
        // keep the reflector in column k below the diagonal for the Q formation
        for (int r = tid; r < m; r += kThreads) A[(long long)(k + 1 + r) * lda + k] = v[r];
        __syncthreads();
    }
    if (tid == 0) {
        if (n >= 2) {
            D.d[n - 2] = A[(long long)(n - 2) * lda + (n - 2)];
            D.e[n - 2] = A[(long long)(n - 1) * lda + (n - 2)];
            D.tau[n - 2] = 0.0;
        }
        if (n >= 1) {
            D.d[n - 1] = A[(long long)(n - 1) * lda + (n - 1)];
            D.e[n - 1] = 0.0;
            D.tau[n - 1] = 0.0;
        }
    }
}

// ----------------------------------------------------------------------------------------- 2. form Q
// zwork is column-major: Q(r, c) at zwork[c * D.n + r]; CTA blockIdx.y owns rows [y*chunk, (y+1)*chunk).
__global__ void __launch_bounds__(kThreads) k_form_q(const EighDesc *__restrict__ descs, int chunk) {
    const EighDesc D = descs[blockIdx.x];
    const int n = order_of(D);
    const int r0 = blockIdx.y * chunk;
    if (r0 >= n) return;
    const int r1 = min(n, r0 + chunk);
    extern __shared__ double v[];
    const long long ld = D.n;
    double *Z = D.zwork;
    for (int r = r0 + threadIdx.x; r < r1; r += kThreads)
        for (int c = 0; c < n; ++c) Z[c * ld + r] = (c == r) ? 1.0 : 0.0;
    for (int k = 0; k + 2 < n; ++k) {
        const double beta = D.tau[k];
        if (beta == 0.0) continue;
        const int m = n - k - 1;
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += kThreads) v[i] = D.A[(long long)(k + 1 + i) * D.lda + k];
        __syncthreads();
        for (int r = r0 + threadIdx.x; r < r1; r += kThreads) {
            double *z = Z + (long long)(k + 1) * ld + r;
            double s = 0.0;
            for (int i = 0; i < m; ++i) s += z[i * ld] * v[i];
            s *= beta;
            for (int i = 0; i < m; ++i) z[i * ld] -= s * v[i];
        }
    }
}

// ------------------------------------------------------------------------------ 3. QL, sort, write out
__global__ void __launch_bounds__(kThreads) k_ql(const EighDesc *__restrict__ descs, int chunk, int *err) {
    const EighDesc D = descs[blockIdx.x];
    const int n = order_of(D);
    const int r0 = blockIdx.y * chunk;
    if (r0 >= n) return;
    const int r1 = min(n, r0 + chunk);
    extern __shared__ double sh[];
    double *d = sh, *e = sh + D.n, *cs = sh + 2 * D.n, *sn = sh + 3 * D.n;
    int *rank = reinterpret_cast<int *>(sh + 4 * D.n);
    __shared__ int s_state, s_lo, s_hi;
    const int tid = threadIdx.x;
    const long long ld = D.n;
    double *Z = D.zwork;
    for (int i = tid; i < n; i += kThreads) {
        d[i] = D.d[i];
        e[i] = D.e[i];
    }
    __syncthreads();
    bool failed = false;
    for (int l = 0; l < n && !failed; ++l) {
        for (int iter = 0;; ++iter) {
            if (tid == 0) {
                int m = l;
                while (m < n - 1) {
                    const double dd = fabs(d[m]) + fabs(d[m + 1]);
                    if (fabs(e[m]) <= DBL_EPSILON * dd) break;
                    ++m;
                }
                if (m == l) {
                    s_state = 0;
                } else if (iter >= kMaxQlIter) {
                    s_state = 2;
                } else {
                    // shift from the leading 2 x 2 block, then chase the bulge from m-1 down to l
                    double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
                    double r = hypot(g, 1.0);
                    g = d[m] - d[l] + e[l] / (g + copysign(r, g));
                    double s = 1.0, c = 1.0, p = 0.0;
                    int lo = l;
                    bool early = false;
                    for (int i = m - 1; i >= l; --i) {
                        const double f = s * e[i], b = c * e[i];
                        r = hypot(f, g);
                        e[i + 1] = r;
                        if (r == 0.0) {
                            d[i + 1] -= p;
                            e[m] = 0.0;
                            lo = i + 1;
                            early = true;
                            break;
                        }
                        s = f / r;
                        c = g / r;
                        g = d[i + 1] - p;
                        r = (d[i] - g) * s + 2.0 * c * b;
                        p = s * r;
                        d[i + 1] = g + p;
                        g = c * r - b;
                        cs[i] = c;
                        sn[i] = s;
                    }
                    if (!early) {
                        d[l] -= p;
                        e[l] = g;
                        e[m] = 0.0;
                    }
                    s_lo = lo;
                    s_hi = m;
                    s_state = 1;
                }
            }
            __syncthreads();
            const int state = s_state;
            if (state == 1) {
                const int lo = s_lo, hi = s_hi;
                for (int r = r0 + tid; r < r1; r += kThreads) {
                    double carry = Z[(long long)hi * ld + r];
                    for (int i = hi - 1; i >= lo; --i) {
                        const double zi = Z[(long long)i * ld + r];
                        Z[(long long)(i + 1) * ld + r] = sn[i] * zi + cs[i] * carry;
                        carry = cs[i] * zi - sn[i] * carry;
                    }
                    Z[(long long)lo * ld + r] = carry;
                }
            }
            __syncthreads();
            if (state == 2) {
                failed = true;
                if (tid == 0 && blockIdx.y == 0) raise_err(err, kDevEighNoConv);
            }
            if (state != 1) break;
        }
    }
    // stable rank by decreasing eigenvalue
    for (int i = tid; i < n; i += kThreads) {
        const double di = d[i];
        int rk = 0;
        for (int j = 0; j < n; ++j) rk += (d[j] > di) || (d[j] == di && j < i);
        rank[i] = rk;
    }
    __syncthreads();
    if (blockIdx.y == 0)
        for (int i = tid; i < n; i += kThreads) D.w[rank[i]] = d[i];
    for (int c = 0; c < n; ++c) {
        const long long dst = (long long)rank[c] * D.ldz;
        for (int r = r0 + tid; r < r1; r += kThreads) D.Zt[dst + r] = Z[(long long)c * ld + r];
    }
}

}  // namespace

cudaError_t eigh_batched(const EighDesc *d_desc, int batch, int n_max, int rows_split, int *err,
                         cudaStream_t s) {
    if (batch <= 0 || n_max <= 0) return cudaSuccess;
    const int split = rows_split > 0 ? rows_split : (n_max + kThreads - 1) / kThreads;
    const int chunk = (n_max + split - 1) / split;
    const size_t sh1 = 2 * (size_t)n_max * sizeof(double);
    const size_t sh2 = (size_t)n_max * sizeof(double);
    const size_t sh3 = 4 * (size_t)n_max * sizeof(double) + (size_t)n_max * sizeof(int);
    cudaError_t e;
    if (sh3 > 48 * 1024) {
        e = cudaFuncSetAttribute(k_ql, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh3);
        if (e != cudaSuccess) return e;
    }
    if (sh1 > 48 * 1024) {
        e = cudaFuncSetAttribute(k_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh1);
        if (e != cudaSuccess) return e;
    }
    count_launch();
    k_tridiag<<<batch, kThreads, sh1, s>>>(d_desc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    count_launch();
    k_form_q<<<dim3(batch, split), kThreads, sh2, s>>>(d_desc, chunk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    count_launch();
    k_ql<<<dim3(batch, split), kThreads, sh3, s>>>(d_desc, chunk, err);
    return cudaGetLastError();
}

}  // namespace osv
