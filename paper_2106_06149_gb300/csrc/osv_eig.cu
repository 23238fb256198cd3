// OSV eigenproblem of Eq. 6 without a full eigendecomposition, and small dense eigensolves by parallel Jacobi.
//
// Only the n_k kept eigenvectors of T_kk enter the energy, and the OSV relaxation of Eq. 8 needs the discarded
// eigenvectors only through the restricted resolvent sum_nu q'_nu q'_nu^T / (omega_mu - omega'_nu).  So:
//   1. Householder tridiagonalisation T = H Tri H^T (one CTA per LMO; reflector k kept contiguous in row k);
//   2. every eigenvalue of Tri by bisection on the Sturm count, one thread per eigenvalue (parallel, no long
//      dependent chain: on GB300 a dependent FP64 operation costs ~64 cycles and a division ~430);
//   3. the kept eigenvectors by inverse iteration on Tri, one thread per vector, then two classical Gram-Schmidt
//      passes (CGS2) inside the kept set;
//   4. back-transformation q = H y through the stored reflectors (warp per vector);
//   5. (adjoint) x_mu = P_perp (omega_mu - Tri)^{-1} P_perp r_mu by a pivoted tridiagonal solve and a CGS2
//      projection, which is exactly the kept x discarded block of the perturbed eigenproblem (Eq. 8).
// Pair overlap / pseudo-canonical eigenproblems (order <= 2 nmax) use a cyclic parallel Jacobi in shared memory.
#include <cfloat>

#include "kernels.cuh"
#include "osv_eig.h"

namespace osv {

namespace {

constexpr int kT = 256;

// ---------------------------------------------------------------------- 1. Householder tridiagonalisation
// A (n x n, lda) overwritten; d, e (n), tau (n); reflector k stored in row k, columns k+1 .. n-1.
__global__ void __launch_bounds__(kT) k_tridiag_osv(const TriDesc *__restrict__ descs) {
    const TriDesc D = descs[blockIdx.x];
    const int n = D.n;
    extern __shared__ double sh[];
    double *v = sh, *p = sh + n;
    __shared__ double red[kT / 32];
    __shared__ double s_beta;
    const int tid = threadIdx.x;
    double *A = D.A;
    const long long lda = D.lda;
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        double ss = 0.0;
        // column k below the diagonal equals row k right of the diagonal (symmetric storage, both kept)
        for (int r = tid; r < m; r += kT) {
            const double x = A[(long long)k * lda + (k + 1 + r)];
            v[r] = x;
            ss += x * x;
        }
        ss = block_sum(ss, red);
        const double alpha = sqrt(ss);
        if (tid == 0) {
            const double x0 = v[0];
            D.d[k] = A[(long long)k * lda + k];
            if (alpha == 0.0) {
                D.e[k] = 0.0;
                s_beta = 0.0;
            } else {
                const double sgn = x0 >= 0.0 ? 1.0 : -1.0;
                v[0] = x0 + sgn * alpha;
                D.e[k] = -sgn * alpha;
                s_beta = 1.0 / (alpha * (alpha + fabs(x0)));
            }
            D.tau[k] = s_beta;
        }
        __syncthreads();
        const double beta = s_beta;
        if (beta != 0.0) {
            // p = beta A' v with A'(r, c) read as A(c, r) (symmetric), coalesced over r; 4 accumulators
            for (int r = tid; r < m; r += kT) {
                double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                const double *col = A + (long long)(k + 1) * lda + (k + 1 + r);
                int c = 0;
                for (; c + 3 < m; c += 4) {
                    a0 = fma(col[(long long)c * lda], v[c], a0);
                    a1 = fma(col[(long long)(c + 1) * lda], v[c + 1], a1);
                    a2 = fma(col[(long long)(c + 2) * lda], v[c + 2], a2);
                    a3 = fma(col[(long long)(c + 3) * lda], v[c + 3], a3);
                }
                for (; c < m; ++c) a0 = fma(col[(long long)c * lda], v[c], a0);
                p[r] = beta * ((a0 + a1) + (a2 + a3));
            }
            __syncthreads();
            double pv = 0.0;
            for (int r = tid; r < m; r += kT) pv += p[r] * v[r];
            const double kc = 0.5 * beta * block_sum(pv, red);
            for (int r = tid; r < m; r += kT) p[r] -= kc * v[r];
            __syncthreads();
            for (long long idx = tid; idx < (long long)m * m; idx += kT) {
                const int r = int(idx / m), c = int(idx % m);
                A[(long long)(k + 1 + r) * lda + (k + 1 + c)] -= v[r] * p[c] + p[r] * v[c];
            }
        }
        // reflector into row k (the row is not read again by the reduction)
        for (int r = tid; r < m; r += kT) A[(long long)k * lda + (k + 1 + r)] = beta != 0.0 ? v[r] : 0.0;
        __syncthreads();
    }
    if (tid == 0) {
        if (n >= 2) {
            D.d[n - 2] = A[(long long)(n - 2) * lda + (n - 2)];
            D.e[n - 2] = A[(long long)(n - 1) * lda + (n - 2)];
            D.tau[n - 2] = 0.0;
        }
        D.d[n - 1] = A[(long long)(n - 1) * lda + (n - 1)];
        D.e[n - 1] = 0.0;
        D.tau[n - 1] = 0.0;
        if (n >= 2) A[(long long)(n - 2) * lda + (n - 1)] = 0.0;   // no reflector for the last two rows
    }
}

// ------------------------------------------------------------------------------------- 2. bisection
// Number of eigenvalues below x: sign changes of the leading principal minors p_i = det(T_0..i - x), computed by
// the three-term recurrence p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (no division: on GB300 an FP64
// division costs ~430 cycles of latency, a multiply-add 64).  Every four steps both carried minors are rescaled
// by an exact power of two, which keeps them finite without changing any sign.  pivmin stands in for an exactly
// zero minor.
__device__ __forceinline__ int sturm_below(const double *d, const double *e2, int n, double x, double pivmin) {
    double pm = 1.0, pc = d[0] - x;
    if (pc == 0.0) pc = -pivmin;
    int cnt = pc < 0.0;
    for (int i = 1; i < n; ++i) {
        double pn = fma(d[i] - x, pc, -e2[i - 1] * pm);
        if (pn == 0.0) pn = (pc < 0.0 ? pivmin : -pivmin) * fabs(pc);   // treat as a tiny value of opposite sign
        cnt += (pn < 0.0) != (pc < 0.0);
        pm = pc;
        pc = pn;
        if ((i & 3) == 0) {
            const double a = fabs(pc);
            if (a > 0x1p+600) {
                pc *= 0x1p-600;
                pm *= 0x1p-600;
            } else if (a < 0x1p-600) {
                pc *= 0x1p+600;
                pm *= 0x1p+600;
            }
        }
    }
    return cnt;
}

// All eigenvalues of each tridiagonal matrix, decreasing, into w (one thread per eigenvalue).
__global__ void __launch_bounds__(kT) k_tri_bisect(const TriDesc *__restrict__ descs) {
    const TriDesc D = descs[blockIdx.x];
    const int n = D.n;
    extern __shared__ double sh[];
    double *d = sh, *e2 = sh + n;
    __shared__ double s_lo, s_hi, s_piv;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        d[i] = D.d[i];
        e2[i] = D.e[i] * D.e[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double lo = DBL_MAX, hi = -DBL_MAX, emax = 0.0;
        for (int i = 0; i < n; ++i) {
            const double r = (i > 0 ? fabs(D.e[i - 1]) : 0.0) + (i + 1 < n ? fabs(D.e[i]) : 0.0);
            lo = fmin(lo, d[i] - r);
            hi = fmax(hi, d[i] + r);
            emax = fmax(emax, e2[i]);
        }
        const double span = fmax(hi - lo, fmax(fabs(lo), fabs(hi)));
        s_lo = lo - 2.0 * DBL_EPSILON * span - 1e-300;
        s_hi = hi + 2.0 * DBL_EPSILON * span + 1e-300;
        s_piv = 1e-30;   // relative size of a stand-in for an exactly vanishing minor
        (void)emax;
    }
    __syncthreads();
    for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < n; j += gridDim.y * blockDim.x) {
        const int k = n - 1 - j;          // j-th largest = k-th smallest (0-based)
        double lo = s_lo, hi = s_hi;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 1e-300) break;
            if (sturm_below(d, e2, n, mid, s_piv) <= k) lo = mid;
            else hi = mid;
        }
        D.w[j] = 0.5 * (lo + hi);
    }
}

// ------------------------------------------------------------ pivoted tridiagonal solve (one thread)
// Solves (Tri - shift) x = rhs.  Work arrays u0,u1,u2 (U rows: diagonal, first and second super-diagonal) and
// the right-hand side / solution x live in global memory at stride `st` (interleaved across threads).
__device__ void tri_solve(const double *d, const double *e, int n, double shift, double *x, double *u0,
                          double *u1, double *u2, long long st, double pivmin) {
    // current row i as (p, q) on columns i, i+1 (no fill yet), rhs in x
    double p = d[0] - shift, q = n > 1 ? e[0] : 0.0;
    for (int i = 0; i + 1 < n; ++i) {
        const double l = e[i];                       // entry (i+1, i)
        const double a = d[i + 1] - shift;           // (i+1, i+1)
        const double b = i + 2 < n ? e[i + 1] : 0.0; // (i+1, i+2)
        double xi = x[(long long)i * st], xn = x[(long long)(i + 1) * st];
        if (fabs(p) >= fabs(l)) {
            if (fabs(p) < pivmin) p = p < 0.0 ? -pivmin : pivmin;
            const double mlt = l / p;
            u0[(long long)i * st] = p;
            u1[(long long)i * st] = q;
            u2[(long long)i * st] = 0.0;
            x[(long long)(i + 1) * st] = xn - mlt * xi;
            p = a - mlt * q;
            q = b;
        } else {
            const double mlt = p / l;
            u0[(long long)i * st] = l;
            u1[(long long)i * st] = a;
            u2[(long long)i * st] = b;
            x[(long long)i * st] = xn;
            x[(long long)(i + 1) * st] = xi - mlt * xn;
            p = q - mlt * a;
            q = -mlt * b;
        }
    }
    if (fabs(p) < pivmin) p = p < 0.0 ? -pivmin : pivmin;
    u0[(long long)(n - 1) * st] = p;
    // back substitution
    double x1 = x[(long long)(n - 1) * st] / p, x2 = 0.0;
    x[(long long)(n - 1) * st] = x1;
    for (int i = n - 2; i >= 0; --i) {
        const double xi = (x[(long long)i * st] - u1[(long long)i * st] * x1 - u2[(long long)i * st] * x2) /
                          u0[(long long)i * st];
        x[(long long)i * st] = xi;
        x2 = x1;
        x1 = xi;
    }
}

// ------------------------------------------------------------------------ 3. inverse iteration (kept)
// Thread (matrix b, vector mu < n_k): two inverse-iteration solves from a pseudo-random start; the result (not
// yet orthogonalised) goes to Y row mu (Y: nmax x n per matrix, row-major).
__global__ void __launch_bounds__(64) k_tri_invit(const TriDesc *__restrict__ descs, const int *__restrict__ nkeep,
                                                  double *__restrict__ Y, double *__restrict__ work, int nmax) {
    const int b = blockIdx.x;
    const TriDesc D = descs[b];
    const int n = D.n;
    const int mu = blockIdx.y * blockDim.x + threadIdx.x;
    const int nk = nkeep[b];
    if (mu >= nk) return;
    const long long st = nmax;
    double *base = work + (long long)b * 4 * n * nmax;
    double *x = base + mu, *u0 = base + (long long)n * nmax + mu, *u1 = base + 2LL * n * nmax + mu,
           *u2 = base + 3LL * n * nmax + mu;
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i) tnorm = fmax(tnorm, fabs(D.d[i]) + fabs(D.e[i]) + (i ? fabs(D.e[i - 1]) : 0.0));
    const double pivmin = fmax(tnorm, 1e-300) * DBL_EPSILON * 1e-3;
    const double lam = D.w[mu];
    unsigned h = 2166136261u ^ (unsigned)(mu * 7919 + 17);
    for (int i = 0; i < n; ++i) {
        h = (h ^ (unsigned)i) * 16777619u;
        x[(long long)i * st] = 0.5 + (double)(h % 1000003u) / 1000003.0;
    }
    for (int rep = 0; rep < 3; ++rep) {
        tri_solve(D.d, D.e, n, lam, x, u0, u1, u2, st, pivmin);
        double s0 = 0.0, s1 = 0.0;
        for (int i = 0; i + 1 < n; i += 2) {
            s0 = fma(x[(long long)i * st], x[(long long)i * st], s0);
            s1 = fma(x[(long long)(i + 1) * st], x[(long long)(i + 1) * st], s1);
        }
        if (n & 1) s0 = fma(x[(long long)(n - 1) * st], x[(long long)(n - 1) * st], s0);
        const double inv = 1.0 / sqrt(s0 + s1);
        for (int i = 0; i < n; ++i) x[(long long)i * st] *= inv;
    }
    double *y = Y + ((long long)b * nmax + mu) * n;
    for (int i = 0; i < n; ++i) y[i] = x[(long long)i * st];
}

// Shifted solves of the OSV relaxation: X row mu = (Tri - omega_mu)^{-1} (-R row mu) for mu < n_k, zero otherwise.
__global__ void __launch_bounds__(64) k_tri_shift_solve(const TriDesc *__restrict__ descs,
                                                        const int *__restrict__ nkeep, const double *__restrict__ R,
                                                        double *__restrict__ X, double *__restrict__ work,
                                                        int nmax) {
    const int b = blockIdx.x;
    const TriDesc D = descs[b];
    const int n = D.n;
    const int mu = blockIdx.y * blockDim.x + threadIdx.x;
    if (mu >= nmax) return;
    const int nk = nkeep[b];
    double *xo = X + ((long long)b * nmax + mu) * n;
    if (mu >= nk) {
        for (int i = 0; i < n; ++i) xo[i] = 0.0;
        return;
    }
    const long long st = nmax;
    double *base = work + (long long)b * 4 * n * nmax;
    double *x = base + mu, *u0 = base + (long long)n * nmax + mu, *u1 = base + 2LL * n * nmax + mu,
           *u2 = base + 3LL * n * nmax + mu;
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i) tnorm = fmax(tnorm, fabs(D.d[i]) + fabs(D.e[i]) + (i ? fabs(D.e[i - 1]) : 0.0));
    const double pivmin = fmax(tnorm, 1e-300) * DBL_EPSILON * 1e-3;
    const double *r = R + ((long long)b * nmax + mu) * n;
    for (int i = 0; i < n; ++i) x[(long long)i * st] = -r[i];
    tri_solve(D.d, D.e, n, D.w[mu], x, u0, u1, u2, st, pivmin);
    for (int i = 0; i < n; ++i) xo[i] = x[(long long)i * st];
}

// ------------------------------------------------------------------------------ CGS2 helpers (per CTA)
__device__ __forceinline__ double warp_dot(const double *a, const double *b, int n) {
    double s0 = 0.0, s1 = 0.0;
    const int lane = threadIdx.x & 31;
    int i = lane;
    for (; i + 32 < n; i += 64) {
        s0 = fma(a[i], b[i], s0);
        s1 = fma(a[i + 32], b[i + 32], s1);
    }
    if (i < n) s0 = fma(a[i], b[i], s0);
    return warp_sum(s0 + s1);
}

// Orthonormalise rows 0..n_k-1 of Y (per matrix) in order with two Gram-Schmidt passes each.
__global__ void __launch_bounds__(kT) k_orthonormalise(const int *__restrict__ nkeep, double *__restrict__ Y, int n,
                                                       int nmax) {
    const int b = blockIdx.x;
    const int nk = nkeep[b];
    double *Yb = Y + (long long)b * nmax * n;
    __shared__ double coef[128];
    __shared__ double red[kT / 32];
    const int wid = threadIdx.x >> 5, nw = kT / 32, lane = threadIdx.x & 31;
    for (int mu = 0; mu < nk; ++mu) {
        double *y = Yb + (long long)mu * n;
        for (int pass = 0; pass < 2; ++pass) {
            for (int nu = wid; nu < mu; nu += nw) {
                const double c = warp_dot(y, Yb + (long long)nu * n, n);
                if (lane == 0) coef[nu] = c;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += kT) {
                double s = y[i];
                for (int nu = 0; nu < mu; ++nu) s -= coef[nu] * Yb[(long long)nu * n + i];
                y[i] = s;
            }
            __syncthreads();
        }
        double ss = 0.0;
        for (int i = threadIdx.x; i < n; i += kT) ss += y[i] * y[i];
        ss = block_sum(ss, red);
        const double inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
        for (int i = threadIdx.x; i < n; i += kT) y[i] *= inv;
        __syncthreads();
    }
}

// X rows mu < nx of each matrix -= projection onto rows 0..n_k-1 of Y (two passes; Y orthonormal).
__global__ void __launch_bounds__(kT) k_project_out(const int *__restrict__ nkeep, const double *__restrict__ Y,
                                                    double *__restrict__ X, int n, int nmax) {
    const int b = blockIdx.x;
    const int nk = nkeep[b];
    const double *Yb = Y + (long long)b * nmax * n;
    double *Xb = X + (long long)b * nmax * n;
    const int wid = threadIdx.x >> 5, nw = kT / 32, lane = threadIdx.x & 31;
    for (int pass = 0; pass < 2; ++pass) {
        for (int mu = wid; mu < nk; mu += nw) {
            double *x = Xb + (long long)mu * n;
            // coefficients against every kept y, then one update (classical Gram-Schmidt, repeated)
            double cbuf[4];
            for (int nu0 = 0; nu0 < nk; nu0 += 4) {
                const int cnt = min(4, nk - nu0);
                for (int t = 0; t < cnt; ++t) cbuf[t] = warp_dot(x, Yb + (long long)(nu0 + t) * n, n);
                __syncwarp();
                for (int i = lane; i < n; i += 32) {
                    double s = x[i];
                    for (int t = 0; t < cnt; ++t) s -= cbuf[t] * Yb[(long long)(nu0 + t) * n + i];
                    x[i] = s;
                }
                __syncwarp();
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------- 4. reflector products
// rows mu < nrow(b) of V (nmax x n per matrix): forward = 0 applies H = H_0 ... H_{n-3} (q = H y),
// forward = 1 applies H^T (y = H^T g).  Reflector k: row k of A, columns k+1..n-1, scalar tau[k].
__global__ void __launch_bounds__(kT) k_reflect(const TriDesc *__restrict__ descs, const int *__restrict__ nrow,
                                                double *__restrict__ V, int nmax, int forward) {
    const int b = blockIdx.x;
    const TriDesc D = descs[b];
    const int n = D.n;
    const int nr = nrow ? nrow[b] : nmax;
    extern __shared__ double v[];
    double *Vb = V + (long long)b * nmax * n;
    const int wid = threadIdx.x >> 5, nw = kT / 32, lane = threadIdx.x & 31;
    for (int s = 0; s + 2 < n; ++s) {
        const int k = forward ? s : n - 3 - s;
        const double beta = D.tau[k];
        if (beta == 0.0) continue;
        const int m = n - k - 1;
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += kT) v[i] = D.A[(long long)k * D.lda + k + 1 + i];
        __syncthreads();
        for (int mu = wid; mu < nr; mu += nw) {
            double *y = Vb + (long long)mu * n + k + 1;
            const double c = beta * warp_dot(y, v, m);
            for (int i = lane; i < m; i += 32) y[i] -= c * v[i];
        }
    }
}

// -------------------------------------------------------------------------------- small dense Jacobi
// Cyclic parallel Jacobi for symmetric matrices of order <= kJacMax held in shared memory (A and V, padded to
// even order).  Round-robin pairing: every round rotates n/2 disjoint planes at once.  Eigenvalues decreasing
// into w, eigenvectors as rows of Zt.  n_dev (optional) gives the order.
__global__ void __launch_bounds__(kT) k_jacobi_small(const EighDesc *__restrict__ descs, int *err) {
    const EighDesc D = descs[blockIdx.x];
    const int n = D.n_dev ? min(*D.n_dev, D.n) : D.n;
    if (n <= 0) return;
    const int ne = (n + 1) & ~1;       // even order (the extra index never couples)
    const int ld = ne + 1;
    extern __shared__ double sh[];
    double *A = sh, *V = sh + (long long)ne * ld;
    double *cs = V + (long long)ne * ld, *sn = cs + ne / 2;
    int *pp = reinterpret_cast<int *>(sn + ne / 2), *qq = pp + ne / 2, *rank = qq + ne / 2;
    __shared__ double red[kT / 32];
    __shared__ int s_done;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < ne * ne; idx += kT) {
        const int r = idx / ne, c = idx % ne;
        A[r * ld + c] = (r < n && c < n) ? D.A[(long long)r * D.lda + c] : 0.0;
        V[r * ld + c] = r == c ? 1.0 : 0.0;
    }
    __syncthreads();
    double fro = 0.0;
    for (int idx = tid; idx < ne * ne; idx += kT) {
        const double a = A[(idx / ne) * ld + idx % ne];
        fro += a * a;
    }
    fro = block_sum(fro, red);
    const int half = ne / 2;
    bool conv = false;
    for (int sweep = 0; sweep < 40 && !conv; ++sweep) {
        for (int round = 0; round < ne - 1; ++round) {
            // round-robin: index 0 fixed, others rotate
            for (int t = tid; t < half; t += kT) {
                int a = t == 0 ? 0 : 1 + (t - 1 + round) % (ne - 1);
                int bb = 1 + (ne - 2 - t + round) % (ne - 1);
                if (t == 0) bb = 1 + (ne - 2 + round) % (ne - 1);
                const int p = min(a, bb), q = max(a, bb);
                pp[t] = p;
                qq[t] = q;
                const double apq = A[p * ld + q];
                double c = 1.0, s = 0.0;
                if (apq != 0.0 && fabs(apq) > 1e-300) {
                    const double th = (A[q * ld + q] - A[p * ld + p]) / (2.0 * apq);
                    const double tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                    c = rsqrt(tt * tt + 1.0);
                    s = tt * c;
                }
                cs[t] = c;
                sn[t] = s;
            }
            __syncthreads();
            // rows: B = J^T A
            for (int idx = tid; idx < half * ne; idx += kT) {
                const int t = idx / ne, k = idx % ne;
                const int p = pp[t], q = qq[t];
                const double c = cs[t], s = sn[t];
                const double ap = A[p * ld + k], aq = A[q * ld + k];
                A[p * ld + k] = c * ap - s * aq;
                A[q * ld + k] = s * ap + c * aq;
            }
            __syncthreads();
            // columns: A' = B J, and V' = V J
            for (int idx = tid; idx < half * ne; idx += kT) {
                const int t = idx / ne, k = idx % ne;
                const int p = pp[t], q = qq[t];
                const double c = cs[t], s = sn[t];
                const double ap = A[k * ld + p], aq = A[k * ld + q];
                A[k * ld + p] = c * ap - s * aq;
                A[k * ld + q] = s * ap + c * aq;
                const double vp = V[k * ld + p], vq = V[k * ld + q];
                V[k * ld + p] = c * vp - s * vq;
                V[k * ld + q] = s * vp + c * vq;
            }
            __syncthreads();
        }
        double off = 0.0;
        for (int idx = tid; idx < ne * ne; idx += kT) {
            const int r = idx / ne, c = idx % ne;
            if (r != c) off += A[r * ld + c] * A[r * ld + c];
        }
        off = block_sum(off, red);
        if (tid == 0) s_done = off <= 1e-30 * fro || off == 0.0;
        __syncthreads();
        conv = s_done;
    }
    if (!conv && tid == 0) atomicExch(err, kDevEighNoConv);
    for (int i = tid; i < n; i += kT) {
        const double di = A[i * ld + i];
        int rk = 0;
        for (int j = 0; j < n; ++j) {
            const double dj = A[j * ld + j];
            rk += (dj > di) || (dj == di && j < i);
        }
        rank[i] = rk;
    }
    __syncthreads();
    for (int i = tid; i < n; i += kT) D.w[rank[i]] = A[i * ld + i];
    for (int idx = tid; idx < n * n; idx += kT) {
        const int c = idx / n, r = idx % n;    // eigenvector c, component r
        D.Zt[(long long)rank[c] * D.ldz + r] = V[r * ld + c];
    }
}

}  // namespace

size_t jacobi_smem_bytes(int n) {
    const int ne = (n + 1) & ~1;
    return (size_t)2 * ne * (ne + 1) * sizeof(double) + (size_t)ne * sizeof(double) + (size_t)3 * (ne / 2 + 1) * sizeof(int) +
           (size_t)ne * sizeof(int) + 64;
}

cudaError_t osv_tridiag(const TriDesc *d, int batch, int n, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    const size_t sh = 2 * (size_t)n * sizeof(double);
    cudaError_t e;
    if (sh > 48 * 1024 && (e = cudaFuncSetAttribute(k_tridiag_osv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh)) != cudaSuccess)
        return e;
    count_launch();
    k_tridiag_osv<<<batch, kT, sh, s>>>(d);
    return cudaGetLastError();
}

cudaError_t osv_tri_eigvals(const TriDesc *d, int batch, int n, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    const size_t sh = 2 * (size_t)n * sizeof(double);
    cudaError_t e;
    if (sh > 48 * 1024 && (e = cudaFuncSetAttribute(k_tri_bisect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh)) != cudaSuccess)
        return e;
    const int gy = (n + kT - 1) / kT;
    count_launch();
    k_tri_bisect<<<dim3(batch, gy), kT, sh, s>>>(d);
    return cudaGetLastError();
}

cudaError_t osv_tri_kept_vectors(const TriDesc *d, int batch, int n, int nmax, const int *nkeep, double *Y,
                                 double *work, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    count_launch();
    k_tri_invit<<<dim3(batch, (nmax + 63) / 64), 64, 0, s>>>(d, nkeep, Y, work, nmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (nmax > 128) return cudaErrorInvalidValue;
    count_launch();
    k_orthonormalise<<<batch, kT, 0, s>>>(nkeep, Y, n, nmax);
    return cudaGetLastError();
}

cudaError_t osv_reflect(const TriDesc *d, int batch, int n, int nmax, const int *nrow, double *V, int forward,
                        cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    const size_t sh = (size_t)n * sizeof(double);
    cudaError_t e;
    if (sh > 48 * 1024 && (e = cudaFuncSetAttribute(k_reflect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh)) != cudaSuccess)
        return e;
    count_launch();
    k_reflect<<<batch, kT, sh, s>>>(d, nrow, V, nmax, forward);
    return cudaGetLastError();
}

cudaError_t osv_project_out(const int *nkeep, const double *Y, double *X, int batch, int n, int nmax, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    count_launch();
    k_project_out<<<batch, kT, 0, s>>>(nkeep, Y, X, n, nmax);
    return cudaGetLastError();
}

cudaError_t osv_tri_shift_solve(const TriDesc *d, int batch, int n, int nmax, const int *nkeep, const double *R,
                                double *X, double *work, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    count_launch();
    k_tri_shift_solve<<<dim3(batch, (nmax + 63) / 64), 64, 0, s>>>(d, nkeep, R, X, work, nmax);
    return cudaGetLastError();
}

cudaError_t eigh_small_jacobi(const EighDesc *d, int batch, int n_max, int *err, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    const size_t sh = jacobi_smem_bytes(n_max);
    cudaError_t e;
    if (sh > 48 * 1024 && (e = cudaFuncSetAttribute(k_jacobi_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh)) != cudaSuccess)
        return e;
    count_launch();
    k_jacobi_small<<<batch, kT, sh, s>>>(d, err);
    return cudaGetLastError();
}

}  // namespace osv
