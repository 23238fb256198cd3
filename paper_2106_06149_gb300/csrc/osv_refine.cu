// Mixed-precision route to the kept OSVs of Eq. 6 and to the relaxation solves of Eq. 8.
//
// On GB300 an FP32 multiply-add issues 64x faster than an FP64 one, so the O(n^3) Householder reduction runs in
// FP32 and only O(n^2 n_max) work stays in FP64:
//   1. FP32: T = H Tri H^T, the n_max largest eigenvalues of Tri, their vectors Y (tridiagonal basis) and the
//      starting vectors Q0 = H Y (cast to FP64).
//   2. FP64 refinement, kOsvRefineSteps times, then once more without the correction:
//        W = Q T;  [G; H] = [Q; W] Q^T;  Rayleigh-Ritz: L L^T = G, L^{-1} H L^{-T} = U Lambda U^T (Jacobi),
//        C^T = U^T L^{-1};  [Q; W] <- C^T [Q; W];  R = W - Lambda Q;
//        Q <- Q + M(Lambda) R,  M(lambda) = H P'_Y (lambda - Tri)^{-1} P'_Y H^T  (FP32),
//      where P'_Y removes the FP32 kept vectors: M approximates (lambda - T)^{-1} on the discarded space with a
//      relative error ~ eps_FP32 |T| / gap, so each correction contracts the eigenvector error by that factor.
//   3. n_k from the refined Ritz values (Eq. 6 selection), rows >= n_k of Q zeroed.
// The relaxation (Eq. 8) solves (omega_mu - T) a_mu = g_mu on the discarded space: a = M g, then FP64
// residual corrections a += M (g - P_perp (omega a - a T)).
#include "kernels.cuh"
#include "jacobi.cuh"
#include "osv_refine.h"

namespace osv {

namespace {

constexpr int kT = 256;

inline int grid_for(long long n) { return (int)std::min<long long>((n + kT - 1) / kT, 152LL * 16); }

// QW[b] rows 0..nm (stride 2 nm nv per LMO) <- (double) X[b] (nm nv per LMO)
__global__ void k_pack_q(const float *__restrict__ X, double *__restrict__ QW, long long per, long long tot) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / per, o = i - b * per;
        QW[b * 2 * per + o] = (double)X[i];
    }
}

// X[b][mu][i] = (float)(W[b][mu][i] - lam[b][mu] Q[b][mu][i]), Q and W the two halves of QW[b]
__global__ void k_ritz_residual(const double *__restrict__ QW, const double *__restrict__ lam, float *__restrict__ X,
                                int nm, int nv, long long tot) {
    const long long per = (long long)nm * nv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / per, o = i - b * per;
        const int mu = (int)(o / nv);
        const double *q = QW + b * 2 * per;
        X[i] = (float)(q[per + o] - lam[b * nm + mu] * q[o]);
    }
}

// QW[b] rows 0..nm += (double) Z[b]
__global__ void k_add_q(double *__restrict__ QW, const float *__restrict__ Z, long long per, long long tot) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / per, o = i - b * per;
        QW[b * 2 * per + o] += (double)Z[i];
    }
}

__global__ void k_cast_f32(const double *__restrict__ in, float *__restrict__ out, long long tot) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// a = (double) Z (assign) or a += (double) Z
__global__ void k_acc_f64(double *__restrict__ a, const float *__restrict__ Z, long long tot, int assign) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x)
        a[i] = assign ? (double)Z[i] : a[i] + (double)Z[i];
}

// RS = g - (lam_mu a - a T) on rows mu < nosv, zero rows otherwise
__global__ void k_relax_resid(const double *__restrict__ g, const double *__restrict__ a,
                              const double *__restrict__ at, const double *__restrict__ lam,
                              const int *__restrict__ nosv, double *__restrict__ rs, int nm, int nv, long long tot) {
    const long long per = (long long)nm * nv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / per;
        const int mu = (int)((i - b * per) / nv);
        rs[i] = mu < nosv[b] ? g[i] - (lam[b * nm + mu] * a[i] - at[i]) : 0.0;
    }
}

// Rayleigh-Ritz of one LMO's block (CTA per LMO): from G = Q Q^T and H = W Q^T (GH rows 0..nm and nm..2nm)
// the rotation Ct = U^T L^{-1} (rows: new vectors, decreasing Ritz values) and the Ritz values lam.
__global__ void __launch_bounds__(kT) k_rr(const double *__restrict__ GH, double *__restrict__ Ct,
                                           double *__restrict__ lam, int nm, int *err) {
    const int b = blockIdx.x;
    const int ne = (nm + 1) & ~1, ld = ne + 1;
    extern __shared__ double sh[];
    double *G = sh, *Li = G + ne * ld, *H = Li + ne * ld, *Tm = H + ne * ld, *V = Tm + ne * ld;
    double *cs = V + ne * ld, *sn = cs + ne / 2;
    int *pp = reinterpret_cast<int *>(sn + ne / 2), *qq = pp + ne / 2, *rank = qq + ne / 2;
    __shared__ double red[kT / 32];
    __shared__ int s_flag;
    const int tid = threadIdx.x;
    const double *g = GH + (long long)b * 2 * nm * nm, *h = g + (long long)nm * nm;
    for (int idx = tid; idx < ne * ne; idx += kT) {
        const int r = idx / ne, c = idx % ne;
        const bool in = r < nm && c < nm;
        G[r * ld + c] = in ? 0.5 * (g[r * nm + c] + g[c * nm + r]) : (r == c ? 1.0 : 0.0);
        H[r * ld + c] = in ? 0.5 * (h[r * nm + c] + h[c * nm + r]) : 0.0;
        V[r * ld + c] = r == c ? 1.0 : 0.0;
    }
    __syncthreads();
    // Cholesky G = L L^T in place (lower)
    for (int j = 0; j < ne; ++j) {
        if (tid == 0) {
            double s = G[j * ld + j];
            for (int k = 0; k < j; ++k) s -= G[j * ld + k] * G[j * ld + k];
            if (!(s > 0.0)) {
                raise_err(err, kDevNonFinite);
                s = 1.0;
            }
            G[j * ld + j] = sqrt(s);
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < ne; i += kT) {
            double s = G[i * ld + j];
            for (int k = 0; k < j; ++k) s -= G[i * ld + k] * G[j * ld + k];
            G[i * ld + j] = s / G[j * ld + j];
        }
        __syncthreads();
    }
    // Li = L^{-1} (lower), column c by thread c
    for (int c = tid; c < ne; c += kT) {
        for (int r = 0; r < ne; ++r) {
            if (r < c) {
                Li[r * ld + c] = 0.0;
                continue;
            }
            double s = r == c ? 1.0 : 0.0;
            for (int k = c; k < r; ++k) s -= G[r * ld + k] * Li[k * ld + c];
            Li[r * ld + c] = s / G[r * ld + r];
        }
    }
    __syncthreads();
    // H' = Li H Li^T
    for (int idx = tid; idx < ne * ne; idx += kT) {
        const int r = idx / ne, c = idx % ne;
        double s = 0.0;
        for (int k = 0; k <= r; ++k) s += Li[r * ld + k] * H[k * ld + c];
        Tm[r * ld + c] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < ne * ne; idx += kT) {
        const int r = idx / ne, c = idx % ne;
        double s = 0.0;
        for (int k = 0; k <= c; ++k) s += Tm[r * ld + k] * Li[c * ld + k];
        H[r * ld + c] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < ne * ne; idx += kT) {
        const int r = idx / ne, c = idx % ne;
        if (r < c) {
            const double m = 0.5 * (H[r * ld + c] + H[c * ld + r]);
            H[r * ld + c] = m;
            H[c * ld + r] = m;
        }
    }
    __syncthreads();
    // Jacobi on H' in double-float (FP32 pipe; an FP64 rotation sweep is bound by the FP64 rate): H' into the Tm
    // space, the rotations into the V space, both as (hi, lo) pairs
    float2 *Hd = reinterpret_cast<float2 *>(Tm), *Vd = reinterpret_cast<float2 *>(V);
    float2 *csd = reinterpret_cast<float2 *>(cs), *snd = reinterpret_cast<float2 *>(sn);
    for (int idx = tid; idx < ne * ne; idx += kT) {
        const int r = idx / ne, c = idx % ne;
        Hd[r * ld + c] = split_df(H[r * ld + c]);
        Vd[r * ld + c] = make_float2(r == c ? 1.f : 0.f, 0.f);
    }
    __syncthreads();
    const bool conv = jacobi_sweeps_df(Hd, Vd, ne, ld, csd, snd, pp, qq, red, &s_flag, 30, 1e-28);
    if (!conv && tid == 0) raise_err(err, kDevEighNoConv);
    for (int i = tid; i < ne; i += kT) H[i * ld + i] = df_val(Hd[i * ld + i].x, Hd[i * ld + i].y);
    __syncthreads();
    diag_rank<double>(H, nm, ld, rank);
    for (int i = tid; i < nm; i += kT) lam[(long long)b * nm + rank[i]] = H[i * ld + i];
    double *ct = Ct + (long long)b * nm * nm;
    for (int idx = tid; idx < nm * nm; idx += kT) {
        const int c = idx / nm, k = idx % nm;   // new vector c, old vector k
        double s = 0.0;
        for (int j = k; j < ne; ++j) s += df_val(Vd[j * ld + c].x, Vd[j * ld + c].y) * Li[j * ld + k];
        ct[(long long)rank[c] * nm + k] = s;
    }
}

size_t rr_smem_bytes(int nm) {
    const int ne = (nm + 1) & ~1, ld = ne + 1;
    return (size_t)5 * ne * ld * sizeof(double) + (size_t)ne * sizeof(double) + (size_t)3 * (ne / 2 + 1) * sizeof(int) +
           (size_t)ne * sizeof(int) + 64;
}

// n_k from the refined Ritz values (Eq. 6: omega > l_osv, capped at nm, or fixed; at least one), omega rows,
// and rows >= n_k of Q zeroed (CTA per LMO).
__global__ void __launch_bounds__(kT) k_osv_finish(const double *__restrict__ lam, double *__restrict__ omega,
                                                   int *__restrict__ nosv, double *__restrict__ Q, int nm, int nv,
                                                   double l_osv, int n_fixed) {
    const int b = blockIdx.x;
    __shared__ int s_nk;
    const double *l = lam + (long long)b * nm;
    if (threadIdx.x == 0) {
        int nk;
        if (n_fixed > 0) {
            nk = min(n_fixed, nm);
        } else {
            nk = 0;
            while (nk < nm && l[nk] > l_osv) ++nk;
        }
        nk = max(nk, 1);
        s_nk = nk;
        nosv[b] = nk;
    }
    for (int mu = threadIdx.x; mu < nm; mu += kT) omega[(long long)b * nv + mu] = l[mu];
    __syncthreads();
    double *q = Q + (long long)b * nm * nv;
    for (long long i = (long long)s_nk * nv + threadIdx.x; i < (long long)nm * nv; i += kT) q[i] = 0.0;
}

// X (FP32 rows, virtual basis) -> Z = M(shift) X: H^T, remove the FP32 kept vectors, (shift - Tri)^{-1},
// remove them again, H.  Rows >= nkeep[b] of Z are zero.
// H or H^T on FP32 rows: blocked (compact WY) when the plan holds the T factors, else reflector by reflector
cudaError_t reflect32(const OsvRefine &r, int n, int nv, int nm, const int *nrow, float *V, int forward,
                      cudaStream_t s) {
    if (r.Twy) return osv_reflect_wy(r.tri_d, r.Twy, n, nv, nm, nrow, V, forward, s);
    return osv_reflect<float>(r.tri_d, n, nv, nm, nrow, V, forward, s);
}

template <class R>
cudaError_t project(const int *nkeep, const R *Y, R *X, int n, int nv, int nm, cudaStream_t s) {
    if (osv_project_rows_fits(nv, nm)) return osv_project_rows<R>(nkeep, Y, X, n, nv, nm, s);
    return osv_project_out<R>(nkeep, Y, X, n, nv, nm, s);
}

cudaError_t apply_precond(const OsvRefine &r, int n, int nv, int nm, const int *nkeep, const double *shift,
                          cudaStream_t s) {
    cudaError_t e;
    if ((e = reflect32(r, n, nv, nm, nkeep, r.X32, 1, s)) != cudaSuccess) return e;
    if ((e = project<float>(nkeep, r.Y32, r.X32, n, nv, nm, s)) != cudaSuccess) return e;
    if ((e = osv_tri_shift_solve<float>(r.tri_d, n, nv, nm, nkeep, r.X32, r.Z32, r.work32, shift, nm, s)) != cudaSuccess)
        return e;
    if ((e = project<float>(nkeep, r.Y32, r.Z32, n, nv, nm, s)) != cudaSuccess) return e;
    return reflect32(r, n, nv, nm, nkeep, r.Z32, 0, s);
}

cudaError_t rayleigh_ritz(const OsvRefine &r, int x, int n, int nm, int *err, cudaStream_t s) {
    cudaError_t e;
    if ((e = gemm_batch_run_df(r.gb_w[x], s)) != cudaSuccess) return e;
    if ((e = gemm_batch_run_df(r.gb_gh[x], s)) != cudaSuccess) return e;
    const size_t sh = rr_smem_bytes(nm);
    if (sh > 48 * 1024 && (e = cudaFuncSetAttribute(k_rr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh)) != cudaSuccess)
        return e;
    count_launch();
    k_rr<<<n, kT, sh, s>>>(r.GH, r.Ct, r.lam, nm, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t osv_mixed_eigh(const OsvRefine &r, int n, int nv, int nm, double *Q, double *omega, int *nosv,
                           double l_osv, int n_fixed, int *err, cudaStream_t s, int steps) {
    if (n <= 0) return cudaSuccess;
    if (nm > kRefineMaxN) return cudaErrorInvalidValue;
    cudaError_t e;
#define CK(x) \
    do { \
        if ((e = (x)) != cudaSuccess) return e; \
    } while (0)
    const long long per = (long long)nm * nv, tot = per * n;
    const int grid = grid_for(tot);
    CK(osv_tridiag<float>(r.tri_d, n, nv, s, r.tri_variant));
    if (r.Twy) CK(osv_wy_prepare(r.tri_d, n, nv, r.Twy, s));
    CK(osv_tri_eigvals<float>(r.tri_d, n, nv, nm, s));
    CK(osv_tri_kept_vectors<float>(r.tri_d, n, nv, nm, r.nm_all, r.Y32, r.work32, s));
    CK(cudaMemcpyAsync(r.X32, r.Y32, tot * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CK(reflect32(r, n, nv, nm, r.nm_all, r.X32, 0, s));
    count_launch();
    k_pack_q<<<grid, kT, 0, s>>>(r.X32, r.QW[0], per, tot);
    CK(cudaGetLastError());
    for (int it = 0; it < steps; ++it) {
        const int x = it & 1, y = x ^ 1;
        CK(rayleigh_ritz(r, x, n, nm, err, s));
        CK(gemm_batch_run_df(r.gb_rot[x], s));
        count_launch();
        k_ritz_residual<<<grid, kT, 0, s>>>(r.QW[y], r.lam, r.X32, nm, nv, tot);
        CK(cudaGetLastError());
        CK(apply_precond(r, n, nv, nm, r.nm_all, r.lam, s));
        count_launch();
        k_add_q<<<grid, kT, 0, s>>>(r.QW[y], r.Z32, per, tot);
        CK(cudaGetLastError());
    }
    const int x = steps & 1;
    CK(rayleigh_ritz(r, x, n, nm, err, s));
    CK(gemm_batch_run_df(r.gb_fin[x], s));
    count_launch();
    k_osv_finish<<<n, kT, 0, s>>>(r.lam, omega, nosv, Q, nm, nv, l_osv, n_fixed);
    CK(cudaGetLastError());
#undef CK
    return cudaSuccess;
}

cudaError_t osv_mixed_relax(const OsvRefine &r, const GemmBatch &gb_at, int n, int nv, int nm, const double *Q,
                            const int *nosv, const double *g, double *a, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e;
#define CK(x) \
    do { \
        if ((e = (x)) != cudaSuccess) return e; \
    } while (0)
    const long long tot = (long long)nm * nv * n;
    const int grid = grid_for(tot);
    count_launch();
    k_cast_f32<<<grid, kT, 0, s>>>(g, r.X32, tot);
    CK(cudaGetLastError());
    CK(apply_precond(r, n, nv, nm, nosv, r.lam, s));
    count_launch();
    k_acc_f64<<<grid, kT, 0, s>>>(a, r.Z32, tot, 1);
    CK(cudaGetLastError());
    for (int it = 0; it < kRelaxRefineSteps; ++it) {
        CK(gemm_batch_run_df(gb_at, s));
        count_launch();
        k_relax_resid<<<grid, kT, 0, s>>>(g, a, r.AT, r.lam, nosv, r.RS, nm, nv, tot);
        CK(cudaGetLastError());
        CK(project<double>(nosv, Q, r.RS, n, nv, nm, s));
        count_launch();
        k_cast_f32<<<grid, kT, 0, s>>>(r.RS, r.X32, tot);
        CK(cudaGetLastError());
        CK(apply_precond(r, n, nv, nm, nosv, r.lam, s));
        count_launch();
        k_acc_f64<<<grid, kT, 0, s>>>(a, r.Z32, tot, 0);
        CK(cudaGetLastError());
    }
    CK(project<double>(nosv, Q, a, n, nv, nm, s));
#undef CK
    return cudaSuccess;
}

}  // namespace osv
