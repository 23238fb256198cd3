// Cyclic parallel Jacobi sweeps on a small symmetric matrix held in shared memory (a device function shared by
// the batched small eigensolver, the Rayleigh-Ritz step of the OSV refinement and the mixed pair bases).
#pragma once
#include "common.cuh"

namespace osv {

// One round's rotations J (planes (pp[t], qq[t]), cosines cs, sines sn) applied as A <- J^T A J by 2 x 2 blocks
// (rows p_t, q_t x columns p_u, q_u: the row rotation, then the column rotation, as two separate passes would)
// and V <- V J; each element is read and written once, by one thread.  Thread work is stepped without divisions.
template <class R>
__device__ __forceinline__ void jacobi_apply_round(R *A, R *V, int ne, int ld, int half, const R *cs, const R *sn,
                                                   const int *pp, const int *qq) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int dt = nt / half, du = nt - dt * half;
    {
        int t = tid / half, u = tid - (tid / half) * half;
        while (t < half) {
            const int p = pp[t], q = qq[t], p2 = pp[u], q2 = qq[u];
            const R ct = cs[t], st = sn[t], cu = cs[u], su = sn[u];
            R *rp = A + p * ld, *rq = A + q * ld;
            const R a = rp[p2], b = rp[q2], c = rq[p2], d = rq[q2];
            const R ra = ct * a - st * c, rc = st * a + ct * c;   // rows
            const R rb = ct * b - st * d, rd = st * b + ct * d;
            rp[p2] = cu * ra - su * rb;                             // columns
            rp[q2] = su * ra + cu * rb;
            rq[p2] = cu * rc - su * rd;
            rq[q2] = su * rc + cu * rd;
            u += du;
            t += dt;
            if (u >= half) {
                u -= half;
                ++t;
            }
        }
    }
    {
        const int dv = nt / ne, dk = nt - dv * ne;   // V: consecutive threads take consecutive rows k
        int u = tid / ne, k = tid - (tid / ne) * ne;
        while (u < half) {
            const int p2 = pp[u], q2 = qq[u];
            const R cu = cs[u], su = sn[u];
            R *vk = V + k * ld;
            const R vp = vk[p2], vq = vk[q2];
            vk[p2] = cu * vp - su * vq;
            vk[q2] = su * vp + cu * vq;
            k += dk;
            u += dv;
            if (k >= ne) {
                k -= ne;
                ++u;
            }
        }
    }
}

// Round-robin pairing: every round rotates ne/2 disjoint planes (p, q) at once, ne - 1 rounds per sweep.
// A: ne x ne symmetric (leading dimension ld, ne even; padding rows/columns must be zero), rotated in place;
// V <- V J accumulates the rotations (start from the identity, or from a basis to be updated).  Sweeps stop
// when the off-diagonal sum of squares is <= tol2 * the Frobenius sum of squares of A at entry, or after
// max_sweeps.  Scratch: cs, sn (ne/2 of R), pp, qq (ne/2 ints), red (blockDim/32 doubles), flag (one int).
// Returns whether the tolerance was met.  Every thread of the block must call it.
template <class R>
__device__ bool jacobi_sweeps(R *A, R *V, int ne, int ld, R *cs, R *sn, int *pp, int *qq, double *red, int *flag,
                              int max_sweeps, double tol2) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const R tiny = sizeof(R) == 8 ? (R)1e-300 : (R)1e-37;
    double fro = 0.0;
    for (int idx = tid; idx < ne * ne; idx += nt) {
        const double a = A[(idx / ne) * ld + idx % ne];
        fro += a * a;
    }
    fro = block_sum(fro, red);
    const int half = ne / 2;
    bool conv = false;
    for (int sweep = 0;; ++sweep) {
        double off = 0.0;
        for (int idx = tid; idx < ne * ne; idx += nt) {
            const int r = idx / ne, c = idx % ne;
            if (r != c) off += (double)A[r * ld + c] * (double)A[r * ld + c];
        }
        off = block_sum(off, red);
        if (tid == 0) *flag = off <= tol2 * fro || off == 0.0;
        __syncthreads();
        conv = *flag;
        __syncthreads();
        if (conv || sweep == max_sweeps) break;
        for (int round = 0; round < ne - 1; ++round) {
            for (int t = tid; t < half; t += nt) {
                int a = t == 0 ? 0 : 1 + (t - 1 + round) % (ne - 1);
                int bb = 1 + (ne - 2 - t + round) % (ne - 1);
                if (t == 0) bb = 1 + (ne - 2 + round) % (ne - 1);
                const int p = min(a, bb), q = max(a, bb);
                pp[t] = p;
                qq[t] = q;
                const R apq = A[p * ld + q];
                R c = 1, s = 0;
                if (apq != (R)0 && fabs(apq) > tiny) {
                    const R th = (A[q * ld + q] - A[p * ld + p]) / (2 * apq);
                    const R tt = (th >= (R)0 ? (R)1 : (R)-1) / (fabs(th) + sqrt(th * th + (R)1));
                    c = rsqrt(tt * tt + (R)1);
                    s = tt * c;
                }
                cs[t] = c;
                sn[t] = s;
            }
            __syncthreads();
            jacobi_apply_round(A, V, ne, ld, half, cs, sn, pp, qq);
            __syncthreads();
        }
    }
    return conv;
}

// ------------------------------------------------------------------ double-float sweeps (FP32-pipe FP64)
// (hi, lo) renormalised so that |lo| <= ulp(hi) / 2
__device__ __forceinline__ float2 df_renorm(float h, float l) {
    const float s = __fadd_rn(h, l);
    return make_float2(s, __fsub_rn(l, __fsub_rn(s, h)));
}

// (x, y) <- (c x - s y, s x + c y) in double-float
__device__ __forceinline__ void df_rot(float2 &x, float2 &y, const float2 c, const float2 sn) {
    float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
    const float2 ms = make_float2(-sn.x, -sn.y);
    df_fma(h1, l1, c, x);
    df_fma(h1, l1, ms, y);
    df_fma(h2, l2, sn, x);
    df_fma(h2, l2, c, y);
    x = df_renorm(h1, l1);
    y = df_renorm(h2, l2);
}

// The same rotation for a small angle (|s| <= 2^-12, so c = 1 - d with d <= 2^-25):
//   x' = x - s y - d x,  y' = y + s x - d y.
// The leading products s_h y_h and s_h x_h are split exactly (FMA), the terms s_h y_l + s_l y_h + d x_h (all below
// 2^-24 of the result) are summed in FP32, and one two-sum per output merges them: ~2^-48 relative like df_rot,
// at about 60% of its FP32 instructions.  d = (1 - c_h) - c_l (1 - c_h is exact for c_h in [0.5, 1]).
__device__ __forceinline__ void df_rot_small(float2 &x, float2 &y, const float2 c, const float2 sn) {
    const float d = __fsub_rn(__fsub_rn(1.f, c.x), c.y);
    const float p1 = __fmul_rn(sn.x, y.x), e1 = __fmaf_rn(sn.x, y.x, -p1);
    const float q1 = __fmaf_rn(sn.x, y.y, __fmaf_rn(sn.y, y.x, __fmul_rn(d, x.x)));
    const float p2 = __fmul_rn(sn.x, x.x), e2 = __fmaf_rn(sn.x, x.x, -p2);
    const float q2 = __fmaf_rn(sn.x, x.y, __fmaf_rn(sn.y, x.x, -__fmul_rn(d, y.x)));
    float h1 = x.x, l1 = __fsub_rn(x.y, __fadd_rn(e1, q1));
    float h2 = y.x, l2 = __fadd_rn(y.y, __fadd_rn(e2, q2));
    df_add(h1, l1, -p1);
    df_add(h2, l2, p2);
    x = df_renorm(h1, l1);
    y = df_renorm(h2, l2);
}

__device__ __forceinline__ void df_rot_sel(float2 &x, float2 &y, const float2 c, const float2 sn) {
    if (fabsf(sn.x) <= 2.44140625e-4f) df_rot_small(x, y, c, sn);
    else df_rot(x, y, c, sn);
}

// Cyclic round-robin Jacobi sweeps in double-float (A, V: ne x ne pairs in shared memory; same pairing as
// jacobi_sweeps, the rotation angle from FP64 values of the three entries).  Stops when off <= tol2 fro, or at the
// arithmetic's floor: double-float rotations leave about 2^-48 |A| of rounding in every off-diagonal entry, a sum of
// squares near ne 2^-96 fro (5e-28 fro at ne = 41), which can sit above tol2 fro; once off <= 1e-26 fro and a sweep
// no longer halves it, further sweeps change nothing and the matrix counts as diagonal.
__device__ inline bool jacobi_sweeps_df(float2 *A, float2 *V, int ne, int ld, float2 *cs, float2 *sn, int *pp, int *qq,
                                 double *red, int *flag, int max_sweeps, double tol2) {
    const int tid = threadIdx.x, nt = blockDim.x;
    double fro = 0.0;
    for (int idx = tid; idx < ne * ne; idx += nt) {
        const double a = A[(idx / ne) * ld + idx % ne].x;
        fro += a * a;
    }
    fro = block_sum(fro, red);
    const int half = ne / 2;
    bool conv = false;
    double prev = -1.0;
    for (int sweep = 0;; ++sweep) {
        double off = 0.0;
        for (int idx = tid; idx < ne * ne; idx += nt) {
            const int r = idx / ne, c = idx % ne;
            if (r != c) {
                const double a = A[r * ld + c].x;
                off += a * a;
            }
        }
        off = block_sum(off, red);
        if (tid == 0) *flag = off <= tol2 * fro || off == 0.0 || (prev >= 0.0 && off <= 1e-26 * fro && off > 0.5 * prev);
        prev = off;
        __syncthreads();
        conv = *flag;
        __syncthreads();
        if (conv || sweep == max_sweeps) break;
        for (int round = 0; round < ne - 1; ++round) {
            for (int t = tid; t < half; t += nt) {
                int a = t == 0 ? 0 : 1 + (t - 1 + round) % (ne - 1);
                int bb = 1 + (ne - 2 - t + round) % (ne - 1);
                if (t == 0) bb = 1 + (ne - 2 + round) % (ne - 1);
                const int p = min(a, bb), q = max(a, bb);
                pp[t] = p;
                qq[t] = q;
                const float2 apq2 = A[p * ld + q];
                double c = 1.0, s = 0.0;
                if (apq2.x != 0.f) {
                    // the angle in FP32 (a rotation within ~1e-7 of the annihilating one still leaves only ~1e-7 of
                    // a_pq, and the sweeps converge as fast); c and s from it in FP64 so that c^2 + s^2 = 1 to
                    // FP64 rounding and the rotation stays orthogonal.  An FP64 division or square root is a
                    // ~500-cycle dependent chain on GB300; one rotation round would otherwise wait on four.
                    const float2 aq = A[q * ld + q], ap = A[p * ld + p];
                    const float diff = __fadd_rn(__fsub_rn(aq.x, ap.x), __fsub_rn(aq.y, ap.y));
                    const float th = diff / (2.f * apq2.x);
                    const float tt = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
                    c = rsqrt(fma((double)tt, (double)tt, 1.0));
                    s = (double)tt * c;
                }
                cs[t] = split_df(c);
                sn[t] = split_df(s);
            }
            __syncthreads();
            // A <- J^T A J by 2 x 2 blocks (row rotation, then column rotation), V <- V J; division-free stepping
            {
                const int dt = nt / half, du = nt - dt * half;
                int t = tid / half, u = tid - (tid / half) * half;
                while (t < half) {
                    const int p = pp[t], q = qq[t], p2 = pp[u], q2 = qq[u];
                    const float2 ct = cs[t], st = sn[t], cu = cs[u], su = sn[u];
                    float2 *rp = A + p * ld, *rq = A + q * ld;
                    float2 a = rp[p2], b = rp[q2], c = rq[p2], d = rq[q2];
                    df_rot_sel(a, c, ct, st);
                    df_rot_sel(b, d, ct, st);
                    df_rot_sel(a, b, cu, su);
                    df_rot_sel(c, d, cu, su);
                    rp[p2] = a;
                    rp[q2] = b;
                    rq[p2] = c;
                    rq[q2] = d;
                    u += du;
                    t += dt;
                    if (u >= half) {
                        u -= half;
                        ++t;
                    }
                }
                const int dv = nt / ne, dk = nt - dv * ne;
                int w = tid / ne, k = tid - (tid / ne) * ne;
                while (w < half) {
                    float2 *vk = V + k * ld;
                    df_rot_sel(vk[pp[w]], vk[qq[w]], cs[w], sn[w]);
                    k += dk;
                    w += dv;
                    if (k >= ne) {
                        k -= ne;
                        ++w;
                    }
                }
            }
            __syncthreads();
        }
    }
    return conv;
}

// rank[i] = position of diagonal entry i in decreasing order (ties by index), for i < n.
template <class R>
__device__ void diag_rank(const R *A, int n, int ld, int *rank) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const R di = A[i * ld + i];
        int rk = 0;
        for (int j = 0; j < n; ++j) {
            const R dj = A[j * ld + j];
            rk += (dj > di) || (dj == di && j < i);
        }
        rank[i] = rk;
    }
    __syncthreads();
}

}  // namespace osv
