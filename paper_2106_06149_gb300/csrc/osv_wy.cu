// Blocked reflector products and row projections of the mixed-precision OSV solves (Eq. 6 and Eq. 8).
//
// The FP32 preconditioner of the mixed route applies H^T, a projection, a tridiagonal solve, a projection and H
// to n_max rows per LMO.  Applied one reflector at a time, H costs n - 2 dependent dot-product / update rounds
// per row; here the reflectors are grouped in blocks of kNB and each block acts as one compact-WY factor
// B_j = H_k0 ... H_{k0+kNB-1} = I - V_j T_j V_j^T (T_j upper triangular), so a row sees (n - 2) / kNB
// block steps whose inner work is a small matrix product on data held in shared memory.  The projections
// x <- x - Y^T (Y x) (classical Gram-Schmidt, twice) likewise run as two small products per pass with Y streamed
// through shared memory; the FP64 variant computes in double-float (FP32 pipe, ~48-bit significands).
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "osv_refine.h"

namespace osv {

namespace {

constexpr int kT = 256;
constexpr int kNB = 32;       // reflectors per compact-WY block (one per lane)
constexpr int kPoRows = 8;    // rows of X per CTA of the projection (one warp each)
constexpr int kPoCW = 64;     // Y column chunk of the projection
constexpr int kPoMaxY = 64;   // projection onto at most 64 rows (two per lane)

// element copies global -> shared that stay in flight together (src_bytes = 0: zero fill, nothing read)
__device__ __forceinline__ void cp_async_zfill(void *dst, const void *src, int bytes, int src_bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__host__ __device__ __forceinline__ int wy_blocks(int n) { return n < 3 ? 0 : (n - 2 + kNB - 1) / kNB; }

// The reflectors of block j stream through shared memory in chunks of kCH columns (chunk rows padded to an odd
// stride, kCH + 1, so that lane i reading reflector i's column c hits bank (i + c) mod 32): the blocks of any order up
// to 4096 fit, not only those whose kNB x n reflector block fits at once.
constexpr int kCH = 256;
constexpr int kLdc = kCH + 1;

// reflector i of block j (k0 = j kNB, kb reflectors), columns [c0 + cbeg, c0 + cbeg + cw) relative to c0 = k0 + 1,
// into Vs (kNB x kLdc): row k0 + i of A from column k0 + 1 + i on, zeros before (and for i >= kb)
__device__ __forceinline__ void load_v_chunk(const TriDesc32 &D, int k0, int kb, int cbeg, int cw, float *Vs) {
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int c0 = k0 + 1;
    for (int i = wid; i < kNB; i += kT / 32) {
        const float *src = D.A + (long long)min(k0 + i, D.n - 1) * D.lda + c0 + cbeg;
        for (int c = lane; c < cw; c += 32)
            cp_async_zfill(Vs + i * kLdc + c, src + c, 4, (i < kb && cbeg + c >= i) ? 4 : 0);
    }
}

// T_j of every block j of every matrix (kNB x kNB row-major, zero outside the upper triangle of the block's kb
// reflectors).  With G = V^T V (accumulated over column chunks), the columns follow
// T[0:i, i] = -tau_i T[0:i, 0:i] G[0:i, i], T[i][i] = tau_i.
__global__ void __launch_bounds__(kT) k_wy_t(const TriDesc32 *__restrict__ descs, float *__restrict__ Tall, int J) {
    const int b = blockIdx.x, j = blockIdx.y;
    const TriDesc32 D = descs[b];
    const int n = D.n;
    float *T = Tall + ((long long)b * J + j) * kNB * kNB;
    const int tid = threadIdx.x;
    const int k0 = j * kNB;
    const int kb = j < wy_blocks(n) ? min(kNB, n - 2 - k0) : 0;
    if (kb <= 0) {
        for (int i = tid; i < kNB * kNB; i += kT) T[i] = 0.f;
        return;
    }
    const int m0 = n - k0 - 1;
    extern __shared__ __align__(16) float wsm[];
    float *Vs = wsm;                       // kNB x kLdc: one column chunk of the block's reflectors
    float *Gs = Vs + kNB * kLdc;           // kNB x (kNB + 1)
    float *Ts = Gs + kNB * (kNB + 1);      // kNB x (kNB + 1)
    for (int idx = tid; idx < kNB * (kNB + 1); idx += kT) Ts[idx] = 0.f;
    // G[l][i], l < i, one thread per (l, i), accumulated over the chunks (registers)
    constexpr int kPairs = kNB * kNB / kT;   // 4 pairs per thread
    float gacc[kPairs];
#pragma unroll
    for (int q = 0; q < kPairs; ++q) gacc[q] = 0.f;
    for (int cbeg = 0; cbeg < m0; cbeg += kCH) {
        const int cw = min(kCH, m0 - cbeg);
        __syncthreads();   // the previous chunk is no longer read
        load_v_chunk(D, k0, kb, cbeg, cw, Vs);
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPairs; ++q) {
            const int pidx = tid + q * kT, l = pidx / kNB, i = pidx % kNB;
            if (l < i && i < kb) {
                const float *vl = Vs + l * kLdc, *vi = Vs + i * kLdc;
                float s = 0.f;
                for (int c = 0; c < cw; ++c) s = fmaf(vl[c], vi[c], s);
                gacc[q] += s;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kPairs; ++q) {
        const int pidx = tid + q * kT, l = pidx / kNB, i = pidx % kNB;
        if (l < i && i < kb) Gs[l * (kNB + 1) + i] = gacc[q];
    }
    __syncthreads();
    for (int i = 0; i < kb; ++i) {
        const float tau = D.tau[k0 + i];
        if (tid < i) {
            float s = 0.f;
            for (int m = tid; m < i; ++m) s = fmaf(Ts[tid * (kNB + 1) + m], Gs[m * (kNB + 1) + i], s);
            Ts[tid * (kNB + 1) + i] = -tau * s;
        } else if (tid == i) {
            Ts[i * (kNB + 1) + i] = tau;
        }
        __syncthreads();
    }
    for (int idx = tid; idx < kNB * kNB; idx += kT) {
        const int i = idx / kNB, l = idx - i * kNB;
        T[idx] = Ts[i * (kNB + 1) + l];
    }
}

constexpr int kTR = 64;          // rows of V per CTA of the tiled product: every kept row of a matrix (n_max <= 64)
constexpr int kTCW = 64;         // column chunk
constexpr int kTLd = kTCW + 4;   // chunk row stride in floats: 16-byte rows; rows r and r + 1 four banks apart
constexpr int kTBuf = (kNB + kTR) * kTLd;   // one chunk buffer: the 32 reflector rows, then the 64 row chunks

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// rows mu < nrow[b] of V (nmax <= 64 rows of n per matrix) <- H V (forward = 0: B_{J-1} first) or H^T V
// (forward = 1: B_0^T first); one CTA per matrix.  Per block j: W = V_j Y^T (32 reflectors x the rows) over column
// chunks of V_j and Y staged in shared memory (thread tile: 4 reflectors x rows {r, r + 32}, float4 along the
// columns, so 6 shared loads feed 32 FMAs), Z = T_j^T W or T_j W, then Y -= Z^T V_j chunk by chunk (thread tile:
// rows {2q, 2q + 1} x columns {4p .. 4p + 3, 32 + 4p .. 35 + 4p}).  Y lives in global memory (L2) between chunks, so
// the CTA's shared memory does not grow with n and several CTAs share an SM.  A block's chunks (pass 1, then the
// same columns again for pass 2) run as one sequence through two buffers: the copies of chunk t + 1 are in flight
// while chunk t is consumed.  Pass 1 leaves Y unchanged and pass 2 writes only the chunk it has consumed, so
// every prefetched chunk holds current data; the sequence restarts at each block, whose columns the previous
// block's pass 2 has just written.
__global__ void __launch_bounds__(kT, 3) k_reflect_wy_tiled(const TriDesc32 *__restrict__ descs,
                                                         const float *__restrict__ Tall, int J,
                                                         const int *__restrict__ nrow, float *__restrict__ V, int nmax,
                                                         int forward) {
    const int b = blockIdx.x;
    const TriDesc32 D = descs[b];
    const int n = D.n;
    const int R = min(nrow ? nrow[b] : nmax, min(nmax, kTR));
    const int Jb = wy_blocks(n);
    if (R <= 0 || Jb == 0) return;
    extern __shared__ __align__(16) float wsm[];
    float *Buf = wsm;                        // two chunk buffers
    float *Ws = Buf + 2 * kTBuf;             // W, then Z (32 x (kTR + 1))
    float *Ts = Ws + kNB * (kTR + 1);        // T_j (32 x 33)
    const int tid = threadIdx.x;
    const int ti = tid >> 5, tr = tid & 31;            // pass 1 / Z: reflectors 4 ti .. 4 ti + 3, rows tr, tr + 32
    const int pq = 2 * (tid >> 3), pp = 4 * (tid & 7);   // pass 2: rows pq, pq + 1; columns pp.., 32 + pp..
    float *Yg = V + (long long)b * nmax * n;
    for (int s = 0; s < Jb; ++s) {
        const int j = forward ? s : Jb - 1 - s;
        const int k0 = j * kNB, kb = min(kNB, n - 2 - k0), m0 = n - k0 - 1, c0 = k0 + 1;
        const int nch = (m0 + kTCW - 1) / kTCW;   // chunks per pass
        __syncthreads();   // the previous block is done with Ts, Ws and both buffers; its writes of Y are visible
        const float *Tg = Tall + ((long long)b * J + j) * kNB * kNB;
        for (int idx = tid; idx < kNB * kNB; idx += kT) Ts[(idx >> 5) * (kNB + 1) + (idx & 31)] = Tg[idx];
        // copies of chunk t (columns [cbeg, cbeg + cw) of the block's c0 .. n - 1, cbeg = (t mod nch) kTCW) into
        // buffer t & 1: reflector i zero before column k0 + 1 + i and for i >= kb, rows >= R zero
        auto issue = [&](int t) {
            const int cbeg = (t % nch) * kTCW, cw = min(kTCW, m0 - cbeg);
            float *Vb = Buf + (t & 1) * kTBuf, *Yb = Vb + kNB * kTLd;
#pragma unroll
            for (int u = 0; u < kNB * kTCW / kT; ++u) {
                const int idx = tid + u * kT, i = idx / kTCW, cc = idx % kTCW;
                const bool ok = i < kb && cc < cw && cbeg + cc >= i;
                cp_async_zfill(Vb + i * kTLd + cc, ok ? D.A + (long long)(k0 + i) * D.lda + c0 + cbeg + cc : D.A, 4,
                               ok ? 4 : 0);
            }
#pragma unroll
            for (int u = 0; u < kTR * kTCW / kT; ++u) {
                const int idx = tid + u * kT, r = idx / kTCW, cc = idx % kTCW;
                const bool ok = r < R && cc < cw;
                cp_async_zfill(Yb + r * kTLd + cc, ok ? Yg + (long long)r * n + c0 + cbeg + cc : Yg, 4, ok ? 4 : 0);
            }
            cp_async_commit();
        };
        float w[4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) w[a][0] = w[a][1] = 0.f;
        issue(0);
        for (int t = 0; t < 2 * nch; ++t) {
            if (t + 1 < 2 * nch) {
                issue(t + 1);
                cp_async_wait_group<1>();
            } else {
                cp_async_wait_group<0>();
            }
            __syncthreads();   // chunk t complete for every thread
            const float *Vc = Buf + (t & 1) * kTBuf, *Yc = Vc + kNB * kTLd;
            if (t < nch) {
                // pass 1: W += V_j Y^T over this chunk
#pragma unroll 4
                for (int cc = 0; cc < kTCW; cc += 4) {
                    const float4 y0 = *reinterpret_cast<const float4 *>(Yc + tr * kTLd + cc);
                    const float4 y1 = *reinterpret_cast<const float4 *>(Yc + (tr + 32) * kTLd + cc);
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const float4 v = *reinterpret_cast<const float4 *>(Vc + (4 * ti + a) * kTLd + cc);
                        w[a][0] = fmaf(v.x, y0.x, fmaf(v.y, y0.y, fmaf(v.z, y0.z, fmaf(v.w, y0.w, w[a][0]))));
                        w[a][1] = fmaf(v.x, y1.x, fmaf(v.y, y1.y, fmaf(v.z, y1.z, fmaf(v.w, y1.w, w[a][1]))));
                    }
                }
                if (t == nch - 1) {
                    // Z = T_j^T W (forward) or T_j W, into Ws
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        Ws[(4 * ti + a) * (kTR + 1) + tr] = w[a][0];
                        Ws[(4 * ti + a) * (kTR + 1) + tr + 32] = w[a][1];
                    }
                    __syncthreads();
                    float z[4][2];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int i = 4 * ti + a;
                        float z0 = 0.f, z1 = 0.f;
#pragma unroll 8
                        for (int l = 0; l < kNB; ++l) {
                            const float tt = forward ? Ts[l * (kNB + 1) + i] : Ts[i * (kNB + 1) + l];
                            z0 = fmaf(tt, Ws[l * (kTR + 1) + tr], z0);
                            z1 = fmaf(tt, Ws[l * (kTR + 1) + tr + 32], z1);
                        }
                        z[a][0] = z0;
                        z[a][1] = z1;
                    }
                    __syncthreads();   // every W read
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        Ws[(4 * ti + a) * (kTR + 1) + tr] = z[a][0];
                        Ws[(4 * ti + a) * (kTR + 1) + tr + 32] = z[a][1];
                    }
                }
            } else if (pq < R) {
                // pass 2: Y -= Z^T V_j over this chunk (Z complete: the barrier after the next chunk's wait)
                const int cbeg = (t - nch) * kTCW, cw = min(kTCW, m0 - cbeg);
                float y[2][8];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const float4 lo = *reinterpret_cast<const float4 *>(Yc + (pq + q) * kTLd + pp);
                    const float4 hi = *reinterpret_cast<const float4 *>(Yc + (pq + q) * kTLd + 32 + pp);
                    y[q][0] = lo.x; y[q][1] = lo.y; y[q][2] = lo.z; y[q][3] = lo.w;
                    y[q][4] = hi.x; y[q][5] = hi.y; y[q][6] = hi.z; y[q][7] = hi.w;
                }
#pragma unroll 4
                for (int i = 0; i < kNB; ++i) {
                    const float z0 = Ws[i * (kTR + 1) + pq], z1 = Ws[i * (kTR + 1) + pq + 1];
                    const float4 lo = *reinterpret_cast<const float4 *>(Vc + i * kTLd + pp);
                    const float4 hi = *reinterpret_cast<const float4 *>(Vc + i * kTLd + 32 + pp);
                    const float ve[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        y[0][e] = fmaf(-z0, ve[e], y[0][e]);
                        y[1][e] = fmaf(-z1, ve[e], y[1][e]);
                    }
                }
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    if (pq + q < R)
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int cc = (e < 4 ? pp : 32 + pp) + (e & 3);
                            if (cc < cw) Yg[(long long)(pq + q) * n + c0 + cbeg + cc] = y[q][e];
                        }
            }
            __syncthreads();   // chunk t consumed before its buffer takes chunk t + 2
        }
    }
}

// Arithmetic of the projection: FP32, or double-float for FP64 data.
struct ProjF32 {
    using In = float;
    using S = float;
    static __device__ __forceinline__ S load(float x) { return x; }
    static __device__ __forceinline__ float store(S x) { return x; }
    static __device__ __forceinline__ S zero() { return 0.f; }
    static __device__ __forceinline__ S neg(S x) { return -x; }
    static __device__ __forceinline__ void fma(S &acc, S a, S b) { acc = fmaf(a, b, acc); }
};
struct ProjDF {
    using In = double;
    using S = float2;
    static __device__ __forceinline__ S load(double x) { return split_df(x); }
    static __device__ __forceinline__ double store(S x) { return df_val(x.x, x.y); }
    static __device__ __forceinline__ S zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ S neg(S x) { return make_float2(-x.x, -x.y); }
    static __device__ __forceinline__ void fma(S &acc, S a, S b) { df_fma(acc.x, acc.y, a, b); }
};

// rows mu < nk = nkeep[b] of X -= their projection on the orthonormal rows 0..nk-1 of Y (two passes of
// C = X Y^T, X -= C Y).  CTA: kPoRows rows of X kept in shared memory; Y streamed in column chunks.
template <class P>
__global__ void __launch_bounds__(kT) k_project_rows(const int *__restrict__ nkeep, const typename P::In *__restrict__ Y,
                                                     typename P::In *__restrict__ X, int n, int nmax) {
    using S = typename P::S;
    const int b = blockIdx.x;
    const int nk = nkeep[b];
    const int g0 = blockIdx.y * kPoRows;
    if (g0 >= nk) return;
    const int rows = min(kPoRows, nk - g0);
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    constexpr int ldy = kPoCW + 1;
    extern __shared__ __align__(16) unsigned char praw[];
    S *Xs = reinterpret_cast<S *>(praw);        // kPoRows x n
    S *Ys = Xs + (long long)kPoRows * n;        // nk x ldy (one chunk)
    S *Cs = Ys + (long long)kPoMaxY * ldy;      // kPoRows x kPoMaxY: -C
    const typename P::In *Yb = Y + (long long)b * nmax * n;
    typename P::In *Xg = X + ((long long)b * nmax + g0) * n;
    // rows of X and chunks of Y arrive by asynchronous element copies into their shared slots (a double in the
    // 8-byte slot of its (hi, lo) pair), then each thread converts the elements it copied
    constexpr int E = (int)sizeof(typename P::In);
    auto convert_own = [&](S *base, int cnt, int ld_s, int w) {
        if constexpr (E == 8) {
            for (int r = wid; r < cnt; r += kT / 32)
                for (int c = lane; c < w; c += 32) {
                    S *p = base + (long long)r * ld_s + c;
                    *p = P::load(*reinterpret_cast<const double *>(p));
                }
        }
    };
    for (int r = wid; r < rows; r += kT / 32)
        for (int c = lane; c < n; c += 32) cp_async_zfill(Xs + (long long)r * n + c, Xg + (long long)r * n + c, E, E);
    cp_async_wait_all();
    convert_own(Xs, rows, n, n);
    auto load_chunk = [&](int ch, int w) {
        for (int nu = wid; nu < nk; nu += kT / 32)
            for (int c = lane; c < w; c += 32) cp_async_zfill(Ys + nu * ldy + c, Yb + (long long)nu * n + ch + c, E, E);
        cp_async_wait_all();
        convert_own(Ys, nk, ldy, w);
    };
    for (int pass = 0; pass < 2; ++pass) {
        S c0 = P::zero(), c1 = P::zero();
        for (int ch = 0; ch < n; ch += kPoCW) {
            const int w = min(kPoCW, n - ch);
            __syncthreads();
            load_chunk(ch, w);
            __syncthreads();
            if (wid < rows) {
                const S *x = Xs + (long long)wid * n + ch;
                if (lane < nk) {
                    const S *yr = Ys + lane * ldy;
                    for (int c = 0; c < w; ++c) P::fma(c0, x[c], yr[c]);
                }
                if (lane + 32 < nk) {
                    const S *yr = Ys + (lane + 32) * ldy;
                    for (int c = 0; c < w; ++c) P::fma(c1, x[c], yr[c]);
                }
            }
        }
        if (wid < rows) {
            if (lane < nk) Cs[wid * kPoMaxY + lane] = P::neg(c0);
            if (lane + 32 < nk) Cs[wid * kPoMaxY + lane + 32] = P::neg(c1);
        }
        for (int ch = 0; ch < n; ch += kPoCW) {
            const int w = min(kPoCW, n - ch);
            __syncthreads();
            load_chunk(ch, w);
            __syncthreads();
            if (wid < rows) {
                S *x = Xs + (long long)wid * n + ch;
                const S *cr = Cs + wid * kPoMaxY;
                for (int c = lane; c < w; c += 32) {
                    S acc = x[c];
                    for (int nu = 0; nu < nk; ++nu) P::fma(acc, cr[nu], Ys[nu * ldy + c]);
                    x[c] = acc;
                }
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < rows * n; i += kT) Xg[i] = P::store(Xs[i]);
}

// Same projection with all of Y resident in shared memory (loaded once for both passes) and one row of X per
// warp: every warp works on its own row against the shared, read-only Y, so after the load no block barrier
// is needed.  W = warps = rows per CTA (blockDim.x = 32 W).
template <class P>
__global__ void __launch_bounds__(1024) k_project_rows_y(const int *__restrict__ nkeep,
                                                         const typename P::In *__restrict__ Y,
                                                         typename P::In *__restrict__ X, int n, int nmax) {
    using S = typename P::S;
    const int W = blockDim.x >> 5;
    const int b = blockIdx.x;
    const int nk = nkeep[b];
    const int g0 = blockIdx.y * W;
    if (g0 >= nk) return;
    const int rows = min(W, nk - g0);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ldy = n | 1;
    extern __shared__ __align__(16) unsigned char praw[];
    S *Ys = reinterpret_cast<S *>(praw);          // nk x ldy
    S *Xs = Ys + (long long)nmax * ldy;           // W x n
    S *Cs = Xs + (long long)W * n;                // W x kPoMaxY: -C
    const typename P::In *Yb = Y + (long long)b * nmax * n;
    typename P::In *Xg = X + ((long long)b * nmax + g0) * n;
    constexpr int E = (int)sizeof(typename P::In);
    for (int nu = wid; nu < nk; nu += W)
        for (int c = lane; c < n; c += 32) cp_async_zfill(Ys + (long long)nu * ldy + c, Yb + (long long)nu * n + c, E, E);
    if (wid < rows)
        for (int c = lane; c < n; c += 32) cp_async_zfill(Xs + (long long)wid * n + c, Xg + (long long)wid * n + c, E, E);
    cp_async_wait_all();
    if constexpr (E == 8) {   // each thread converts the doubles it copied into (hi, lo) pairs
        for (int nu = wid; nu < nk; nu += W)
            for (int c = lane; c < n; c += 32) {
                S *q = Ys + (long long)nu * ldy + c;
                *q = P::load(*reinterpret_cast<const double *>(q));
            }
        if (wid < rows)
            for (int c = lane; c < n; c += 32) {
                S *q = Xs + (long long)wid * n + c;
                *q = P::load(*reinterpret_cast<const double *>(q));
            }
    }
    __syncthreads();
    if (wid >= rows) return;
    S *x = Xs + (long long)wid * n;
    S *cr = Cs + wid * kPoMaxY;
    for (int pass = 0; pass < 2; ++pass) {
        S c0 = P::zero(), c1 = P::zero();
        if (lane < nk) {
            const S *yr = Ys + (long long)lane * ldy;
            for (int c = 0; c < n; ++c) P::fma(c0, x[c], yr[c]);
        }
        if (lane + 32 < nk) {
            const S *yr = Ys + (long long)(lane + 32) * ldy;
            for (int c = 0; c < n; ++c) P::fma(c1, x[c], yr[c]);
        }
        if (lane < nk) cr[lane] = P::neg(c0);
        if (lane + 32 < nk) cr[lane + 32] = P::neg(c1);
        __syncwarp();
        for (int c = lane; c < n; c += 32) {
            S acc = x[c];
            for (int nu = 0; nu < nk; ++nu) P::fma(acc, cr[nu], Ys[(long long)nu * ldy + c]);
            x[c] = acc;
        }
        __syncwarp();
    }
    for (int c = lane; c < n; c += 32) Xg[(long long)wid * n + c] = P::store(x[c]);
}

template <class K>
cudaError_t smem_attr(K kernel, size_t sh) {
    if (sh > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    return cudaSuccess;
}

constexpr size_t kSmemCap = 227 * 1024;

template <class P>
size_t project_rows_smem(int n) {
    return ((size_t)kPoRows * n + (size_t)kPoMaxY * (kPoCW + 1) + (size_t)kPoRows * kPoMaxY) * sizeof(typename P::S);
}

}  // namespace

size_t osv_wy_floats(int batch, int n) { return (size_t)batch * std::max(wy_blocks(n), 1) * kNB * kNB; }

cudaError_t osv_wy_prepare(const TriDesc32 *d, int batch, int n, float *T, cudaStream_t s) {
    const int J = wy_blocks(n);
    if (batch <= 0 || J == 0) return cudaSuccess;
    const size_t sh = ((size_t)kNB * kLdc + 2 * (size_t)kNB * (kNB + 1)) * sizeof(float);
    if (sh > kSmemCap) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = smem_attr(k_wy_t, sh)) != cudaSuccess) return e;
    count_launch();
    k_wy_t<<<dim3(batch, J), kT, sh, s>>>(d, T, J);
    return cudaGetLastError();
}

cudaError_t osv_reflect_wy(const TriDesc32 *d, const float *T, int batch, int n, int nmax, const int *nrow, float *V,
                           int forward, cudaStream_t s) {
    if (batch <= 0 || nmax <= 0 || wy_blocks(n) == 0) return cudaSuccess;
    if (nmax > kTR) return cudaErrorInvalidValue;
    const size_t sh = (2 * (size_t)kTBuf + (size_t)kNB * (kTR + 1) + (size_t)kNB * (kNB + 1)) * sizeof(float);
    cudaError_t e;
    if ((e = smem_attr(k_reflect_wy_tiled, sh)) != cudaSuccess) return e;
    count_launch();
    k_reflect_wy_tiled<<<batch, kT, sh, s>>>(d, T, wy_blocks(n), nrow, V, nmax, forward);
    return cudaGetLastError();
}

bool osv_project_rows_fits(int n, int nmax) {
    return nmax <= kPoMaxY && project_rows_smem<ProjDF>(n) <= kSmemCap;
}

template <class R>
cudaError_t osv_project_rows(const int *nkeep, const R *Y, R *X, int batch, int n, int nmax, cudaStream_t s) {
    using P = std::conditional_t<sizeof(R) == 4, ProjF32, ProjDF>;
    if (batch <= 0 || nmax <= 0) return cudaSuccess;
    if (nmax <= kPoMaxY) {
        // Y resident: rows per CTA so that the grid is about one CTA per SM (at most 32 rows, one warp each)
        const int per = std::max(1, 152 / batch);
        const int W = std::min(32, std::max(1, (nmax + per - 1) / per));
        const size_t shy = ((size_t)nmax * (n | 1) + (size_t)W * n + (size_t)W * kPoMaxY) * sizeof(typename P::S);
        if (shy <= kSmemCap) {
            cudaError_t e;
            if ((e = smem_attr(k_project_rows_y<P>, shy)) != cudaSuccess) return e;
            count_launch();
            k_project_rows_y<P><<<dim3(batch, (nmax + W - 1) / W), 32 * W, shy, s>>>(nkeep, Y, X, n, nmax);
            return cudaGetLastError();
        }
    }
    const size_t sh = project_rows_smem<P>(n);
    if (nmax > kPoMaxY || sh > kSmemCap) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = smem_attr(k_project_rows<P>, sh)) != cudaSuccess) return e;
    count_launch();
    k_project_rows<P><<<dim3(batch, (nmax + kPoRows - 1) / kPoRows), kT, sh, s>>>(nkeep, Y, X, n, nmax);
    return cudaGetLastError();
}

template cudaError_t osv_project_rows<float>(const int *, const float *, float *, int, int, int, cudaStream_t);
template cudaError_t osv_project_rows<double>(const int *, const double *, double *, int, int, int, cudaStream_t);

}  // namespace osv
