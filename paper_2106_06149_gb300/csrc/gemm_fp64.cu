// Grouped FP64 GEMM on the CUDA cores: one launch runs every problem of a batch (the FP64 path's dense
// contractions: T_kk Gram products, half transforms, pair blocks, adjoint products).  64 x 64 output tile per
// CTA, 256 threads with a 4 x 4 register tile each, K staged through shared memory in steps of 16.
// Optional row/column index maps let one descriptor read a gathered operand (local fitting domains, stacked
// OSV sets) without a copy.
#include "common.cuh"

namespace osv {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__global__ void __launch_bounds__(NT) k_gemm_fp64(const GemmDesc *__restrict__ descs,
                                                   const long long *__restrict__ tile0, int nprob) {
    // locate the problem of this tile (tile0 is increasing, tile0[nprob] = total)
    const long long t = blockIdx.x;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile0[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const GemmDesc g = descs[lo];
    const long long local = t - tile0[lo];
    const int tiles_n = (g.N + BN - 1) / BN;
    const int m0 = int(local / tiles_n) * BM, n0 = int(local % tiles_n) * BN;

    __shared__ double As[2][BK][BM + 1];
    __shared__ double Bs[2][BK][BN + 1];

    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;   // 16 x 16 thread grid, 4 x 4 outputs each (stride 16)
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

    auto load = [&](int buf, int k0) {
        // A tile: BM x BK elements, 4 per thread
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + r * NT;
            int mm, kk;
            if (g.transA == 0) { mm = e / BK; kk = e % BK; } else { kk = e / BM; mm = e % BM; }
            const int m = m0 + mm, k = k0 + kk;
            double v = 0.0;
            if (m < g.M && k < g.K) {
                const long long kc = g.k_idx_a ? g.k_idx_a[k] : k;
                if (g.transA == 0) {
                    const long long mr = g.a_rows ? g.a_rows[m] : m;
                    v = g.A[mr * g.lda + kc];
                } else {
                    v = g.A[kc * g.lda + m];
                }
            }
            As[buf][kk][mm] = v;
        }
        // B tile: BK x BN elements
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + r * NT;
            int kk, nn;
            if (g.transB == 0) { kk = e / BN; nn = e % BN; } else { nn = e / BK; kk = e % BK; }
            const int n = n0 + nn, k = k0 + kk;
            double v = 0.0;
            if (n < g.N && k < g.K) {
                const long long kr = g.k_idx_b ? g.k_idx_b[k] : k;
                const long long nc = g.n_idx_b ? g.n_idx_b[n] : n;
                v = (g.transB == 0) ? g.B[kr * g.ldb + nc] : g.B[nc * g.ldb + kr];
            }
            Bs[buf][kk][nn] = v;
        }
    };

    const int nk = (g.K + BK - 1) / BK;
    if (nk > 0) load(0, 0);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) load(buf ^ 1, (kt + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][tr + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[buf][kk][tc + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + tr + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tc + 16 * j;
            if (n >= g.N) continue;
            const long long nc = g.n_idx_c ? g.n_idx_c[n] : n;
            double *c = g.C + (long long)m * g.ldc + nc;
            if (g.atomic) atomicAdd(c, g.alpha * acc[i][j]);
            else *c = g.alpha * acc[i][j] + (g.beta != 0.0 ? g.beta * *c : 0.0);
        }
    }
}

// The same grouped GEMM in double-float arithmetic (mixed modes): operands split into FP32 (hi, lo) pairs by
// integer operations while staged, products and sums on the FP32 pipe (common.cuh); ~2^-44 relative.
// TM x TM outputs per thread and a (16 TM) x (16 TM) tile per CTA: TM = 4 (64 x 64) for general batches,
// TM = 5 (80 x 80) where it pads less (pair-domain products of order <= 80 fill one tile).  The next K step's
// operands are loaded into registers before the current step's products, and staged after them.
template <int TM>
__global__ void __launch_bounds__(NT) k_gemm_df(const GemmDesc *__restrict__ descs,
                                                 const long long *__restrict__ tile0, int nprob) {
    constexpr int TB = 16 * TM;                 // tile edge
    constexpr int LA = TB * BK / NT;            // operand elements per thread and K step
    static_assert(TB * BK % NT == 0, "tile");
    const long long t = blockIdx.x;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile0[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const GemmDesc g = descs[lo];
    const long long local = t - tile0[lo];
    const int tiles_n = (g.N + TB - 1) / TB;
    const int m0 = int(local / tiles_n) * TB, n0 = int(local % tiles_n) * TB;

    __shared__ float2 As[2][BK][TB + 1];
    __shared__ float2 Bs[2][BK][TB + 1];

    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;
    float ah[TM][TM], al[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) ah[a][b] = al[a][b] = 0.f;

    double ra[LA], rb[LA];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            const int e = tid + r * NT;
            int mm, kk;
            if (g.transA == 0) { mm = e / BK; kk = e % BK; } else { kk = e / TB; mm = e % TB; }
            const int m = m0 + mm, k = k0 + kk;
            double v = 0.0;
            if (m < g.M && k < g.K) {
                const long long kc = g.k_idx_a ? g.k_idx_a[k] : k;
                if (g.transA == 0) {
                    const long long mr = g.a_rows ? g.a_rows[m] : m;
                    v = g.A[mr * g.lda + kc];
                } else {
                    v = g.A[kc * g.lda + m];
                }
            }
            ra[r] = v;
        }
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            const int e = tid + r * NT;
            int kk, nn;
            if (g.transB == 0) { kk = e / TB; nn = e % TB; } else { nn = e / BK; kk = e % BK; }
            const int n = n0 + nn, k = k0 + kk;
            double v = 0.0;
            if (n < g.N && k < g.K) {
                const long long kr = g.k_idx_b ? g.k_idx_b[k] : k;
                const long long nc = g.n_idx_b ? g.n_idx_b[n] : n;
                v = (g.transB == 0) ? g.B[kr * g.ldb + nc] : g.B[nc * g.ldb + kr];
            }
            rb[r] = v;
        }
    };
    auto stage = [&](int buf) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            const int e = tid + r * NT;
            int mm, kk;
            if (g.transA == 0) { mm = e / BK; kk = e % BK; } else { kk = e / TB; mm = e % TB; }
            As[buf][kk][mm] = split_df(ra[r]);
        }
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            const int e = tid + r * NT;
            int kk, nn;
            if (g.transB == 0) { kk = e / TB; nn = e % TB; } else { nn = e / BK; kk = e % BK; }
            Bs[buf][kk][nn] = split_df(rb[r]);
        }
    };

    const int nk = (g.K + BK - 1) / BK;
    if (nk > 0) {
        fetch(0);
        stage(0);
    }
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) fetch((kt + 1) * BK);
#pragma unroll 2
        for (int kk = 0; kk < BK; ++kk) {
            float2 a[TM], b[TM];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][tr + 16 * i];
#pragma unroll
            for (int j = 0; j < TM; ++j) b[j] = Bs[buf][kk][tc + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TM; ++j) df_fma(ah[i][j], al[i][j], a[i], b[j]);
        }
        if (kt + 1 < nk) stage(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int m = m0 + tr + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < TM; ++j) {
            const int n = n0 + tc + 16 * j;
            if (n >= g.N) continue;
            const long long nc = g.n_idx_c ? g.n_idx_c[n] : n;
            double *c = g.C + (long long)m * g.ldc + nc;
            const double v = df_val(ah[i][j], al[i][j]);
            if (g.atomic) atomicAdd(c, g.alpha * v);
            else *c = g.alpha * v + (g.beta != 0.0 ? g.beta * *c : 0.0);
        }
    }
}

}  // namespace

cudaError_t gemm_batch_run_df(const GemmBatch &b, cudaStream_t s) {
    if (b.tiles == 0) return cudaSuccess;
    count_launch();
    if (b.tiles80 > 0 && b.tiles80 * 80LL * 80 < b.tiles * 64LL * 64)
        k_gemm_df<5><<<(unsigned)b.tiles80, NT, 0, s>>>(b.d_desc, b.d_tile0_80, (int)b.h.size());
    else
        k_gemm_df<4><<<(unsigned)b.tiles, NT, 0, s>>>(b.d_desc, b.d_tile0, (int)b.h.size());
    return cudaGetLastError();
}

cudaError_t gemm_batch_upload(GemmBatch &b) {
    gemm_batch_free(b);
    if (b.h.empty()) return cudaSuccess;
    // per-problem tile offsets for 64 x 64 tiles and, for the double-float kernel, 80 x 80 tiles
    std::vector<long long> t0(b.h.size() + 1, 0), t80(b.h.size() + 1, 0);
    for (size_t i = 0; i < b.h.size(); ++i) {
        const GemmDesc &g = b.h[i];
        const bool live = g.M > 0 && g.N > 0;
        t0[i + 1] = t0[i] + (live ? (long long)((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN) : 0);
        t80[i + 1] = t80[i] + (live ? (long long)((g.M + 79) / 80) * ((g.N + 79) / 80) : 0);
    }
    b.tiles = t0.back();
    b.tiles80 = t80.back();
    cudaError_t e = cudaMalloc(&b.d_desc, b.h.size() * sizeof(GemmDesc));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&b.d_tile0, t0.size() * sizeof(long long));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&b.d_tile0_80, t80.size() * sizeof(long long));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(b.d_desc, b.h.data(), b.h.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(b.d_tile0_80, t80.data(), t80.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(b.d_tile0, t0.data(), t0.size() * sizeof(long long), cudaMemcpyHostToDevice);
}

cudaError_t gemm_batch_run(const GemmBatch &b, cudaStream_t s) {
    if (b.tiles == 0) return cudaSuccess;
    // problems without tiles are skipped by the search: tile0 is non-decreasing and the search picks the
    // last problem whose first tile is <= t, which is the one owning t.
    count_launch();
    k_gemm_fp64<<<(unsigned)b.tiles, NT, 0, s>>>(b.d_desc, b.d_tile0, (int)b.h.size());
    return cudaGetLastError();
}

void gemm_batch_free(GemmBatch &b) {
    if (b.d_desc) cudaFree(b.d_desc);
    if (b.d_tile0) cudaFree(b.d_tile0);
    if (b.d_tile0_80) cudaFree(b.d_tile0_80);
    b.d_desc = nullptr;
    b.d_tile0 = nullptr;
    b.d_tile0_80 = nullptr;
    b.tiles = b.tiles80 = 0;
}

}  // namespace osv
