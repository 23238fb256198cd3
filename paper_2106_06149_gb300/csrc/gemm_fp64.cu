// Grouped FP64 GEMM on the CUDA cores: one launch runs every problem of a batch (the FP64 path's dense
// contractions: T_kk Gram products, half transforms, pair blocks, adjoint products).  64 x 64 output tile per
// CTA, 256 threads with a 4 x 4 register tile each, K staged through shared memory in steps of 16.
// Optional row/column index maps let one descriptor read a gathered operand (local fitting domains, stacked
// OSV sets) without a copy.
#include <algorithm>

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
// TM x TN outputs per thread and a (16 TM) x (16 TN) tile per CTA, the shape chosen per batch (64 x 64 in
// general, 80 x 80 for pair-domain products of order <= 80, 48-row or 48-column tiles for 40-row / 40-column
// problems).  The next K step's operands are loaded into registers before the current step's
// products, and staged after them.
template <int TM, int TN>
__global__ void __launch_bounds__(NT) k_gemm_df(const GemmDesc *__restrict__ descs,
                                                 const long long *__restrict__ tile0, int nprob) {
    constexpr int TBM = 16 * TM, TBN = 16 * TN;   // tile edges
    constexpr int LA = TBM * BK / NT, LB = TBN * BK / NT;   // operand elements per thread and K step
    const long long t = blockIdx.x;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile0[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const GemmDesc g = descs[lo];
    const long long local = t - tile0[lo];
    const int tiles_n = (g.N + TBN - 1) / TBN;
    const int m0 = int(local / tiles_n) * TBM, n0 = int(local % tiles_n) * TBN;

    __shared__ float2 As[2][BK][TBM + 1];
    __shared__ float2 Bs[2][BK][TBN + 1];

    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;
    float ah[TM][TN], al[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) ah[a][b] = al[a][b] = 0.f;

    double ra[LA], rb[LB];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            const int e = tid + r * NT;
            int mm, kk;
            if (g.transA == 0) { mm = e / BK; kk = e % BK; } else { kk = e / TBM; mm = e % TBM; }
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
        for (int r = 0; r < LB; ++r) {
            const int e = tid + r * NT;
            int kk, nn;
            if (g.transB == 0) { kk = e / TBN; nn = e % TBN; } else { nn = e / BK; kk = e % BK; }
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
            if (g.transA == 0) { mm = e / BK; kk = e % BK; } else { kk = e / TBM; mm = e % TBM; }
            As[buf][kk][mm] = split_df(ra[r]);
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {
            const int e = tid + r * NT;
            int kk, nn;
            if (g.transB == 0) { kk = e / TBN; nn = e % TBN; } else { nn = e / BK; kk = e % BK; }
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
            float2 a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][tr + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tc + 16 * j];
            if constexpr (TM == 5 && TN == 5) {
                df_tile5(ah, al, a, b);
            } else {
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) df_fma(ah[i][j], al[i][j], a[i], b[j]);
            }
        }
        if (kt + 1 < nk) stage(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int m = m0 + tr + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + tc + 16 * j;
            if (n >= g.N) continue;
            const long long nc = g.n_idx_c ? g.n_idx_c[n] : n;
            double *c = g.C + (long long)m * g.ldc + nc;
            const double v = df_val(ah[i][j], al[i][j]);
            const double av = g.alpha == 1.0 ? v : g.alpha * v;
            if (g.atomic) atomicAdd(c, av);
            else *c = g.beta != 0.0 ? av + g.beta * *c : av;
        }
    }
}

}  // namespace

cudaError_t gemm_batch_run_df(const GemmBatch &b, cudaStream_t s) {
    if (b.tiles == 0) return cudaSuccess;
    count_launch();
    const int c = b.df_shape;
    const GemmDesc *d = b.d_desc;
    const long long *t0 = b.d_tile0_df;
    const unsigned grid = (unsigned)b.tiles_df;
    const int np = (int)b.h.size();
    switch (c) {
        case 1: k_gemm_df<5, 5><<<grid, NT, 0, s>>>(d, t0, np); break;
        case 2: k_gemm_df<3, 5><<<grid, NT, 0, s>>>(d, t0, np); break;
        case 3: k_gemm_df<5, 3><<<grid, NT, 0, s>>>(d, t0, np); break;
        case 4: k_gemm_df<3, 3><<<grid, NT, 0, s>>>(d, t0, np); break;
        default: k_gemm_df<4, 4><<<grid, NT, 0, s>>>(d, t0, np); break;
    }
    return cudaGetLastError();
}

cudaError_t gemm_batch_upload(GemmBatch &b) {
    gemm_batch_free(b);
    if (b.h.empty()) return cudaSuccess;
    // 64 x 64 tile offsets (FP64 kernel) and the double-float kernel's tile shape: the one with the least
    // ceil(tiles / SMs) x (tile area), the padded work of the busiest SM (the kernel is FP32-throughput bound, so
    // an SM's co-resident tiles share its pipes; a near-empty last round still costs a whole tile)
    constexpr int kShapes = 5;
    const int sm[kShapes] = {64, 80, 48, 80, 48}, sn[kShapes] = {64, 80, 80, 48, 48};
    std::vector<long long> t[kShapes];
    for (int c = 0; c < kShapes; ++c) {
        t[c].assign(b.h.size() + 1, 0);
        for (size_t i = 0; i < b.h.size(); ++i) {
            const GemmDesc &g = b.h[i];
            const bool live = g.M > 0 && g.N > 0;
            t[c][i + 1] = t[c][i] + (live ? (long long)((g.M + sm[c] - 1) / sm[c]) * ((g.N + sn[c] - 1) / sn[c]) : 0);
        }
    }
    int best = 0;
    double best_cost = 0.0;
    for (int c = 0; c < kShapes; ++c) {
        const double per_sm = (double)((t[c].back() + 151) / 152);
        const double cost = per_sm * sm[c] * sn[c];
        if (c == 0 || cost < best_cost) {
            best = c;
            best_cost = cost;
        }
    }
    b.tiles = t[0].back();
    b.df_shape = best;
    b.df_rule = best;
    b.tiles_df = t[best].back();
    cudaError_t e = cudaMalloc(&b.d_desc, b.h.size() * sizeof(GemmDesc));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&b.d_tile0, t[0].size() * sizeof(long long));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&b.d_tile0_df, t[best].size() * sizeof(long long));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(b.d_desc, b.h.data(), b.h.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(b.d_tile0_df, t[best].data(), t[best].size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(b.d_tile0, t[0].data(), t[0].size() * sizeof(long long), cudaMemcpyHostToDevice);
}

cudaError_t gemm_batch_run(const GemmBatch &b, cudaStream_t s) {
    if (b.tiles == 0) return cudaSuccess;
    // problems without tiles are skipped by the search: tile0 is non-decreasing and the search picks the
    // last problem whose first tile is <= t, which is the one owning t.
    count_launch();
    k_gemm_fp64<<<(unsigned)b.tiles, NT, 0, s>>>(b.d_desc, b.d_tile0, (int)b.h.size());
    return cudaGetLastError();
}

cudaError_t gemm_batch_set_df_shape(GemmBatch &b, int shape) {
    if (b.h.empty() || shape == b.df_shape) return cudaSuccess;
    if (shape < 0 || shape > 4) return cudaErrorInvalidValue;
    const int sm[5] = {64, 80, 48, 80, 48}, sn[5] = {64, 80, 80, 48, 48};
    std::vector<long long> t(b.h.size() + 1, 0);
    for (size_t i = 0; i < b.h.size(); ++i) {
        const GemmDesc &g = b.h[i];
        const bool live = g.M > 0 && g.N > 0;
        t[i + 1] = t[i] + (live ? (long long)((g.M + sm[shape] - 1) / sm[shape]) * ((g.N + sn[shape] - 1) / sn[shape]) : 0);
    }
    if (b.d_tile0_df) cudaFree(b.d_tile0_df);
    b.d_tile0_df = nullptr;
    cudaError_t e = cudaMalloc(&b.d_tile0_df, t.size() * sizeof(long long));
    if (e != cudaSuccess) return e;
    b.df_shape = shape;
    b.tiles_df = t.back();
    return cudaMemcpy(b.d_tile0_df, t.data(), t.size() * sizeof(long long), cudaMemcpyHostToDevice);
}

void gemm_batch_free(GemmBatch &b) {
    if (b.d_desc) cudaFree(b.d_desc);
    if (b.d_tile0) cudaFree(b.d_tile0);
    if (b.d_tile0_df) cudaFree(b.d_tile0_df);
    b.d_desc = nullptr;
    b.d_tile0 = nullptr;
    b.d_tile0_df = nullptr;
    b.tiles = b.tiles_df = 0;
    b.df_shape = b.df_rule = 0;
}

}  // namespace osv
