// Grouped GEMM on tcgen05 tensor cores with exactly accumulated BF16 slices (unbiased, ~31 significant bits).
//
// Each operand row (A: row m over k; B: column n over k) gets a power-of-two scale 2^e with every |element| <=
// 2^e (a pre-pass).  An FP64 element x is rounded (integer arithmetic on its bit pattern, round half away from
// zero) to N = round(x 2^(31-e)), |N| <= 2^31, and N is cut into four signed base-256 digits
//   N = s1 2^24 + s2 2^16 + s3 2^8 + s4,   |s_i| <= 128  (exact BF16 values),
// so a product of slices is an integer of magnitude <= 2^14 and a sum of <= 1024 of them is exact in FP32.
// All sixteen slice products are accumulated in seven TMEM accumulators, one per order d = i + j, over chunks
// of 128 K: every partial sum stays exact, so the tensor-core accumulation has no rounding and no bias.  (Small
// elements of rows with a wide dynamic range live mostly in the low slices; dropping any low product would bias
// sums of squares such as the K_(ii,ii) and T_kk diagonals.)  After each chunk the accumulators are drained: the
// d = 0 part is an exact integer (int32 accumulator), the d >= 1 parts (2^-8 and smaller) are combined in FP32.
// The epilogue restores 2^(e_m + e_n - 14) in FP64.  The only errors are the rounding of x to 31 bits below its
// row scale and the FP32 rounding of the d >= 1 sum (2^-32 relative), both unbiased.
//
// One CTA = 256 threads = one 128 x 64 tile.  Slabs of 32 K are prefetched into registers while the tensor core
// works, sliced and stored in the canonical no-swizzle K-major layout (8 rows x 16 bytes = 8 BF16 per core-matrix
// row), double-buffered; thread 0 issues 2 k-steps x 16 tcgen05.mma.kind::f16 (BF16, M = 128, N = 64, K = 16).
// Waits are bounded (error word, bounded wait for in-flight MMAs, TMEM freed).
#include <cuda_bf16.h>

#include <cstdint>

#include "kernels.cuh"
#include "tc_gemm.h"

namespace osv {

namespace {

constexpr int BM = 128, BN = 64, BK = 32, NT = 256;
constexpr int NSLICE = 4;
constexpr int CHUNK_SLABS = 4;                        // 128 K per exact chunk
constexpr int A_SL = BM * BK * 2;                     // 8 KB per A slice
constexpr int B_SL = BN * BK * 2;                     // 4 KB per B slice
constexpr int STAGE = NSLICE * (A_SL + B_SL);          // 48 KB
constexpr int SMEM = 2 * STAGE + 1024;
constexpr int A_PER_T = BM * BK / NT;                 // 16
constexpr int B_PER_T = BN * BK / NT;                 // 8
constexpr long long kWaitBudget = 4LL << 30;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// bf16 K-major no swizzle: core matrix = 8 rows x 16 bytes (8 elements); a 32-wide slab row holds 4 core matrices
// (LBO = 128 B along K), 8-row groups are SBO = 512 B apart.
__device__ __forceinline__ uint32_t koff(int r, int k) {
    return (uint32_t)((r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((512u >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool bwait(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    uint32_t done = 0;
    while (true) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitBudget) return false;
    }
}

__device__ __forceinline__ void ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// element e of a rows x 32 slab (rows = 128 or 64): lanes cover (row % 8, k-pair % 4) -> distinct banks
__device__ __forceinline__ void slab_rc(int e, int &r, int &k) {
    const int lane = e & 31, grp = e >> 5;
    r = ((grp >> 2) << 3) + (lane >> 2);
    k = ((grp & 3) << 3) + ((lane & 3) << 1);   // this thread handles k and k + 1
}

// x = N 2^(e-31) + rounding, N cut into four signed base-256 digits (integer arithmetic only).
__device__ __forceinline__ void slice4(double x, int e, __nv_bfloat16 *s) {
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    long long n = 0;
    if (ex != 0) {                                           // zero and subnormal inputs slice to zero
        const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;   // value = mant 2^(ex-1075)
        const int sh = 1075 - ex + e - 31;                   // N = mant / 2^sh, sh >= 21 since |x| <= 2^e
        if (sh < 63) n = (mant + (1LL << (sh - 1))) >> sh;
        if (bits < 0) n = -n;
    }
    const int s1 = (int)((n + (1LL << 23)) >> 24);
    int r = (int)(n - ((long long)s1 << 24));
    const int s2 = (r + (1 << 15)) >> 16;
    r -= s2 << 16;
    const int s3 = (r + (1 << 7)) >> 8;
    const int s4 = r - (s3 << 8);
    s[0] = __float2bfloat16_rn((float)s1);
    s[1] = __float2bfloat16_rn((float)s2);
    s[2] = __float2bfloat16_rn((float)s3);
    s[3] = __float2bfloat16_rn((float)s4);
}

__global__ void __launch_bounds__(NT, 1) k_gemm_bf16x4(const GemmDesc *__restrict__ descs,
                                                      const long long *__restrict__ tile0, int nprob, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t s_taddr;
    __shared__ int s_fail;

    const long long t = blockIdx.x;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile0[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const GemmDesc g = descs[lo];
    const long long local = t - tile0[lo];
    const int tiles_n = (g.N + BN - 1) / BN;
    const int m0 = int(local / tiles_n) * BM, n0 = int(local % tiles_n) * BN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&s_taddr)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = s_taddr;

    // per-thread drain targets: TMEM lanes of warp % 4, columns 32 * (warp / 4) .. + 31
    int acc_i[32];
    float acc_s[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        acc_i[j] = 0;
        acc_s[j] = 0.f;
    }

    const int nslab = (g.K + BK - 1) / BK;
    double ra[A_PER_T], rb[B_PER_T];
    int rea[A_PER_T / 2], reb[B_PER_T / 2];
    auto prefetch = [&](int sl) {
        const int k0 = sl * BK;
#pragma unroll
        for (int i = 0; i < A_PER_T / 2; ++i) {
            int r, k;
            slab_rc(tid + i * NT, r, k);
            const int m = m0 + r;
            rea[i] = m < g.M ? g.ea[m] : 0;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int kk = k0 + k + q;
                double v = 0.0;
                if (m < g.M && kk < g.K) {
                    const long long kc = g.k_idx_a ? g.k_idx_a[kk] : kk;
                    v = g.transA == 0 ? g.A[(long long)(g.a_rows ? g.a_rows[m] : m) * g.lda + kc] : g.A[kc * g.lda + m];
                }
                ra[2 * i + q] = v;
            }
        }
#pragma unroll
        for (int i = 0; i < B_PER_T / 2; ++i) {
            int nn, k;
            slab_rc(tid + i * NT, nn, k);
            const int n = n0 + nn;
            reb[i] = n < g.N ? g.eb[n] : 0;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int kk = k0 + k + q;
                double v = 0.0;
                if (n < g.N && kk < g.K) {
                    const long long kr = g.k_idx_b ? g.k_idx_b[kk] : kk;
                    const long long nc = g.n_idx_b ? g.n_idx_b[n] : n;
                    v = g.transB == 0 ? g.B[kr * g.ldb + nc] : g.B[nc * g.ldb + kr];
                }
                rb[2 * i + q] = v;
            }
        }
    };

    auto drain = [&]() {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t lbase = taddr + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 32);
#pragma unroll
        for (int c = 0; c < 32; c += 16) {
            float v[16], l[16];
            ld16(lbase + c, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                acc_i[c + i] += __float2int_rn(v[i]);                        // exact integer (< 2^24)
                l[i] = 0.f;
            }
            // orders d = 6 .. 1 (smallest first), each worth 2^(-8 d) of the d = 0 unit
            const float sc[7] = {1.f, 3.90625e-3f, 1.52587890625e-5f, 5.9604644775390625e-8f, 2.3283064365386963e-10f,
                                 9.094947017729282e-13f, 3.552713678800501e-15f};
#pragma unroll
            for (int d = 2 * NSLICE - 2; d >= 1; --d) {
                ld16(lbase + (uint32_t)(d * BN) + c, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int i = 0; i < 16; ++i) l[i] = fmaf(v[i], sc[d], l[i]);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) acc_s[c + i] += l[i];
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
    };

    int issued[2] = {0, 0};
    bool ok = true;
    if (nslab > 0) prefetch(0);
    for (int sl = 0; sl < nslab; ++sl) {
        const int st = sl & 1;
        if (sl >= 2) {
            if (!bwait(&bar[st], (uint32_t)(((sl >> 1) - 1) & 1))) {
                if (tid == 0) raise_err(err, kDevTimeout);
                s_fail = 1;
            }
        }
        unsigned char *sA = smem + st * STAGE;
        unsigned char *sB = sA + NSLICE * A_SL;
#pragma unroll
        for (int i = 0; i < A_PER_T / 2; ++i) {
            int r, k;
            slab_rc(tid + i * NT, r, k);
            __nv_bfloat16 s0[NSLICE], s1[NSLICE];
            slice4(ra[2 * i], rea[i], s0);
            slice4(ra[2 * i + 1], rea[i], s1);
            const uint32_t o = koff(r, k);
#pragma unroll
            for (int q = 0; q < NSLICE; ++q) {
                __nv_bfloat162 pr;
                pr.x = s0[q];
                pr.y = s1[q];
                *(__nv_bfloat162 *)(sA + q * A_SL + o) = pr;
            }
        }
#pragma unroll
        for (int i = 0; i < B_PER_T / 2; ++i) {
            int nn, k;
            slab_rc(tid + i * NT, nn, k);
            __nv_bfloat16 s0[NSLICE], s1[NSLICE];
            slice4(rb[2 * i], reb[i], s0);
            slice4(rb[2 * i + 1], reb[i], s1);
            const uint32_t o = koff(nn, k);
#pragma unroll
            for (int q = 0; q < NSLICE; ++q) {
                __nv_bfloat162 pr;
                pr.x = s0[q];
                pr.y = s1[q];
                *(__nv_bfloat162 *)(sB + q * B_SL + o) = pr;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (s_fail) { ok = false; break; }
        const bool first_of_chunk = (sl % CHUNK_SLABS) == 0;
        const bool last_of_chunk = (sl % CHUNK_SLABS) == CHUNK_SLABS - 1 || sl == nslab - 1;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                const uint32_t off = ks * 256;
                bool fresh[2 * NSLICE - 1];
#pragma unroll
                for (int d = 0; d < 2 * NSLICE - 1; ++d) fresh[d] = first_of_chunk && ks == 0;
#pragma unroll
                for (int i = 0; i < NSLICE; ++i)
#pragma unroll
                    for (int j = 0; j < NSLICE; ++j) {
                        const int d = i + j;   // slices (i+1, j+1): order i + j + 2, accumulator d
                        mma_bf16(taddr + (uint32_t)(d * BN), sdesc(a0 + i * A_SL + off), sdesc(b0 + j * B_SL + off),
                                 fresh[d] ? 0u : 1u);
                        fresh[d] = false;
                    }
            }
            commit(&bar[st]);
        }
        ++issued[st];
        if (sl + 1 < nslab) prefetch(sl + 1);
        if (last_of_chunk) {
            // every MMA of the chunk (tracked by this stage's commit) must finish before TMEM is read
            if (!bwait(&bar[st], (uint32_t)((issued[st] - 1) & 1))) {
                if (tid == 0) raise_err(err, kDevTimeout);
                s_fail = 1;
            }
            __syncthreads();
            if (s_fail) { ok = false; break; }
            drain();
            __syncthreads();
        }
    }
    if (!ok) {
        for (int st = 0; st < 2; ++st)
            if (issued[st] > 0) bwait(&bar[st], (uint32_t)((issued[st] - 1) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(taddr));
    }
    if (!ok) return;
    const int m = m0 + (warp & 3) * 32 + lane;
    if (m >= g.M) return;
    const int em = g.ea[m];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const int n = n0 + (warp >> 2) * 32 + j;
        if (n < g.N) {
            const double v = ldexp((double)acc_i[j] + (double)acc_s[j], em + g.eb[n] - 14);
            const double val = g.alpha * v;
            const long long nc = g.n_idx_c ? g.n_idx_c[n] : n;
            double *cp = g.C + (long long)m * g.ldc + nc;
            if (g.atomic) atomicAdd(cp, val);
            else *cp = val + (g.beta != 0.0 ? g.beta * *cp : 0.0);
        }
    }
}

// Row / column scales of every problem: ea[m] = smallest e with max_k |A(m,k)| <= 2^e (0 for a zero row), and
// eb[n] likewise over B(k, n).  One CTA per problem; a warp per row when the row is contiguous, else a thread.
__device__ __forceinline__ int scale_exp(double mx) {
    if (!(mx > 0.0)) return 0;
    int e;
    const double f = frexp(mx, &e);   // mx = f 2^e, f in [0.5, 1)
    (void)f;
    return e;
}

__global__ void __launch_bounds__(256) k_gemm_scales(const GemmDesc *__restrict__ descs) {
    const GemmDesc g = descs[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // A rows
    if (g.transA == 0) {
        for (int m = wid; m < g.M; m += 8) {
            const double *row = g.A + (long long)(g.a_rows ? g.a_rows[m] : m) * g.lda;
            double mx = 0.0;
            for (int k = lane; k < g.K; k += 32) mx = fmax(mx, fabs(row[g.k_idx_a ? g.k_idx_a[k] : k]));
            mx = warp_max(mx);
            if (lane == 0) g.ea[m] = scale_exp(mx);
        }
    } else {
        for (int m = tid; m < g.M; m += 256) {
            double mx = 0.0;
            for (int k = 0; k < g.K; ++k) mx = fmax(mx, fabs(g.A[(long long)(g.k_idx_a ? g.k_idx_a[k] : k) * g.lda + m]));
            g.ea[m] = scale_exp(mx);
        }
    }
    // B columns
    if (g.transB == 1) {
        for (int n = wid; n < g.N; n += 8) {
            const double *row = g.B + (long long)(g.n_idx_b ? g.n_idx_b[n] : n) * g.ldb;
            double mx = 0.0;
            for (int k = lane; k < g.K; k += 32) mx = fmax(mx, fabs(row[g.k_idx_b ? g.k_idx_b[k] : k]));
            mx = warp_max(mx);
            if (lane == 0) g.eb[n] = scale_exp(mx);
        }
    } else {
        for (int n = tid; n < g.N; n += 256) {
            const long long nc = g.n_idx_b ? g.n_idx_b[n] : n;
            double mx = 0.0;
            for (int k = 0; k < g.K; ++k) mx = fmax(mx, fabs(g.B[(long long)(g.k_idx_b ? g.k_idx_b[k] : k) * g.ldb + nc]));
            g.eb[n] = scale_exp(mx);
        }
    }
}

}  // namespace

cudaError_t bf16x4_batch_prepare(GemmBatch &b, TcTiles &tt) {
    tc_tiles_free(tt);
    if (b.h.empty()) return cudaSuccess;
    // exponent scratch: M + N ints per problem, then re-upload the descriptors with the pointers set
    long long tot = 0;
    for (const GemmDesc &g : b.h) tot += (long long)g.M + g.N;
    cudaError_t e = cudaMalloc(&tt.d_exps, (size_t)std::max<long long>(tot, 1) * sizeof(int));
    if (e != cudaSuccess) return e;
    std::vector<GemmDesc> h = b.h;
    long long off = 0;
    std::vector<long long> t0(h.size() + 1, 0);
    for (size_t i = 0; i < h.size(); ++i) {
        h[i].ea = tt.d_exps + off;
        off += h[i].M;
        h[i].eb = tt.d_exps + off;
        off += h[i].N;
        const long long tiles = (h[i].M > 0 && h[i].N > 0) ? (long long)((h[i].M + BM - 1) / BM) * ((h[i].N + BN - 1) / BN) : 0;
        t0[i + 1] = t0[i] + tiles;
    }
    tt.tiles = t0.back();
    if ((e = cudaMalloc(&tt.d_desc, h.size() * sizeof(GemmDesc))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(tt.d_desc, h.data(), h.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    tt.nprob = (int)h.size();
    if ((e = cudaMalloc(&tt.d_tile0, t0.size() * sizeof(long long))) != cudaSuccess) return e;
    return cudaMemcpy(tt.d_tile0, t0.data(), t0.size() * sizeof(long long), cudaMemcpyHostToDevice);
}

cudaError_t bf16x4_batch_run(const TcTiles &tt, int *err, cudaStream_t s) {
    if (tt.tiles == 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16x4, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    count_launch();
    k_gemm_scales<<<tt.nprob, 256, 0, s>>>(tt.d_desc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_launch();
    k_gemm_bf16x4<<<(unsigned)tt.tiles, NT, SMEM, s>>>(tt.d_desc, tt.d_tile0, tt.nprob, err);
    return cudaGetLastError();
}

}  // namespace osv
