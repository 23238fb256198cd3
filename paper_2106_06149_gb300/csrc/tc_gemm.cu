// Grouped GEMM on the 5th-generation tensor cores (tcgen05, sm_103a) in split TF32 ("TF32x3"):
//   a = a_hi + a_lo with a_hi = tf32(a), a_lo = tf32(a - a_hi);  A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi,
// FP32 accumulation in tensor memory.  Same descriptors (GemmDesc) and semantics as the FP64 grouped GEMM, so a
// batch runs on either.
//
// One CTA = 256 threads = one 128 x 128 output tile, accumulated over the whole K in TMEM (128 columns).  K is
// consumed in slabs of 32.  The next slab is prefetched into registers (global loads in flight) while the
// tensor core works on the current one; each slab is converted to FP32, split into TF32 hi/lo and stored in
// shared memory in the canonical no-swizzle K-major layout (8-row x 16-byte core matrices), double-buffered.
// Thread 0 issues 4 k-steps x 3 products of tcgen05.mma.kind::tf32 (M = 128, N = 128, K = 8) and commits to
// the stage's mbarrier.  The epilogue drains TMEM with tcgen05.ld (warps 0-3: columns 0-63, warps 4-7:
// 64-127).  Every mbarrier wait is bounded by a clock budget; on expiry the kernel sets an error word, waits
// (bounded) for its own MMAs, frees TMEM and returns.
#include <cstdint>

#include "kernels.cuh"
#include "tc_gemm.h"

namespace osv {

namespace {

constexpr int TBM = 128, TBN = 128, TBK = 32, TNT = 256;
constexpr int A_BYTES = TBM * TBK * 4;       // 16 KB per split
constexpr int B_BYTES = TBN * TBK * 4;       // 16 KB per split
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 1024;   // + alignment slack
constexpr int PER_T = TBM * TBK / TNT;               // A (and B) elements per thread per slab = 16
constexpr long long kWaitBudget = 4LL << 30;         // clock cycles (~2 s at 2 GHz)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// canonical K-major, no swizzle: core matrix = 8 rows x 16 bytes; LBO (K direction) = 128 B, SBO (rows) = 1024 B
__device__ __forceinline__ uint32_t kmajor_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;    // leading (K) byte offset between core matrices
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;   // stride (M/N) byte offset between 8-row groups
    d |= (uint64_t)1 << 46;                          // descriptor version
    return d;                                        // base offset 0, swizzle none
}

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, N = 128, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TBN >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long budget) {
    const long long t0 = clock64();
    uint32_t done = 0;
    while (true) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > budget) return false;
    }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Element e of a 128 x 32 slab: lane = e % 32 picks (row % 8, k % 4) so that a warp's 32 shared-memory stores
// land in 32 distinct banks of the core-matrix layout; e / 32 picks the 8-row group and the 4-wide k group.
__device__ __forceinline__ void slab_coord(int e, int &r, int &k) {
    const int lane = e & 31, grp = e >> 5;
    r = ((grp >> 3) << 3) + (lane >> 2);
    k = ((grp & 7) << 2) + (lane & 3);
}

__global__ void __launch_bounds__(TNT, 1) k_gemm_tf32x3(const GemmDesc *__restrict__ descs,
                                                       const long long *__restrict__ tile0, int nprob, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bar_stage[2];
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
    const int tiles_n = (g.N + TBN - 1) / TBN;
    const int m0 = int(local / tiles_n) * TBM, n0 = int(local % tiles_n) * TBN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_stage[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_stage[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&s_taddr)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = s_taddr;

    const int nslab = (g.K + TBK - 1) / TBK;
    double ra[PER_T], rb[PER_T];
    auto prefetch = [&](int sl) {
        const int k0 = sl * TBK;
#pragma unroll
        for (int i = 0; i < PER_T; ++i) {
            int r, k;
            slab_coord(tid + i * TNT, r, k);
            const int m = m0 + r, kk = k0 + k;
            double v = 0.0;
            if (m < g.M && kk < g.K) {
                const long long kc = g.k_idx_a ? g.k_idx_a[kk] : kk;
                v = g.transA == 0 ? g.A[(long long)(g.a_rows ? g.a_rows[m] : m) * g.lda + kc] : g.A[kc * g.lda + m];
            }
            ra[i] = v;
        }
#pragma unroll
        for (int i = 0; i < PER_T; ++i) {
            int nn, k;
            slab_coord(tid + i * TNT, nn, k);
            const int n = n0 + nn, kk = k0 + k;
            double v = 0.0;
            if (n < g.N && kk < g.K) {
                const long long kr = g.k_idx_b ? g.k_idx_b[kk] : kk;
                const long long nc = g.n_idx_b ? g.n_idx_b[n] : n;
                v = g.transB == 0 ? g.B[kr * g.ldb + nc] : g.B[nc * g.ldb + kr];
            }
            rb[i] = v;
        }
    };

    int issued[2] = {0, 0};
    bool ok = true;
    if (nslab > 0) prefetch(0);
    for (int sl = 0; sl < nslab; ++sl) {
        const int st = sl & 1;
        if (sl >= 2) {
            // the MMAs that read this stage two slabs ago must be done before it is overwritten
            if (!mbar_wait(&bar_stage[st], (uint32_t)(((sl >> 1) - 1) & 1), kWaitBudget)) {
                if (tid == 0) raise_err(err, kDevTimeout);
                s_fail = 1;
            }
        }
        unsigned char *sA = smem + st * STAGE_BYTES;
        unsigned char *sAl = sA + A_BYTES, *sB = sA + 2 * A_BYTES, *sBl = sB + B_BYTES;
#pragma unroll
        for (int i = 0; i < PER_T; ++i) {
            int r, k;
            slab_coord(tid + i * TNT, r, k);
            const float x = (float)ra[i];
            const uint32_t h = tf32_bits(x);
            const uint32_t o = kmajor_off(r, k);
            *(uint32_t *)(sA + o) = h;
            *(uint32_t *)(sAl + o) = tf32_bits(x - __uint_as_float(h));
        }
#pragma unroll
        for (int i = 0; i < PER_T; ++i) {
            int nn, k;
            slab_coord(tid + i * TNT, nn, k);
            const float x = (float)rb[i];
            const uint32_t h = tf32_bits(x);
            const uint32_t o = kmajor_off(nn, k);
            *(uint32_t *)(sB + o) = h;
            *(uint32_t *)(sBl + o) = tf32_bits(x - __uint_as_float(h));
        }
        // generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (s_fail) { ok = false; break; }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t aH = smem_u32(sA), aL = smem_u32(sAl), bH = smem_u32(sB), bL = smem_u32(sBl);
#pragma unroll
            for (int ks = 0; ks < TBK / 8; ++ks) {
                const uint32_t off = ks * 256;   // two core matrices along K per k-step
                mma_tf32(taddr, smem_desc(aH + off), smem_desc(bH + off), (sl > 0 || ks > 0) ? 1u : 0u);
                mma_tf32(taddr, smem_desc(aH + off), smem_desc(bL + off), 1u);
                mma_tf32(taddr, smem_desc(aL + off), smem_desc(bH + off), 1u);
            }
            mma_commit(&bar_stage[st]);
        }
        ++issued[st];
        if (sl + 1 < nslab) prefetch(sl + 1);   // global loads overlap the tensor-core work
    }
    // wait for the last slab's MMAs (tcgen05.commit covers every earlier MMA of this thread)
    if (ok && nslab > 0) {
        const int st = (nslab - 1) & 1;
        if (!mbar_wait(&bar_stage[st], (uint32_t)((issued[st] - 1) & 1), kWaitBudget)) {
            if (tid == 0) raise_err(err, kDevTimeout);
            ok = false;
        }
    }
    if (!ok) {
        for (int st = 0; st < 2; ++st)
            if (issued[st] > 0) mbar_wait(&bar_stage[st], (uint32_t)((issued[st] - 1) & 1), kWaitBudget);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: warp w drains TMEM lanes 32 (w % 4) .. (its tile rows), columns 64 (w / 4) .. + 63
    const int row = (warp & 3) * 32 + lane;
    const int cbase = (warp >> 2) * 64;
    const int m = m0 + row;
    if (ok) {
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            if (nslab > 0) {
                tmem_ld16(taddr + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(cbase + c), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.f;
            }
            if (m < g.M) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int n = n0 + cbase + c + i;
                    if (n < g.N) {
                        const double val = g.alpha * (double)v[i];
                        const long long nc = g.n_idx_c ? g.n_idx_c[n] : n;
                        double *cp = g.C + (long long)m * g.ldc + nc;
                        if (g.atomic) atomicAdd(cp, val);
                        else *cp = val + (g.beta != 0.0 ? g.beta * *cp : 0.0);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(taddr));
    }
}

}  // namespace

cudaError_t tc_batch_prepare(GemmBatch &b, TcTiles &tt) {
    tc_tiles_free(tt);
    if (b.h.empty()) return cudaSuccess;
    std::vector<long long> t0(b.h.size() + 1, 0);
    for (size_t i = 0; i < b.h.size(); ++i) {
        const GemmDesc &g = b.h[i];
        const long long tiles = (g.M > 0 && g.N > 0) ? (long long)((g.M + TBM - 1) / TBM) * ((g.N + TBN - 1) / TBN) : 0;
        t0[i + 1] = t0[i] + tiles;
    }
    tt.tiles = t0.back();
    cudaError_t e = cudaMalloc(&tt.d_tile0, t0.size() * sizeof(long long));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(tt.d_tile0, t0.data(), t0.size() * sizeof(long long), cudaMemcpyHostToDevice);
}

cudaError_t tc_batch_run(const GemmBatch &b, const TcTiles &tt, int *err, cudaStream_t s) {
    if (tt.tiles == 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    count_launch();
    k_gemm_tf32x3<<<(unsigned)tt.tiles, TNT, SMEM_BYTES, s>>>(b.d_desc, tt.d_tile0, (int)b.h.size(), err);
    return cudaGetLastError();
}

void tc_tiles_free(TcTiles &tt) {
    if (tt.d_tile0) cudaFree(tt.d_tile0);
    if (tt.d_desc) cudaFree(tt.d_desc);
    if (tt.d_exps) cudaFree(tt.d_exps);
    if (tt.d_jobs) cudaFree(tt.d_jobs);
    if (tt.d_otiles) cudaFree(tt.d_otiles);
    if (tt.d_rows) cudaFree(tt.d_rows);
    if (tt.d_sjobs0) cudaFree(tt.d_sjobs0);
    if (tt.d_ops) cudaFree(tt.d_ops);
    tt = TcTiles{};
}

}  // namespace osv
