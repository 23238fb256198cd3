// Grouped GEMM on tcgen05 tensor cores with exactly accumulated BF16 slices of pre-sliced operands.
//
// Each operand row (A: row m over k; B: column n over k) gets a power-of-two scale 2^e with every |element| <=
// 2^e.  An FP64 element x is rounded (integer arithmetic on its bit pattern, round half away from zero) to
// N = round(x 2^(31-e)), |N| <= 2^31, and N is cut into four signed base-256 digits
//   N = s0 2^24 + s1 2^16 + s2 2^8 + s3,   |s_i| <= 128  (exact BF16 values).
// Slice i is stored as s_i 2^(-8 i) (still exact in BF16), so the product of slices i and j carries its weight
// 2^(-8 (i + j)) and the tensor core sums the products of one order class directly.  Over a chunk of 256 K:
//   acc0: i + j = 0      integers, |sum| <= 2^22: exact in FP32;
//   acc1: i + j = 1      multiples of 2^-8, |sum| <= 2^15: exact;
//   acc2: i + j = 2      multiples of 2^-16, |sum| < 2^8: exact;
//   acc3: i + j = 3, 4   (7 products) rounded in FP32 (the tensor core may truncate): an error of a few 2^-24 of
//                        a term that is itself <= 2^-24 of the result, so below 2^-40 relative even if biased.
// Products with i + j >= 5 (weight <= 2^-40) are not formed.  After each chunk the accumulators are drained
// into double-float register pairs (hi, lo): acc0..acc2 by an error-free two-sum, acc3 (at most 2^-20 of the
// scale) added to the low word, a rounding below 2^-43 of the scale per chunk.  The epilogue restores
// 2^(e_m + e_n - 14).
//
// Two kernels per batch: (1) the row scales, then every operand tile (128 rows x 16 K) is sliced once into four
// 4 KB images already in the canonical no-swizzle K-major shared-memory layout (8 rows x 16 bytes per core
// matrix; K-adjacent core matrices 128 B apart, 8-row groups 256 B apart), two tiles per slicing job; (2) the
// GEMM: one CTA (256 threads) per 128 x 128 output tile, a six-stage pipeline of 32 KB stages filled by four
// producer warps with 16-byte asynchronous copies (completion counted per thread on the stage's mbarrier; five
// stages in flight), thread 0 issuing 13 tcgen05.mma.kind::f16 (M = 128, N = 128, K = 16) per stage into four
// TMEM accumulators (512 columns), and rows of the result leaving by bulk stores or bulk add-reductions.  Every
// wait is bounded: on expiry the error word is set, in-flight MMAs are waited for (bounded), TMEM is freed and
// the CTA returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>
#include <cstdint>

#include "kernels.cuh"
#include "oz_pack.h"
#include "tc_common.cuh"
#include "tc_gemm.h"

namespace osv {

namespace {

constexpr int BM = 128, BN = 128, BK = 16, NT = 256;
constexpr int SK = 32;                            // K extent of one slicing job: SK / BK image tiles
constexpr int NSLICE = 4;
constexpr int IMG = BM * BK * 2;                  // 4 KB: one slice of one 128 x 16 tile
constexpr int TILE_BYTES = NSLICE * IMG;          // 16 KB: the four slices of one operand tile
constexpr int STAGE = 2 * TILE_BYTES;             // A and B
constexpr int NSTAGE = 6;                         // five stages of copies in flight ahead of the MMAs
constexpr int kProducers = 128;                   // copy threads (warps 4..7)
constexpr int SMEM = NSTAGE * STAGE + 1024;
constexpr int CHUNK_KT = 256 / BK;                // 256 K per exact chunk
constexpr int KT_PER_JOB = SK / BK;
// image tiles per operand row tile: whole slicing jobs (the padding tile, if any, holds zeros)
__host__ __device__ constexpr int padded_nkt(int K) { return ((K + SK - 1) / SK) * KT_PER_JOB; }
constexpr uint32_t kIdesc = idesc_bf16(BM, BN);

__device__ __forceinline__ uint32_t koff(int r, int k) { return kmajor_off(r, k, BK); }
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) { return smem_desc(saddr, 16 * BK); }
constexpr int NACC = 4;


__device__ __forceinline__ int find_prob(const long long *__restrict__ pre, int nprob, long long t) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One GEMM operand as the slicing passes see it: R rows over K, element (r, k) = ptr[row(r) ld + kk(k)] when the
// rows are K-contiguous (A, transA = 0; B, transB = 1), ptr[kk(k) ld + row(r)] otherwise, with optional row and
// K index maps.  Problems that read the same operand (same pointer, layout, maps and sizes) share one entry: its
// row scales and slice images are computed once per batch.  An A operand read only by row-packed problems gets its
// scales but no images of its own (its rows are sliced into the packed tiles).
struct OzOperand {
    const double *ptr;
    long long ld;
    const int *rowmap, *kmap;
    int R, K, kcontig;
    int *exps;         // row scale exponents (R)
    long long soff;    // byte offset of its slice images in the scratch (-1: not sliced on its own)
};

// Row scales: exps[r] = e with max_k |X(r,k)| = f 2^e, f in [0.5, 1) (0 for a zero row).  One CTA per block of
// 32 operand rows.  K-contiguous rows: a warp per row; otherwise the 32 lanes take 32 adjacent rows and the
// eight warps split K.
constexpr int SROWS = 32;
__global__ void __launch_bounds__(256) k_oz_scales(const OzOperand *__restrict__ ops, const long long *__restrict__ sj0,
                                                   int nops) {
    __shared__ unsigned long long part[8][SROWS];
    const long long t = blockIdx.x;
    const int p = find_prob(sj0, nops, t);
    const OzOperand o = ops[p];
    const int r0 = (int)(t - sj0[p]) * SROWS;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (o.kcontig) {
        for (int r = wid; r < SROWS; r += 8) {
            const int rr = r0 + r;
            if (rr >= o.R) break;
            const double *row = o.ptr + (long long)(o.rowmap ? o.rowmap[rr] : rr) * o.ld;
            unsigned long long mx = 0ULL;
            for (int k = lane; k < o.K; k += 32) {
                const unsigned long long b = abs_bits64(row[o.kmap ? o.kmap[k] : k]);
                mx = b > mx ? b : mx;
            }
            mx = warp_max_bits(mx);
            if (lane == 0) o.exps[rr] = scale_exp_of_bits(mx);
        }
        return;
    }
    const int rr = r0 + lane;
    unsigned long long mx = 0ULL;
    if (rr < o.R) {
        const double *base = o.ptr + (o.rowmap ? o.rowmap[rr] : rr);
        for (int k = wid; k < o.K; k += 8) {
            const unsigned long long b = abs_bits64(base[(long long)(o.kmap ? o.kmap[k] : k) * o.ld]);
            mx = b > mx ? b : mx;
        }
    }
    part[wid][lane] = mx;
    __syncthreads();
    if (wid == 0 && rr < o.R) {
        for (int w = 1; w < 8; ++w) mx = part[w][lane] > mx ? part[w][lane] : mx;
        o.exps[rr] = scale_exp_of_bits(mx);
    }
}

// Output tile of the GEMM kernel: byte offsets of the first k tile of its A and B slice images, the problem and
// tile origin, its k-tile count, and for a packed tile (rt >= 0) the row table naming each row's problem.
struct OzTile {
    long long aoff, boff;
    int p, m0, n0, nkt, rt;
};
// Row r of a packed tile: problem p (-1: empty row), its A operand q and the row m of that problem.
struct OzRow {
    int p, q, m;
};
// Slicing job: the 128 x 32 block kt (two 16-K image tiles) of operand q, row tile rt (packed < 0), or of packed
// tile `packed`.
struct OzJob {
    long long dst;
    int q, rt, kt, packed;
};

// One CTA per slicing job: stage the FP64 values in shared memory (coalesced for either orientation of the
// rows' operand), then write the four slice images.  Rows are addressed through per-row (base, k stride, k map)
// triples, so a packed tile gathers the rows of several problems.
__global__ void __launch_bounds__(NT) k_oz_slice(const OzOperand *__restrict__ ops, const OzJob *__restrict__ jobs,
                                                 const OzRow *__restrict__ rows, unsigned char *__restrict__ scratch) {
    __shared__ double xs[SK][BM + 1];
    __shared__ int es[BM], kn[BM];
    __shared__ const double *rbase[BM];
    __shared__ const int *rkmap[BM];
    __shared__ long long rks[BM];
    __shared__ int s_along_k;
    const OzJob J = jobs[blockIdx.x];
    const int k0 = J.kt * SK;
    const int tid = threadIdx.x;
    for (int r = tid; r < BM; r += NT) {
        int q = -1, m = 0;
        if (J.packed < 0) {
            q = J.q;
            m = J.rt * BM + r;
            if (m >= ops[q].R) q = -1;
        } else {
            const OzRow x = rows[(long long)J.packed * BM + r];
            if (x.p >= 0) { q = x.q; m = x.m; }
        }
        if (q >= 0) {
            const OzOperand &o = ops[q];
            const long long rr = o.rowmap ? o.rowmap[m] : m;
            rbase[r] = o.kcontig ? o.ptr + rr * o.ld : o.ptr + rr;
            rks[r] = o.kcontig ? 1 : o.ld;
            rkmap[r] = o.kmap;
            kn[r] = o.K;
            es[r] = o.exps[m];
        } else {
            rbase[r] = nullptr;
            rks[r] = 0;
            rkmap[r] = nullptr;
            kn[r] = 0;
            es[r] = 0;
        }
        if (r == 0) s_along_k = q >= 0 ? ops[q].kcontig : 1;
    }
    __syncthreads();
    // all of a thread's element addresses first, then all its loads, then the shared-memory stores: sixteen
    // loads in flight per thread instead of one (the loop with a load, a store and a branch per element was
    // latency-bound)
    constexpr int PER = BM * SK / NT;
    const bool along_k = s_along_k;
    const double *src[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int idx = tid + q * NT;
        const int r = along_k ? idx / SK : idx % BM, k = along_k ? idx % SK : idx / BM;
        const int kk = k0 + k;
        const int *km = rkmap[r];
        src[q] = kk < kn[r] ? rbase[r] + (km ? (long long)km[kk] : (long long)kk) * rks[r] : nullptr;
    }
    double val[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) val[q] = src[q] ? __ldg(src[q]) : 0.0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int idx = tid + q * NT;
        const int r = along_k ? idx / SK : idx % BM, k = along_k ? idx % SK : idx / BM;
        xs[k][r] = val[q];
    }
    __syncthreads();
    unsigned char *img = scratch + J.dst;
    for (int c = tid; c < BM * (SK / 8); c += NT) {   // one core-matrix row (8 K of one row) per step
        const int r = c % BM, kg = c / BM;
        const int sub = kg / (BK / 8), kgl = kg % (BK / 8);   // image tile of the job, 8-K group inside it
        float sl[8][NSLICE];
#pragma unroll
        for (int q = 0; q < 8; ++q) slice4_exact(xs[kg * 8 + q][r], es[r], sl[q]);
        const uint32_t off = (uint32_t)sub * TILE_BYTES + koff(r, kgl * 8);
#pragma unroll
        for (int i = 0; i < NSLICE; ++i) {
            __nv_bfloat162 h[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn(sl[2 * q][i], sl[2 * q + 1][i]);
            *reinterpret_cast<uint4 *>(img + i * IMG + off) = *reinterpret_cast<uint4 *>(h);
        }
    }
}

__global__ void __launch_bounds__(NT, 1) k_oz_gemm(const GemmDesc *__restrict__ descs, const OzTile *__restrict__ tiles,
                                                  const OzRow *__restrict__ rows,
                                                  const unsigned char *__restrict__ scratch, int *err, long long budget) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[NSTAGE], empty[NSTAGE], dbar;
    __shared__ uint32_t s_taddr;
    __shared__ int s_fail, s_issued;

    const OzTile T = tiles[blockIdx.x];
    const int m0 = T.m0, n0 = T.n0, nkt = T.nkt;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned char *Aimg = scratch + T.aoff;
    const unsigned char *Bimg = scratch + T.boff;

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(kProducers));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&dbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
        s_issued = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&s_taddr)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = s_taddr;

    // drain targets: TMEM lanes of warp % 4 (rows), columns 64 * (warp / 4) .. + 63.  The chunk sums are added
    // into FP32 double-float pairs (hi, lo) on the FP32 ALU only (an FP64 add runs at 1/64 of the FP32 rate on
    // this part and made the drain the bottleneck); well beyond the ~31 significant bits of the products.
    float chi[64], clo[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) {
        chi[j] = 0.f;
        clo[j] = 0.f;
    }

    // Roles: warps 4..7 copy k tile j into stage j % NSTAGE (16-byte asynchronous copies, 16 per thread, each
    // thread's completion counted on the stage's mbarrier) as soon as the MMAs of tile j - NSTAGE are done; thread
    // 0 waits for each tile's data and issues its MMAs, and never waits for MMA completion inside a chunk.  All
    // threads drain the accumulators after each 256-K chunk; the copies of the next chunk's first stages are in
    // flight meanwhile.
    volatile int *fail = &s_fail;
    int loaded = 0;   // k tiles whose copies were issued (producer threads)
    int issued = 0;   // MMA groups committed (thread 0)
    const int ptid = tid - (NT - kProducers);   // producer index, or negative
    auto load_stage = [&](int kt) {
        const int st = kt % NSTAGE;
        ++loaded;
        const uint32_t dst = smem_u32(smem + st * STAGE);
        const unsigned char *srcA = Aimg + (long long)kt * TILE_BYTES, *srcB = Bimg + (long long)kt * TILE_BYTES;
#pragma unroll
        for (int q = 0; q < STAGE / 16 / kProducers; ++q) {
            const int ch = ptid + q * kProducers;   // 16-byte chunk of the stage: A images, then B images
            const unsigned char *src = ch < TILE_BYTES / 16 ? srcA + ch * 16 : srcB + (ch - TILE_BYTES / 16) * 16;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + ch * 16), "l"(src) : "memory");
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[st])) : "memory");
    };
    bool ok = true;
    const int nchunk = (nkt + CHUNK_KT - 1) / CHUNK_KT;
    for (int chunk = 0; chunk < nchunk; ++chunk) {
        const int kt0 = chunk * CHUNK_KT, kt1 = min(nkt, kt0 + CHUNK_KT);
        if (ptid >= 0) {
            const int jend = min(nkt, kt1 + NSTAGE - 1);
            while (loaded < jend && !*fail) {
                const int j = loaded;
                if (j >= NSTAGE && !tc_wait(&empty[j % NSTAGE], (uint32_t)((j / NSTAGE - 1) & 1), budget)) {
                    raise_err(err, kDevTimeout);
                    *fail = 1;
                    break;
                }
                load_stage(j);
            }
        } else if (tid == 0) {
            for (int kt = kt0; kt < kt1 && !*fail; ++kt) {
                const int st = kt % NSTAGE;
                if (!tc_wait(&full[st], (uint32_t)((kt / NSTAGE) & 1), budget)) {
                    raise_err(err, kDevTimeout);
                    *fail = 1;
                    break;
                }
                // the stage was written through the generic proxy: order it before the tensor core's reads
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::after_thread_sync;");
                // descriptors of the stage's images: the start-address field (address / 16, 14 bits) of the base
                // descriptor plus the image offset / 16 (no carry: shared addresses are below 256 KB)
                const uint64_t da = sdesc(smem_u32(smem + st * STAGE)), db = da + (uint64_t)(TILE_BYTES >> 4);
                const bool first = kt == kt0;
#pragma unroll
                for (int ks = 0; ks < BK / 16; ++ks) {
                    const uint32_t off = ks * 256;
                    bool fresh[NACC];
#pragma unroll
                    for (int a = 0; a < NACC; ++a) fresh[a] = first && ks == 0;
#pragma unroll
                    for (int i = 0; i < NSLICE; ++i)
#pragma unroll
                        for (int j = 0; j < NSLICE; ++j) {
                            const int d = i + j;
                            if (d > 4) continue;
                            const int a = d < 3 ? d : 3;
                            tc_mma_bf16(taddr + (uint32_t)(a * BN), da + (uint64_t)((i * IMG + off) >> 4),
                                        db + (uint64_t)((j * IMG + off) >> 4), kIdesc, !fresh[a]);
                            fresh[a] = false;
                        }
                }
                tc_commit(&empty[st]);
                ++issued;
            }
            s_issued = issued;
            if (!*fail) tc_commit(&dbar);
        }
        __syncthreads();
        if (*fail) { ok = false; break; }
        if (!tc_wait(&dbar, (uint32_t)(chunk & 1), budget)) {
            raise_err(err, kDevTimeout);
            *fail = 1;
        }
        __syncthreads();
        if (*fail) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t lbase = taddr + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 64);
#pragma unroll
        for (int a = 0; a < NACC; ++a)
#pragma unroll
            for (int c = 0; c < 64; c += 32) {
                float v0[16], v1[16];
                tc_ld16(lbase + a * BN + c, v0);
                tc_ld16(lbase + a * BN + c + 16, v1);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (a < 3) {   // acc0..acc2: error-free two-sum into (hi, lo)
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        two_sum_f32(chi[c + i], clo[c + i], v0[i]);
                        two_sum_f32(chi[c + 16 + i], clo[c + 16 + i], v1[i]);
                    }
                } else {       // acc3 (below 2^-20 of the scale): into the low word
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        clo[c + i] = __fadd_rn(clo[c + i], v0[i]);
                        clo[c + 16 + i] = __fadd_rn(clo[c + 16 + i], v1[i]);
                    }
                }
            }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    if (ptid >= 0) asm volatile("cp.async.wait_all;" ::: "memory");   // every copy of this thread has landed
    if (!ok && tid == 0) {
        // let every committed MMA group finish before TMEM is released (bounded)
        const int iss = s_issued;
        for (int s = 0; s < NSTAGE; ++s) {
            const int uses = iss / NSTAGE + (s < iss % NSTAGE ? 1 : 0);
            if (uses > 0) tc_wait(&empty[s], (uint32_t)((uses - 1) & 1));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(taddr));
    }
    if (!ok) return;
    // Epilogue.  The per-row destinations (the tile's own problem, or a packed tile's row table) and the per-column
    // scale exponents are fetched first, one load per thread, so that the element loop reads shared memory only
    // (a chain of dependent global loads per row made this phase longer than the main loop).  The (hi, lo) sums
    // then pass through shared memory (the stage buffers are idle), are converted there in place, and rows leave
    // as wholes.  alpha = +-2^k folds into the exponent; the FP64 value is assembled with integer operations
    // (df_to_double_nb).
    __shared__ double *s_crow[BM];
    __shared__ const int *s_nmap[BM];
    __shared__ double s_alpha[BM], s_beta[BM];
    __shared__ int s_em[BM], s_rf[BM], s_eb[BN];
    if (tid < BM) {
        const int r = tid;
        int p = T.p, m = m0 + r;
        bool valid;
        if (T.rt >= 0) {
            const OzRow x = rows[(long long)T.rt * BM + r];
            valid = x.p >= 0;
            p = x.p;
            m = x.m;
        } else {
            valid = m < descs[p].M;
        }
        s_crow[r] = nullptr;
        s_em[r] = 0;
        s_rf[r] = 0;
        s_alpha[r] = 1.0;
        s_beta[r] = 0.0;
        s_nmap[r] = nullptr;
        if (valid) {
            const GemmDesc &g = descs[p];
            const double alpha = g.alpha;
            const unsigned long long abits = (unsigned long long)__double_as_longlong(alpha);
            const int aexp = (int)((abits >> 52) & 0x7FF);
            const bool alpha_p2 = (abits & 0xFFFFFFFFFFFFFULL) == 0 && aexp > 0 && aexp < 0x7FF;
            s_em[r] = g.ea[m] - 14 + (alpha_p2 ? aexp - 1023 : 0);
            s_rf[r] = (g.atomic ? 1 : 0) | (alpha_p2 ? 2 : 0) | ((alpha_p2 && (abits >> 63)) ? 4 : 0);
            s_alpha[r] = alpha;
            s_beta[r] = g.beta;
            s_nmap[r] = g.n_idx_c;
            s_crow[r] = g.C + (long long)m * g.ldc;
        }
    } else if (tid < BM + BN) {
        const int c = tid - BM, n = n0 + c;
        const GemmDesc &g0 = descs[T.p];   // every row of the tile reads the same B operand
        s_eb[c] = n < g0.N ? g0.eb[n] : 0;
    }
    // row stride of 130 elements: every row starts on a 16-byte boundary (bulk copies below)
    float2 *sC = reinterpret_cast<float2 *>(smem);
    double *sD = reinterpret_cast<double *>(smem);   // the same storage after the in-place conversion
    constexpr int LDC = BN + 2;
    {
        const int r = (warp & 3) * 32 + lane;
#pragma unroll
        for (int j = 0; j < 64; ++j) sC[r * LDC + (warp >> 2) * 64 + j] = make_float2(chi[j], clo[j]);
    }
    __syncthreads();   // the (hi, lo) tile, row constants and column exponents in shared memory
    const int N = descs[T.p].N;
    const int nvalid = max(0, min(BN, N - n0));
    // (hi, lo) -> alpha times the FP64 value, in place (each element read and written by the same thread)
    for (int r = warp; r < BM; r += NT / 32) {
        if (!s_crow[r]) continue;
        const int em = s_em[r], rf = s_rf[r];
        const double alpha = s_alpha[r];
        const long long asign = (rf & 4) ? (long long)0x8000000000000000ULL : 0LL;
        // the lane's four conversions branch-free (they interleave), then the rare special cases
        constexpr int CU = BN / 32;
        double v[CU];
        bool sp[CU], any = false;
#pragma unroll
        for (int u = 0; u < CU; ++u) {
            const int c = lane + 32 * u;
            const float2 hl = sC[r * LDC + c];
            v[u] = df_to_double_nb(hl.x, hl.y, em + s_eb[c], sp[u]);
            sp[u] = sp[u] && c < nvalid;
            any |= sp[u];
        }
        if (any) {
#pragma unroll
            for (int u = 0; u < CU; ++u)
                if (sp[u]) {
                    const int c = lane + 32 * u;
                    const float2 hl = sC[r * LDC + c];
                    v[u] = df_to_double(hl.x, hl.y, em + s_eb[c]);
                }
        }
        if (rf & 2) {   // alpha = +-2^k, already in the exponent (uniform per row: no FP64 multiply issued)
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const int c = lane + 32 * u;
                if (c < nvalid) sD[r * LDC + c] = __longlong_as_double(__double_as_longlong(v[u]) ^ asign);
            }
        } else {
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const int c = lane + 32 * u;
                if (c < nvalid) sD[r * LDC + c] = v[u] * alpha;
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes -> bulk-copy reads
    __syncthreads();
    // rows with a contiguous, 16-byte aligned destination leave by one bulk copy each: a store (C = alpha AB) or
    // an element-wise atomic add (accumulating rows, and beta = 1); the others take the element path below
    __shared__ int s_slow[BM];
    bool issued_bulk = false;
    if (tid < BM) {
        const int r = tid;
        double *crow = s_crow[r];
        int slow = 0;
        if (crow && nvalid > 0) {
            const int rf = s_rf[r];
            const double beta = s_beta[r];
            double *dst = crow + n0;
            const uint32_t bytes = (uint32_t)nvalid * 8u;
            const bool fits = !s_nmap[r] && (bytes & 15u) == 0 && ((uintptr_t)dst & 15u) == 0;
            const bool store = !(rf & 1) && beta == 0.0, add = (rf & 1) || beta == 1.0;
            if (fits && (store || add)) {
                const uint32_t src = smem_u32(sD + r * LDC);
                if (store)
                    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src),
                                 "r"(bytes)
                                 : "memory");
                else
                    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;" ::"l"(dst),
                                 "r"(src), "r"(bytes)
                                 : "memory");
                issued_bulk = true;
            } else {
                slow = 1;
            }
        }
        s_slow[r] = slow;
        if (issued_bulk) asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    __syncthreads();
    for (int r = warp; r < BM; r += NT / 32) {
        if (!s_slow[r]) continue;
        double *crow = s_crow[r];
        const int rf = s_rf[r];
        const double beta = s_beta[r];
        const int *__restrict__ nmap = s_nmap[r];
        for (int c = lane; c < nvalid; c += 32) {
            const int n = n0 + c;
            const double v = sD[r * LDC + c];
            double *cp = crow + (nmap ? nmap[n] : n);
            if (rf & 1) atomicAdd(cp, v);
            else *cp = v + (beta != 0.0 ? beta * *cp : 0.0);
        }
    }
    // the bulk copies read shared memory until they complete: wait before the CTA exits
    if (issued_bulk) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

}  // namespace

void tc_tiles_free(TcTiles &tt) {
    for (TcTiles &p : tt.parts) tc_tiles_free(p);
    if (tt.d_desc) cudaFree(tt.d_desc);
    if (tt.d_exps) cudaFree(tt.d_exps);
    if (tt.d_jobs) cudaFree(tt.d_jobs);
    if (tt.d_otiles) cudaFree(tt.d_otiles);
    if (tt.d_rows) cudaFree(tt.d_rows);
    if (tt.d_sjobs0) cudaFree(tt.d_sjobs0);
    if (tt.d_ops) cudaFree(tt.d_ops);
    tt = TcTiles{};
}

namespace {

// One launch group: the problems h (a consecutive range of a batch), their operands, slicing jobs and tiles.
cudaError_t prepare_part(std::vector<GemmDesc> h, TcTiles &tt) {
    // distinct operands (A of every problem, B of every problem), identified by pointer, layout, maps and sizes
    struct Key {
        const double *ptr;
        long long ld;
        const int *rowmap, *kmap;
        int R, K, kcontig;
        bool operator<(const Key &o) const {
            return std::tie(ptr, ld, rowmap, kmap, R, K, kcontig) < std::tie(o.ptr, o.ld, o.rowmap, o.kmap, o.R, o.K, o.kcontig);
        }
    };
    std::map<Key, int> index;
    std::vector<OzOperand> ops;
    std::vector<int> opA(h.size(), -1), opB(h.size(), -1);
    auto add = [&](const Key &k) -> int {
        auto it = index.find(k);
        if (it != index.end()) return it->second;
        OzOperand o{};
        o.ptr = k.ptr;
        o.ld = k.ld;
        o.rowmap = k.rowmap;
        o.kmap = k.kmap;
        o.R = k.R;
        o.K = k.K;
        o.kcontig = k.kcontig;
        ops.push_back(o);
        index[k] = (int)ops.size() - 1;
        return (int)ops.size() - 1;
    };
    for (size_t i = 0; i < h.size(); ++i) {
        const GemmDesc &g = h[i];
        if (g.M <= 0 || g.N <= 0) continue;
        opA[i] = add(Key{g.A, g.lda, g.transA == 0 ? g.a_rows : nullptr, g.k_idx_a, g.M, g.K, g.transA == 0 ? 1 : 0});
        opB[i] = add(Key{g.B, g.ldb, g.n_idx_b, g.k_idx_b, g.N, g.K, g.transB == 1 ? 1 : 0});
    }
    // row packing (oz_pack.h): problems of fewer than BM rows that read the same B operand (hence the same K and N)
    // share BM-row tiles
    std::vector<int> packed_in(h.size(), -1);   // packed tile of each problem
    std::vector<std::vector<OzRow>> ptab;       // row tables
    std::vector<int> pB;                        // B operand of each packed tile
    {
        std::vector<int> rows(h.size());
        for (size_t i = 0; i < h.size(); ++i) rows[i] = opB[i] >= 0 ? h[i].M : 0;
        for (const OzPackTile &pt : oz_pack_rows(rows, opB, BM)) {
            const int t = (int)ptab.size();
            ptab.emplace_back(BM, OzRow{-1, -1, 0});
            pB.push_back(pt.key);
            for (const auto &mb : pt.members) {
                const int p = mb.first;
                packed_in[p] = t;
                for (int m = 0; m < h[p].M; ++m) ptab[t][mb.second + m] = OzRow{p, opA[p], m};
            }
        }
    }
    // operands that are sliced on their own: every B operand and the A operands of unpacked problems
    std::vector<char> sliced(ops.size(), 0);
    for (size_t i = 0; i < h.size(); ++i) {
        if (opB[i] < 0) continue;
        sliced[opB[i]] = 1;
        if (packed_in[i] < 0) sliced[opA[i]] = 1;
    }
    // scale arrays (all operands), slice images and jobs
    long long nexp = 0, bytes = 0;
    std::vector<long long> s0(ops.size() + 1, 0), eoff(ops.size());
    std::vector<OzJob> jobs;
    for (size_t q = 0; q < ops.size(); ++q) {
        OzOperand &o = ops[q];
        eoff[q] = nexp;
        nexp += o.R;
        s0[q + 1] = s0[q] + (o.R + SROWS - 1) / SROWS;
        o.soff = -1;
        if (!sliced[q]) continue;
        const int nkp = padded_nkt(o.K), rt = (o.R + BM - 1) / BM;
        o.soff = bytes;
        for (int r = 0; r < rt; ++r)
            for (int k = 0; k < nkp / KT_PER_JOB; ++k)
                jobs.push_back(OzJob{bytes + ((long long)r * nkp + k * KT_PER_JOB) * TILE_BYTES, (int)q, r, k, -1});
        bytes += (long long)rt * nkp * TILE_BYTES;
    }
    std::vector<long long> poff(ptab.size());
    for (size_t t = 0; t < ptab.size(); ++t) {
        const int nkp = padded_nkt(ops[pB[t]].K);
        poff[t] = bytes;
        for (int k = 0; k < nkp / KT_PER_JOB; ++k)
            jobs.push_back(OzJob{bytes + (long long)k * KT_PER_JOB * TILE_BYTES, -1, 0, k, (int)t});
        bytes += (long long)nkp * TILE_BYTES;
    }
    cudaError_t e = cudaMalloc(&tt.d_exps, (size_t)std::max<long long>(nexp, 1) * sizeof(int));
    if (e != cudaSuccess) return e;
    for (size_t q = 0; q < ops.size(); ++q) ops[q].exps = tt.d_exps + eoff[q];
    // output tiles: unpacked problems (M tiles x N tiles), then packed tiles (x N tiles); longest K first
    std::vector<OzTile> tiles;
    for (size_t i = 0; i < h.size(); ++i) {
        if (opB[i] < 0) continue;
        GemmDesc &g = h[i];
        g.ea = ops[opA[i]].exps;
        g.eb = ops[opB[i]].exps;
        if (packed_in[i] >= 0) continue;
        const int nkt = (g.K + BK - 1) / BK, nkp = padded_nkt(g.K);
        for (int mt = 0; mt < (g.M + BM - 1) / BM; ++mt)
            for (int nt = 0; nt < (g.N + BN - 1) / BN; ++nt)
                tiles.push_back(OzTile{ops[opA[i]].soff + (long long)mt * nkp * TILE_BYTES,
                                       ops[opB[i]].soff + (long long)nt * nkp * TILE_BYTES, (int)i, mt * BM, nt * BN, nkt, -1});
    }
    std::vector<OzRow> rows;
    for (size_t t = 0; t < ptab.size(); ++t) {
        const OzOperand &ob = ops[pB[t]];
        const int nkt = (ob.K + BK - 1) / BK, nkp = padded_nkt(ob.K);
        for (int nt = 0; nt < (ob.R + BN - 1) / BN; ++nt)
            tiles.push_back(OzTile{poff[t], ob.soff + (long long)nt * nkp * TILE_BYTES, ptab[t][0].p, 0, nt * BN, nkt, (int)t});
        rows.insert(rows.end(), ptab[t].begin(), ptab[t].end());
    }
    std::stable_sort(tiles.begin(), tiles.end(), [](const OzTile &x, const OzTile &y) { return x.nkt > y.nkt; });
    tt.tiles = (long long)tiles.size();
    tt.jobs = (long long)jobs.size();
    tt.sjobs = s0.back();
    tt.scratch_bytes = bytes;
    tt.nprob = (int)h.size();
    tt.nops = (int)ops.size();
    tt.packed_tiles = (long long)ptab.size();
    auto up = [](auto *&dst, const auto &v) -> cudaError_t {
        cudaError_t ee = cudaMalloc(&dst, std::max<size_t>(v.size(), 1) * sizeof(v[0]));
        if (ee != cudaSuccess || v.empty()) return ee;
        return cudaMemcpy(dst, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice);
    };
    if ((e = up(tt.d_desc, h)) != cudaSuccess) return e;
    if ((e = up(tt.d_sjobs0, s0)) != cudaSuccess) return e;
    OzOperand *dops = nullptr;
    OzJob *djobs = nullptr;
    OzTile *dtiles = nullptr;
    OzRow *drows = nullptr;
    e = up(dops, ops);
    tt.d_ops = dops;
    if (e != cudaSuccess) return e;
    e = up(djobs, jobs);
    tt.d_jobs = djobs;
    if (e != cudaSuccess) return e;
    e = up(dtiles, tiles);
    tt.d_otiles = dtiles;
    if (e != cudaSuccess) return e;
    e = up(drows, rows);
    tt.d_rows = drows;
    return e;
}

// Slice-image bytes of one problem's operands on their own (an upper bound: problems of a part may share them).
long long problem_image_bytes(const GemmDesc &g) {
    if (g.M <= 0 || g.N <= 0) return 0;
    const long long nkp = padded_nkt(g.K);
    return ((long long)(g.M + BM - 1) / BM + (g.N + BN - 1) / BN) * nkp * TILE_BYTES;
}

cudaError_t run_part(const TcTiles &tt, unsigned char *scratch, int *err, long long budget, cudaStream_t s);

}  // namespace

// Batches whose slice images exceed kOzPartBytes run as consecutive parts (ranges of problems, in batch order),
// each sliced into the same scratch after the previous part's GEMM: the scratch is bounded by the largest part
// instead of growing with the batch (the relaxation products at n_vir = 3000 would need ~60 GB at once).
constexpr long long kOzPartBytes = 8LL << 30;

cudaError_t bf16x4_batch_prepare(GemmBatch &b, TcTiles &tt) {
    tc_tiles_free(tt);
    if (b.h.empty()) return cudaSuccess;
    std::vector<std::pair<size_t, size_t>> ranges;
    size_t first = 0;
    long long acc = 0;
    for (size_t i = 0; i < b.h.size(); ++i) {
        const long long x = problem_image_bytes(b.h[i]);
        if (i > first && acc + x > kOzPartBytes) {
            ranges.push_back({first, i});
            first = i;
            acc = 0;
        }
        acc += x;
    }
    ranges.push_back({first, b.h.size()});
    if (ranges.size() == 1) return prepare_part(b.h, tt);
    tt.parts.resize(ranges.size());
    for (size_t q = 0; q < ranges.size(); ++q) {
        std::vector<GemmDesc> h(b.h.begin() + ranges[q].first, b.h.begin() + ranges[q].second);
        cudaError_t e = prepare_part(h, tt.parts[q]);
        if (e != cudaSuccess) return e;
        tt.scratch_bytes = std::max(tt.scratch_bytes, tt.parts[q].scratch_bytes);
        tt.tiles += tt.parts[q].tiles;
        tt.packed_tiles += tt.parts[q].packed_tiles;
    }
    return cudaSuccess;
}

cudaError_t bf16x4_batch_run(const TcTiles &tt, unsigned char *scratch, int *err, long long budget, cudaStream_t s) {
    if (tt.parts.empty()) return run_part(tt, scratch, err, budget, s);
    for (const TcTiles &p : tt.parts) {
        cudaError_t e = run_part(p, scratch, err, budget, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {

cudaError_t run_part(const TcTiles &tt, unsigned char *scratch, int *err, long long budget, cudaStream_t s) {
    if (tt.tiles == 0) return cudaSuccess;
    if (!scratch) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaError_t e;
    const OzOperand *ops = static_cast<const OzOperand *>(tt.d_ops);
    const OzRow *rows = static_cast<const OzRow *>(tt.d_rows);
    if (tt.sjobs > 0) {
        count_launch();
        k_oz_scales<<<(unsigned)tt.sjobs, 256, 0, s>>>(ops, tt.d_sjobs0, tt.nops);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (tt.jobs > 0) {
        count_launch();
        k_oz_slice<<<(unsigned)tt.jobs, NT, 0, s>>>(ops, static_cast<const OzJob *>(tt.d_jobs), rows, scratch);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    count_launch();
    k_oz_gemm<<<(unsigned)tt.tiles, NT, SMEM, s>>>(tt.d_desc, static_cast<const OzTile *>(tt.d_otiles), rows, scratch, err,
                                                   budget);
    return cudaGetLastError();
}

}  // namespace

}  // namespace osv
