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
// into FP64 registers (exactly for acc0..acc2); the epilogue restores 2^(e_m + e_n - 14).
//
// Two kernels per batch: (1) the row scales, then every operand tile (128 rows x 32 K) is sliced once into four
// 8 KB images already in the canonical no-swizzle K-major shared-memory layout (8 rows x 16 bytes per core
// matrix; K-adjacent core matrices 128 B apart, 8-row groups 512 B apart); (2) the GEMM: one CTA (256 threads)
// per 128 x 128 output tile, a three-stage pipeline of 64 KB stages filled by bulk asynchronous copies
// (cp.async.bulk + mbarrier transaction counts), thread 0 issuing 2 x 13 tcgen05.mma.kind::f16 (M = 128,
// N = 128, K = 16) per stage into four TMEM accumulators (512 columns).  Every wait is bounded: on expiry the
// error word is set, in-flight MMAs are waited for (bounded), TMEM is freed and the CTA returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>
#include <cstdint>

#include "kernels.cuh"
#include "tc_common.cuh"
#include "tc_gemm.h"

namespace osv {

namespace {

constexpr int BM = 128, BN = 128, BK = 32, NT = 256;
constexpr int NSLICE = 4;
constexpr int IMG = BM * BK * 2;                  // 8 KB: one slice of one 128 x 32 tile
constexpr int TILE_BYTES = NSLICE * IMG;          // 32 KB: the four slices of one operand tile
constexpr int STAGE = 2 * TILE_BYTES;             // A and B
constexpr int NSTAGE = 3;
constexpr int SMEM = NSTAGE * STAGE + 1024;
constexpr int CHUNK_KT = 8;                       // 256 K per exact chunk
constexpr uint32_t kIdesc = idesc_bf16(BM, BN);

__device__ __forceinline__ uint32_t koff(int r, int k) { return kmajor_off(r, k, BK); }
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) { return smem_desc(saddr, 16 * BK); }
constexpr int NACC = 4;


__device__ __forceinline__ void expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bulk asynchronous copy global -> shared, completion counted on bar (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}


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
// row scales and slice images are computed once per batch.
struct OzOperand {
    const double *ptr;
    long long ld;
    const int *rowmap, *kmap;
    int R, K, kcontig;
    int *exps;         // row scale exponents (R)
    long long soff;    // byte offset of its slice images in the scratch
};

__device__ __forceinline__ double oz_elem(const OzOperand &o, int r, int k) {
    const long long rr = o.rowmap ? o.rowmap[r] : r, kk = o.kmap ? o.kmap[k] : k;
    return o.kcontig ? o.ptr[rr * o.ld + kk] : o.ptr[kk * o.ld + rr];
}

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

// One CTA per operand tile (128 rows x 32 K): stage the FP64 values in shared memory (coalesced for either
// orientation), then write the four slice images (row tile major, then K tile).
__global__ void __launch_bounds__(NT) k_oz_slice(const OzOperand *__restrict__ ops, const long long *__restrict__ jobs0,
                                                 int nops, unsigned char *__restrict__ scratch) {
    __shared__ double xs[BK][BM + 1];
    __shared__ int es[BM];
    const long long t = blockIdx.x;
    const int p = find_prob(jobs0, nops, t);
    const OzOperand o = ops[p];
    const int nkt = (o.K + BK - 1) / BK;
    const long long j = t - jobs0[p];
    const int rt = (int)(j / nkt), kt = (int)(j % nkt);
    const int r0 = rt * BM, k0 = kt * BK;
    const int tid = threadIdx.x;
    for (int r = tid; r < BM; r += NT) es[r] = r0 + r < o.R ? o.exps[r0 + r] : 0;
    if (o.kcontig) {
        for (int idx = tid; idx < BM * BK; idx += NT) {   // lanes along k
            const int r = idx / BK, k = idx % BK;
            xs[k][r] = (r0 + r < o.R && k0 + k < o.K) ? oz_elem(o, r0 + r, k0 + k) : 0.0;
        }
    } else {
        for (int idx = tid; idx < BM * BK; idx += NT) {   // lanes along rows
            const int k = idx / BM, r = idx % BM;
            xs[k][r] = (r0 + r < o.R && k0 + k < o.K) ? oz_elem(o, r0 + r, k0 + k) : 0.0;
        }
    }
    __syncthreads();
    unsigned char *img = scratch + o.soff + ((long long)rt * nkt + kt) * TILE_BYTES;
    for (int c = tid; c < BM * (BK / 8); c += NT) {   // one core-matrix row (8 K of one row) per step
        const int r = c % BM, kg = c / BM;
        float sl[8][NSLICE];
#pragma unroll
        for (int q = 0; q < 8; ++q) slice4_exact(xs[kg * 8 + q][r], es[r], sl[q]);
        const uint32_t off = koff(r, kg * 8);
#pragma unroll
        for (int i = 0; i < NSLICE; ++i) {
            __nv_bfloat162 h[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn(sl[2 * q][i], sl[2 * q + 1][i]);
            *reinterpret_cast<uint4 *>(img + i * IMG + off) = *reinterpret_cast<uint4 *>(h);
        }
    }
}

__global__ void __launch_bounds__(NT, 1) k_oz_gemm(const GemmDesc *__restrict__ descs,
                                                  const long long *__restrict__ tile0, const long long *__restrict__ soff,
                                                  int nprob, const unsigned char *__restrict__ scratch, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[NSTAGE], empty[NSTAGE], dbar;
    __shared__ uint32_t s_taddr;
    __shared__ int s_fail;

    const long long t = blockIdx.x;
    const int p = find_prob(tile0, nprob, t);
    const GemmDesc g = descs[p];
    const long long local = t - tile0[p];
    const int tiles_n = (g.N + BN - 1) / BN;
    const int mt = int(local / tiles_n), ntile = int(local % tiles_n);
    const int m0 = mt * BM, n0 = ntile * BN;
    const int nkt = (g.K + BK - 1) / BK;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned char *Aimg = scratch + soff[2 * p] + (long long)mt * nkt * TILE_BYTES;
    const unsigned char *Bimg = scratch + soff[2 * p + 1] + (long long)ntile * nkt * TILE_BYTES;

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&dbar)));
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

    // drain targets: TMEM lanes of warp % 4 (rows), columns 64 * (warp / 4) .. + 63.  The chunk sums are added
    // into FP32 double-float pairs (hi, lo) with an error-free two-sum: FP32 ALU only (an FP64 add runs at 1/64 of
    // the FP32 rate on this part and made the drain the bottleneck); ~48 significant bits, ample for the
    // ~31-bit products.
    float chi[64], clo[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) {
        chi[j] = 0.f;
        clo[j] = 0.f;
    }

    int loaded = 0;   // k-tiles whose copies were issued (thread 0's view)
    auto load_stage = [&](int kt) {   // thread 0 only
        const int st = kt % NSTAGE;
        ++loaded;
        unsigned char *sA = smem + st * STAGE;
        expect_tx(&full[st], STAGE);
#pragma unroll
        for (int i = 0; i < NSLICE; ++i) {   // one copy per slice image keeps several requests in flight
            bulk_g2s(sA + i * IMG, Aimg + (long long)kt * TILE_BYTES + i * IMG, IMG, &full[st]);
            bulk_g2s(sA + TILE_BYTES + i * IMG, Bimg + (long long)kt * TILE_BYTES + i * IMG, IMG, &full[st]);
        }
    };

    int issued = 0;   // MMA groups committed (thread 0's view)
    bool ok = true;
    if (tid == 0)
        for (int kt = 0; kt < nkt && kt < NSTAGE - 1; ++kt) load_stage(kt);
    int chunk = 0;
    for (int kt = 0; kt < nkt; ++kt) {
        const int st = kt % NSTAGE;
        const bool first_of_chunk = (kt % CHUNK_KT) == 0;
        const bool last_of_chunk = (kt % CHUNK_KT) == CHUNK_KT - 1 || kt == nkt - 1;
        if (tid == 0 && !s_fail) {
            if (!tc_wait(&full[st], (uint32_t)((kt / NSTAGE) & 1))) {
                raise_err(err, kDevTimeout);
                s_fail = 1;
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t a0 = smem_u32(smem + st * STAGE), b0 = a0 + TILE_BYTES;
#pragma unroll
                for (int ks = 0; ks < BK / 16; ++ks) {
                    const uint32_t off = ks * 256;
                    bool fresh[NACC];
#pragma unroll
                    for (int a = 0; a < NACC; ++a) fresh[a] = first_of_chunk && ks == 0;
#pragma unroll
                    for (int i = 0; i < NSLICE; ++i)
#pragma unroll
                        for (int j = 0; j < NSLICE; ++j) {
                            const int d = i + j;
                            if (d > 4) continue;
                            const int a = d < 3 ? d : 3;
                            tc_mma_bf16(taddr + (uint32_t)(a * BN), sdesc(a0 + i * IMG + off), sdesc(b0 + j * IMG + off),
                                        kIdesc, !fresh[a]);
                            fresh[a] = false;
                        }
                }
                tc_commit(&empty[st]);
                ++issued;
                // refill the stage that kt - 1 used with kt + 2, once its MMAs are done
                const int nk = kt + NSTAGE - 1;
                if (nk < nkt) {
                    if (kt >= 1 && !tc_wait(&empty[(kt - 1) % NSTAGE], (uint32_t)(((kt - 1) / NSTAGE) & 1))) {
                        raise_err(err, kDevTimeout);
                        s_fail = 1;
                    } else {
                        load_stage(nk);
                    }
                }
            }
        }
        if (last_of_chunk) {
            if (tid == 0) tc_commit(&dbar);
            __syncthreads();
            if (s_fail) { ok = false; break; }
            if (!tc_wait(&dbar, (uint32_t)(chunk & 1))) {
                raise_err(err, kDevTimeout);
                s_fail = 1;
            }
            __syncthreads();
            if (s_fail) { ok = false; break; }
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
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        two_sum_f32(chi[c + i], clo[c + i], v0[i]);
                        two_sum_f32(chi[c + 16 + i], clo[c + 16 + i], v1[i]);
                    }
                }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            ++chunk;
        }
    }
    if (!ok && tid == 0) {
        // let every committed MMA group finish before TMEM is released, and every issued copy land before the
        // shared memory is given up (both bounded)
        for (int s = 0; s < NSTAGE; ++s) {
            const int uses = issued / NSTAGE + (s < issued % NSTAGE ? 1 : 0);
            if (uses > 0) tc_wait(&empty[s], (uint32_t)((uses - 1) & 1));
        }
        for (int kt = issued; kt < loaded; ++kt) tc_wait(&full[kt % NSTAGE], (uint32_t)((kt / NSTAGE) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(taddr));
    }
    if (!ok) return;
    // epilogue through shared memory (the stage buffers are idle): the (hi, lo) pairs of the row-major 128 x 128
    // tile, then coalesced stores; the only FP64 operations are one add and one or two multiplies per element
    float2 *sC = reinterpret_cast<float2 *>(smem);
    constexpr int LDC = BN + 1;
    {
        const int r = (warp & 3) * 32 + lane;
#pragma unroll
        for (int j = 0; j < 64; ++j) sC[r * LDC + (warp >> 2) * 64 + j] = make_float2(chi[j], clo[j]);
    }
    __syncthreads();
    // alpha = +-2^k folds into the exponent (no FP64 multiply); the value itself is assembled with integer
    // operations (df_to_double)
    const unsigned long long abits = (unsigned long long)__double_as_longlong(g.alpha);
    const int aexp = (int)((abits >> 52) & 0x7FF);
    const bool alpha_p2 = (abits & 0xFFFFFFFFFFFFFULL) == 0 && aexp > 0 && aexp < 0x7FF;
    const int ashift = alpha_p2 ? aexp - 1023 : 0;
    const unsigned long long asign = alpha_p2 ? (abits & 0x8000000000000000ULL) : 0ULL;
    for (int r = warp; r < BM; r += NT / 32) {
        const int m = m0 + r;
        if (m >= g.M) break;
        const int em = g.ea[m] - 14 + ashift;
        for (int c = lane; c < BN; c += 32) {
            const int n = n0 + c;
            if (n >= g.N) break;
            const float2 hl = sC[r * LDC + c];
            double val = __longlong_as_double(__double_as_longlong(df_to_double(hl.x, hl.y, em + g.eb[n])) ^ (long long)asign);
            if (!alpha_p2) val *= g.alpha;
            const long long nc = g.n_idx_c ? g.n_idx_c[n] : n;
            double *cp = g.C + (long long)m * g.ldc + nc;
            if (g.atomic) atomicAdd(cp, val);
            else *cp = val + (g.beta != 0.0 ? g.beta * *cp : 0.0);
        }
    }
}

}  // namespace

cudaError_t bf16x4_batch_prepare(GemmBatch &b, TcTiles &tt) {
    tc_tiles_free(tt);
    if (b.h.empty()) return cudaSuccess;
    std::vector<GemmDesc> h = b.h;
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
    std::vector<int> opA(h.size()), opB(h.size());
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
        if (g.M <= 0 || g.N <= 0) {
            opA[i] = opB[i] = -1;
            continue;
        }
        opA[i] = add(Key{g.A, g.lda, g.transA == 0 ? g.a_rows : nullptr, g.k_idx_a, g.M, g.K, g.transA == 0 ? 1 : 0});
        opB[i] = add(Key{g.B, g.ldb, g.n_idx_b, g.k_idx_b, g.N, g.K, g.transB == 1 ? 1 : 0});
    }
    // scale arrays, slice regions and job prefixes per operand
    long long nexp = 0, bytes = 0;
    std::vector<long long> j0(ops.size() + 1, 0), s0(ops.size() + 1, 0), eoff(ops.size());
    for (size_t q = 0; q < ops.size(); ++q) {
        OzOperand &o = ops[q];
        const long long nkt = (o.K + BK - 1) / BK, rt = (o.R + BM - 1) / BM;
        eoff[q] = nexp;
        nexp += o.R;
        o.soff = bytes;
        bytes += rt * nkt * TILE_BYTES;
        j0[q + 1] = j0[q] + rt * nkt;
        s0[q + 1] = s0[q] + (o.R + SROWS - 1) / SROWS;
    }
    cudaError_t e = cudaMalloc(&tt.d_exps, (size_t)std::max<long long>(nexp, 1) * sizeof(int));
    if (e != cudaSuccess) return e;
    for (size_t q = 0; q < ops.size(); ++q) ops[q].exps = tt.d_exps + eoff[q];
    std::vector<long long> t0(h.size() + 1, 0), so(2 * h.size(), 0);
    for (size_t i = 0; i < h.size(); ++i) {
        GemmDesc &g = h[i];
        long long tiles = 0;
        if (opA[i] >= 0) {
            g.ea = ops[opA[i]].exps;
            g.eb = ops[opB[i]].exps;
            so[2 * i] = ops[opA[i]].soff;
            so[2 * i + 1] = ops[opB[i]].soff;
            tiles = (long long)((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
        }
        t0[i + 1] = t0[i] + tiles;
    }
    tt.tiles = t0.back();
    tt.jobs = j0.back();
    tt.sjobs = s0.back();
    tt.scratch_bytes = bytes;
    tt.nprob = (int)h.size();
    tt.nops = (int)ops.size();
    auto up = [](auto *&dst, const auto &v) -> cudaError_t {
        cudaError_t ee = cudaMalloc(&dst, std::max<size_t>(v.size(), 1) * sizeof(v[0]));
        if (ee != cudaSuccess || v.empty()) return ee;
        return cudaMemcpy(dst, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice);
    };
    if ((e = up(tt.d_desc, h)) != cudaSuccess) return e;
    if ((e = up(tt.d_tile0, t0)) != cudaSuccess) return e;
    if ((e = up(tt.d_soff, so)) != cudaSuccess) return e;
    if ((e = up(tt.d_jobs0, j0)) != cudaSuccess) return e;
    if ((e = up(tt.d_sjobs0, s0)) != cudaSuccess) return e;
    OzOperand *dops = nullptr;
    if ((e = up(dops, ops)) != cudaSuccess) return e;
    tt.d_ops = dops;
    return cudaSuccess;
}

cudaError_t bf16x4_batch_run(const TcTiles &tt, unsigned char *scratch, int *err, cudaStream_t s) {
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
    if (tt.sjobs > 0) {
        count_launch();
        k_oz_scales<<<(unsigned)tt.sjobs, 256, 0, s>>>(ops, tt.d_sjobs0, tt.nops);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (tt.jobs > 0) {
        count_launch();
        k_oz_slice<<<(unsigned)tt.jobs, NT, 0, s>>>(ops, tt.d_jobs0, tt.nops, scratch);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    count_launch();
    k_oz_gemm<<<(unsigned)tt.tiles, NT, SMEM, s>>>(tt.d_desc, tt.d_tile0, tt.d_soff, tt.nprob, scratch, err);
    return cudaGetLastError();
}

}  // namespace osv
