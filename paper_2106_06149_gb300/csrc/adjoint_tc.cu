// Per-cluster gradient partials (the densities of Eqs. 14-16 and 33-34 in the pseudo-canonical pair bases, the
// same quantities as k_cluster_adjoint_df) with every product on the tcgen05 tensor cores.
//
// One CTA (512 threads) per SM walks clusters.  Every operand of a product (order <= 80) is cut, in shared
// memory, into four exact BF16 digit planes with one power-of-two scale per matrix (the slicing of tc_oz.cu:
// N = round(x 2^(31-e)), base-256 digits, slice i stored as s_i 2^(-8 i)) in the canonical no-swizzle K-major
// layout of an 80 x 80 tile (K = 80, zero-padded).  Thread 0 issues the 13 digit products with i + j <= 4 as
// tcgen05.mma.kind::f16 (M = 128, N = 80, K = 16; rows 80..127 of A are never read back) into three tensor-memory
// accumulators by order: i + j = 0 and 1 (exact integer sums over K <= 160) and i + j >= 2 (rounded at 2^-24 of a
// term <= 2^-16 of the result, ~2^-40).  Two products run side by side in 480 of the 512 tensor-memory columns.
// Warps 0-3 read the sums back (tcgen05.ld, one row per lane), combine the three accumulators with an FP32
// two-sum and assemble FP64 values with integer operations.  Relative accuracy ~2^-31 of the operand scales,
// ample for a gradient held to ~1e-7.
//
// Coupling term (dst pair p, src pair q, block S~, Fock factor f):
//   U1 = Tb_p S~, U2 = Tb_p^T S~  (Tb = 2T - T^T), then  M2 = U1 T'^T + U2 T',  dE/dS~ += -w m f M2,
//   dE/df_xy += -w <S~, U1 T'^T>  (= <S~ T', Tb S~>).
// Slot (pair p): M2 = Tb T^T + T^T Tb, M1' = (Tb L') T^T + (L' T)^T Tb (L' = diag(e) - f_ii - f_jj),
//   dE/dS~_p += w m M1', dE/dF~_p += w m M2, dE/df_ii, dE/df_jj -= w m <T, Tb>.
// Every wait on the MMA completion barrier is bounded: on expiry the error word is set, the CTA waits (bounded)
// for its MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "adjoint.h"
#include "tc_common.cuh"

namespace osv {

namespace {

constexpr int kTC = 512;                  // threads
constexpr int kR = kAdjTcMaxOrder;        // 80: rows, K and N of every product
constexpr int kPlane = kR * kR * 2;       // one BF16 digit plane of an 80 x 80 operand
constexpr int kImg = 4 * kPlane;          // its four planes
constexpr uint32_t kSBO = 16 * kR;        // 8-row groups of a K = 80 image
constexpr uint32_t kIdesc = idesc_bf16(128, kR);
constexpr uint32_t kColA = 0, kColB = 3 * kR;     // accumulator triples of the two products in flight
constexpr size_t kSmem = 4 * (size_t)kImg + 1024;

static_assert(6 * kR <= 512, "two accumulator triples must fit the 512 tensor-memory columns");

__device__ __forceinline__ void tc_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// The four digit planes of the eight elements (r, k0 .. k0 + 7) of an operand image (scale 2^e): one 16-byte
// store per plane (a core-matrix row).  A warp's items take 32 consecutive rows of one K chunk, so its 16-byte
// stores cover all 32 banks four times (the minimum for 512 bytes).
__device__ __forceinline__ void put8(unsigned char *img, int r, int k0, const double *x, int e) {
    uint32_t w[4][4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
        float s0[4], s1[4];
        slice4_exact(x[j], e, s0);
        slice4_exact(x[j + 1], e, s1);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 v = __floats2bfloat162_rn(s0[i], s1[i]);
            w[i][j >> 1] = *reinterpret_cast<const uint32_t *>(&v);
        }
    }
    const uint32_t off = kmajor_off(r, k0, kR);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        *reinterpret_cast<uint4 *>(img + i * kPlane + off) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
}

// K-chunk items of an 80 x 80 image: item it -> row it % 80, K chunk it / 80 (800 items)
constexpr int kItems = kR * (kR / 8);

struct Tc {
    unsigned char *img[4];   // image slots: 0, 1 A operands; 2, 3 B operands (slot 0's and 1's reads of rows
                             // 80..127 fall inside the next slot)
    uint64_t *bar;
    uint32_t phase;
    uint32_t taddr;
    int *fail;
    unsigned long long *red;   // kTC / 32 words
    long long budget;          // clock cycles of a product wait (<= 0: the default)
};

// largest |x| over the CTA (bit patterns), broadcast
__device__ unsigned long long block_max_bits(unsigned long long v, unsigned long long *red) {
    v = warp_max_bits(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    unsigned long long m = 0;
    for (int w = 0; w < kTC / 32; ++w) m = red[w] > m ? red[w] : m;
    return m;
}

// D[col] (+)= A[slot a] B[slot b]^T over K = 80 for the 13 digit products (thread 0)
__device__ __forceinline__ void issue_product(const Tc &c, int a, int b, uint32_t col, bool fresh) {
    const uint32_t sa = smem_u32(c.img[a]), sb = smem_u32(c.img[b]);
    bool first[3] = {fresh, fresh, fresh};
#pragma unroll
    for (int ks = 0; ks < kR / 16; ++ks)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (i + j > 4) continue;
                const int acc = i + j < 2 ? i + j : 2;
                tc_mma_bf16(c.taddr + col + (uint32_t)(acc * kR), smem_desc(sa + i * kPlane + ks * 256, kSBO),
                            smem_desc(sb + j * kPlane + ks * 256, kSBO), kIdesc, !first[acc]);
                first[acc] = false;
            }
}

// make every thread's digit stores visible to the tensor core, issue, and wait (bounded) for completion.
// issue(c) runs on thread 0 between the barrier and the commit.  Returns false when the CTA must stop.
template <class F>
__device__ bool run_mma(Tc &c, F issue, int *err) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        issue(c);
        tc_commit(c.bar);
    }
    const bool done = tc_wait(c.bar, c.phase, c.budget);
    if (done) c.phase ^= 1u;   // on expiry the pending phase is waited for once more before tensor memory is freed
    if (!done && threadIdx.x == 0) {
        raise_err(err, kDevTimeout);
        *c.fail = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    return *c.fail == 0;
}

// this lane's row (lane quarter (warp & 3)) of an accumulator triple at columns col .. col + 7, as (hi, lo) pairs
__device__ __forceinline__ void read8(const Tc &c, uint32_t col, float *hi, float *lo) {
    const uint32_t base = c.taddr + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16) + col;
    float a0[8], a1[8], a2[8];
    tc_ld8(base, a0);
    tc_ld8(base + kR, a1);
    tc_ld8(base + 2 * kR, a2);
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        hi[i] = a0[i];
        lo[i] = 0.f;
        two_sum_f32(hi[i], lo[i], a1[i]);
        two_sum_f32(hi[i], lo[i], a2[i]);
    }
}

__global__ void __launch_bounds__(kTC, 1) k_cluster_adjoint_tc(AdjArgsS A, int *err, long long budget) {
    extern __shared__ __align__(16) unsigned char tc_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_taddr;
    __shared__ int s_fail;
    __shared__ unsigned long long s_red[kTC / 32];
    __shared__ double s_dred[kTC / 32];
    __shared__ double s_ep[kR];   // slot phase: e' = e - f_ii - f_jj (zero beyond the pair order)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar)));
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
    Tc c{{smem, smem + kImg, smem + 2 * kImg, smem + 3 * kImg}, &s_bar, 0u, s_taddr, &s_fail, s_red, budget};
    // tensor-memory reads: warp w reads lane quarter w & 3 (rows 32 (w & 3) + lane) and the 8-column chunks
    // w >> 2, w >> 2 + 4, ... of an 80-column accumulator
    const int row = (warp & 3) * 32 + lane, ch0 = warp >> 2;

    for (int q = blockIdx.x; q < A.ncl && !s_fail; q += gridDim.x) {
        const int cl = A.order[q];
        const ClusterInfo C = A.clusters[cl];
        if (C.weight == 0) continue;
        const double w = (double)C.weight;
        // ------------------------------------------------------------------------------------------- slots
        for (int s = C.slot0; s < C.slot1 && !s_fail; ++s) {
            const Slot S = A.slots[s];
            const PairInfo P = A.pairs[S.pair];
            const int r = A.rdim[S.pair], np = P.np;
            const double *T = A.Tslot + S.t_off;
            const double *e = A.e + P.e_off;
            const double fii = A.focc[(long long)P.i * A.n_occ + P.i], fjj = A.focc[(long long)P.j * A.n_occ + P.j];
            const double wm = w * S.mult;
            const float2 wmd = split_df(wm);
            for (int k = tid; k < kR; k += kTC) s_ep[k] = k < r ? e[k] - fii - fjj : 0.0;   // read after barriers below
            // item (a, k0): T(a, k), T(k, a) for k = k0 .. k0 + 7 (zero outside r x r)
            auto load = [&](int it, int &a, int &k0, double *x, double *xt) {
                a = it % kR;
                k0 = (it / kR) * 8;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const bool in = a < r && k0 + j < r;
                    x[j] = in ? T[(long long)a * np + k0 + j] : 0.0;
                    xt[j] = in ? T[(long long)(k0 + j) * np + a] : 0.0;
                }
            };
            double *Tbs = A.TbS + S.t_off;
            auto tbval = [&](int x_, int y_) -> double {   // Tb(x, y), zero outside r x r
                return (x_ < r && y_ < r) ? Tbs[(long long)x_ * np + y_] : 0.0;
            };
            unsigned long long mt = 0, mb = 0;
            double tt = 0.0;
            for (int it = tid; it < kItems; it += kTC) {
                int a, k0;
                double x[8], xt[8];
                load(it, a, k0, x, xt);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const double xb = 2.0 * x[j] - xt[j];   // Tb(a, k)
                    tt = fma(x[j], xb, tt);
                    mt = max(mt, abs_bits64(x[j]));
                    mb = max(mb, abs_bits64(xb));
                    // kept for the passes below and the coupling terms of this destination slot
                    if (a < r && k0 + j < r) Tbs[(long long)a * np + k0 + j] = xb;
                }
            }
            tt = block_sum(tt, s_dred);
            if (tid == 0) {
                atomicAdd(&A.dF[(long long)P.i * A.n_occ + P.i], -wm * tt);
                atomicAdd(&A.dF[(long long)P.j * A.n_occ + P.j], -wm * tt);
            }
            const int eT = scale_exp_of_bits(block_max_bits(mt, s_red));
            const int eB = scale_exp_of_bits(block_max_bits(mb, s_red));
            if (tid == 0) A.ebS[s] = eB;
            // slot 0: Tb (A), slot 1: T^T (A), slot 2: T (B), slot 3: Tb^T (B): at (a, k) they hold Tb(a, k),
            // T(k, a), T(a, k), Tb(k, a) = 2 T(k, a) - T(a, k)
            for (int it = tid; it < kItems; it += kTC) {
                int a, k0;
                double x[8], xt[8], v[8];
                load(it, a, k0, x, xt);
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = tbval(a, k0 + j);
                put8(c.img[0], a, k0, v, eB);
                put8(c.img[1], a, k0, xt, eT);
                put8(c.img[2], a, k0, x, eT);
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = tbval(k0 + j, a);
                put8(c.img[3], a, k0, v, eB);
            }
            // M2 = Tb T^T + T^T Tb (columns kColA)
            if (!run_mma(c, [](const Tc &cc) { issue_product(cc, 0, 2, kColA, true); issue_product(cc, 1, 3, kColA, false); }, err))
                break;
            // slots 0, 1 <- Tb L' and (L' T)^T: at (a, k) Tb(a, k) e'_k and e'_k T(k, a) (e' = e - f_ii - f_jj),
            // with scales making the two products' exponents equal
            unsigned long long m3 = 0, m4 = 0;
            for (int it = tid; it < kItems; it += kTC) {
                int a, k0;
                double x[8], xt[8];
                load(it, a, k0, x, xt);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const double ep = s_ep[k0 + j];
                    m3 = max(m3, abs_bits64(tbval(a, k0 + j) * ep));
                    m4 = max(m4, abs_bits64(ep * xt[j]));
                }
            }
            const int e3raw = scale_exp_of_bits(block_max_bits(m3, s_red));
            const int e4raw = scale_exp_of_bits(block_max_bits(m4, s_red));
            const int e3 = max(e3raw, e4raw + eB - eT), e4 = e3 + eT - eB;   // e3 >= e3raw, e4 >= e4raw
            for (int it = tid; it < kItems; it += kTC) {
                int a, k0;
                double x[8], xt[8], v3[8], v4[8];
                load(it, a, k0, x, xt);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const double ep = s_ep[k0 + j];
                    v3[j] = tbval(a, k0 + j) * ep;
                    v4[j] = ep * xt[j];
                }
                put8(c.img[0], a, k0, v3, e3);
                put8(c.img[1], a, k0, v4, e4);
            }
            // M1' = (Tb L') T^T + (L' T)^T Tb (columns kColB)
            if (!run_mma(c, [](const Tc &cc) { issue_product(cc, 0, 2, kColB, true); issue_product(cc, 1, 3, kColB, false); }, err))
                break;
            {
                const int E2 = eB + eT - 14, E1 = e3 + eT - 14;
                for (int ch = ch0; ch < kR / 8; ch += 4) {
                    float h2[8], l2[8], h1[8], l1[8];
                    read8(c, kColA + ch * 8, h2, l2);
                    read8(c, kColB + ch * 8, h1, l1);
                    if (row >= r) continue;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int b = ch * 8 + i;
                        if (b >= r) break;
                        const long long o = P.off + (long long)row * np + b;
                        // w m times the sums in double-float, then integer FP64 assembly (no FP64-pipe work)
                        atomicAdd(&A.GS[o], df_to_double_mul(h1[i], l1[i], wmd, E1));
                        atomicAdd(&A.GF[o], df_to_double_mul(h2[i], l2[i], wmd, E2));
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
        }
        // ------------------------------------------------------------------------------------------- terms
        for (int t = C.term0; t < C.term1 && !s_fail; ++t) {
            const Term Tm = A.terms[t];
            const Slot Sd = A.slots[Tm.dst], Ssl = A.slots[Tm.src];
            const PairInfo Pd = A.pairs[Sd.pair], Ps = A.pairs[Ssl.pair];
            const int rp = A.rdim[Sd.pair], rq = A.rdim[Ssl.pair];
            const int np = Pd.np, nq = Ps.np;
            const double f = A.focc[(long long)Tm.fx * A.n_occ + Tm.fy];
            const double *Sb = A.Stil + Tm.sblk;
            const long long lds = Tm.s_trans ? np : nq;
            const double *Tq = A.Tslot + Ssl.t_off;
            const double wm = w * Sd.mult;
            auto sval = [&](int c_, int b_) -> double {   // S~(c, b), zero outside rp x rq
                return (c_ < rp && b_ < rq) ? (Tm.s_trans ? Sb[(long long)b_ * lds + c_] : Sb[(long long)c_ * lds + b_]) : 0.0;
            };
            auto tqval = [&](int x_, int y_) -> double {   // T'(x, y), zero outside rq x rq
                return (x_ < rq && y_ < rq) ? (Tm.t_trans ? Tq[(long long)y_ * nq + x_] : Tq[(long long)x_ * nq + y_]) : 0.0;
            };
            // scales: S~, T' (Tb's, and Tb itself, from the destination slot's pass above: no FP64 work here)
            const double *Tbp = A.TbS + Sd.t_off;
            unsigned long long ms = 0, mq = 0;
            for (int it = tid; it < kItems; it += kTC) {
                const int a = it % kR, k0 = (it / kR) * 8;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int k = k0 + j;
                    ms = max(ms, abs_bits64(sval(k, a)));
                    mq = max(mq, abs_bits64(tqval(a, k)));
                }
            }
            const int eTb = A.ebS[Tm.dst];
            const int eS = scale_exp_of_bits(block_max_bits(ms, s_red));
            const int eTq = scale_exp_of_bits(block_max_bits(mq, s_red));
            // slot 0: Tb (A), slot 1: Tb^T (A), slot 2: B[b][c] = S~(c, b), slot 3: B[b][c] = T'(c, b)
            for (int it = tid; it < kItems; it += kTC) {
                const int a = it % kR, k0 = (it / kR) * 8;
                double v0[8], v1[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int k = k0 + j;
                    const bool in = a < rp && k < rp;
                    v0[j] = in ? Tbp[(long long)a * np + k] : 0.0;
                    v1[j] = in ? Tbp[(long long)k * np + a] : 0.0;
                }
                put8(c.img[0], a, k0, v0, eTb);
                put8(c.img[1], a, k0, v1, eTb);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    v0[j] = sval(k0 + j, a);
                    v1[j] = tqval(k0 + j, a);
                }
                put8(c.img[2], a, k0, v0, eS);
                put8(c.img[3], a, k0, v1, eTq);
            }
            // U1 = Tb S~ (columns kColA), U2 = Tb^T S~ (kColB)
            if (!run_mma(c, [](const Tc &cc) { issue_product(cc, 0, 2, kColA, true); issue_product(cc, 1, 2, kColB, true); }, err))
                break;
            // one scale for U1 and U2 (so that U1 T'^T and U2 T' share the tensor-memory sums' exponent)
            const int EU = eTb + eS - 14;
            unsigned long long mu = 0;
            for (int ch = ch0; ch < kR / 8; ch += 4) {
                float h[8], l[8], h2[8], l2[8];
                read8(c, kColA + ch * 8, h, l);
                read8(c, kColB + ch * 8, h2, l2);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (row < rp && ch * 8 + i < rq) {
                        mu = max(mu, abs_bits64(df_to_double(h[i], l[i], EU)));
                        mu = max(mu, abs_bits64(df_to_double(h2[i], l2[i], EU)));
                    }
            }
            const int eU = scale_exp_of_bits(block_max_bits(mu, s_red));
            // U1 -> slot 0, U2 -> slot 1 (A: row a, K = b < rq, zero beyond)
            for (int ch = ch0; ch < kR / 8; ch += 4) {
                float h[8], l[8], h2[8], l2[8];
                read8(c, kColA + ch * 8, h, l);
                read8(c, kColB + ch * 8, h2, l2);
                if (row >= kR) continue;
                double v1[8], v2[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const bool in = row < rp && ch * 8 + i < rq;
                    v1[i] = in ? df_to_double(h[i], l[i], EU) : 0.0;
                    v2[i] = in ? df_to_double(h2[i], l2[i], EU) : 0.0;
                }
                put8(c.img[0], row, ch * 8, v1, eU);
                put8(c.img[1], row, ch * 8, v2, eU);
            }
            // slot 2 <- B[b][c] = T'(b, c) (slot 2's S~ was read by the MMAs above, which have completed)
            for (int it = tid; it < kItems; it += kTC) {
                const int a = it % kR, k0 = (it / kR) * 8;
                double v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = tqval(a, k0 + j);
                put8(c.img[2], a, k0, v, eTq);
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            // M2a = U1 T'^T (columns kColA), M2b = U2 T' (kColB)
            if (!run_mma(c, [](const Tc &cc) { issue_product(cc, 0, 2, kColA, true); issue_product(cc, 1, 3, kColB, true); }, err))
                break;
            double xs = 0.0;
            {
                const int EM = eU + eTq - 14;
                const float2 gd = split_df(-wm * f);
                float xh = 0.f, xl = 0.f;   // <S~, M2a> in double-float, exponent EM
                double *G = A.GSc + Tm.sblk;
                for (int ch = ch0; ch < kR / 8; ch += 4) {
                    float h[8], l[8], h2[8], l2[8];
                    read8(c, kColA + ch * 8, h, l);
                    read8(c, kColB + ch * 8, h2, l2);
                    if (row >= rp) continue;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int b = ch * 8 + i;
                        if (b >= rq) break;
                        df_fma(xh, xl, split_df(sval(row, b)), make_float2(h[i], l[i]));
                        two_sum_f32(h[i], l[i], h2[i]);   // M2a + M2b (same exponent)
                        l[i] = __fadd_rn(l[i], l2[i]);
                        const double v = df_to_double_mul(h[i], l[i], gd, EM);
                        if (Tm.s_trans) atomicAdd(&G[(long long)b * np + row], v);   // stored (src pair) x (dst pair)
                        else atomicAdd(&G[(long long)row * nq + b], v);
                    }
                }
                xs = df_to_double(xh, xl, EM);
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            xs = block_sum(xs, s_dred);
            if (tid == 0) {
                atomicAdd(&A.dF[(long long)Tm.fx * A.n_occ + Tm.fy], -w * xs);
                if (Pd.i != Pd.j) atomicAdd(&A.dF[(long long)Tm.fy * A.n_occ + Tm.fx], -w * xs);
            }
            __syncthreads();
        }
    }
    if (s_fail && tid == 0) tc_wait(c.bar, c.phase);   // a timed-out batch: let its MMAs finish (bounded)
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(c.taddr));
    }
}

}  // namespace

cudaError_t launch_cluster_adjoint_tc(const AdjArgsS &a, int ncl, int *err, long long budget, cudaStream_t s) {
    if (ncl <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_cluster_adjoint_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    count_launch();
    k_cluster_adjoint_tc<<<std::min(ncl, 152), kTC, kSmem, s>>>(a, err, budget);
    return cudaGetLastError();
}

}  // namespace osv
