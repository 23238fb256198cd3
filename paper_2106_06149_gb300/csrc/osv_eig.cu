// OSV eigenproblem of Eq. 6 without a full eigendecomposition, and small dense eigensolves by parallel Jacobi.
//
// Only the n_k kept eigenvectors of T_kk enter the energy, and the OSV relaxation of Eq. 8 needs the discarded
// eigenvectors only through the restricted resolvent sum_nu q'_nu q'_nu^T / (omega_mu - omega'_nu).  So:
//   1. Householder tridiagonalisation T = H Tri H^T (reflector k kept contiguous in row k).  One pass over the
//      lower triangle of the trailing matrix per step: the rank-2 update of step k-1 is applied lazily in the
//      same pass that forms the product A v_k of step k from the row and column sums of the stored triangle
//      (warp per row, coalesced, division free).  FP64: one CTA per LMO.  FP32 (a first stage, refined to FP64
//      accuracy afterwards), launch shapes picked by the plan's autotuner: a pair of CTAs per matrix, one CTA
//      (two per SM), clusters of 4 / 8 / 16 CTAs (k_tridiag_cl), and delayed updates (k_tridiag_delayed: the
//      rank-2 updates of NB steps written together, read-only passes in between, optionally with the row chunks
//      staged through a per-lane cp.async ring in shared memory);
//   2. the n_max largest eigenvalues of Tri by 32-point multisection of the Sturm count (one warp per
//      eigenvalue, FP64 arithmetic): ~11 rounds instead of ~60 bisection steps, each a chain of n dependent
//      multiply-adds (on GB300 a dependent FP64 operation costs ~64 cycles and a division ~430);
//   3. the kept eigenvectors by inverse iteration on Tri, one thread per vector, then two classical Gram-Schmidt
//      passes (CGS2) inside the kept set;
//   4. back-transformation q = H y through the stored reflectors (warp per vector);
//   5. (adjoint) x_mu = P_perp (omega_mu - Tri)^{-1} P_perp r_mu by a pivoted tridiagonal solve and a CGS2
//      projection, which is exactly the kept x discarded block of the perturbed eigenproblem (Eq. 8).
// Every step is templated on the working precision R: double for the FP64 path, float for the first stage of
// the mixed path (refined to FP64 accuracy afterwards).
// Pair overlap / pseudo-canonical eigenproblems (order <= 2 nmax) use a cyclic parallel Jacobi in shared memory.
#include <algorithm>
#include <cfloat>
#include <cstdint>

#include <cooperative_groups.h>

#include "jacobi.cuh"
#include "kernels.cuh"
#include "osv_eig.h"

namespace osv {

namespace cg = cooperative_groups;

namespace {

constexpr int kT = 256;
constexpr int kTT = 512;   // tridiagonalisation block
constexpr int kTJ = 512;   // mixed Jacobi block (one CTA per SM: its shared memory)

template <class R>
struct Lim;
template <>
struct Lim<double> {
    static constexpr double eps = DBL_EPSILON;
    static constexpr double tiny = 1e-300;
};
template <>
struct Lim<float> {
    static constexpr float eps = FLT_EPSILON;
    static constexpr float tiny = 1e-37f;
};

template <class R>
__device__ __forceinline__ R warp_sum_t(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Pass (b) of step k of the Householder reduction over one CTA's rows: the rows rstart + RS j (j >= 0) of the lower
// triangle of the trailing matrix, warp w taking the rows rstart + RS (w + NW q), q < 4, per round so that several
// independent loads are in flight per lane.  Applies the pending update of step k-1 (vo, po) to columns k+1 .. r of
// each row, writes the row sum of A v into p[r], scatters the column sums into cs (one shared-memory add per column
// and group of four rows) and hands the updated element of column k+1 of each row to stash(r, x).  UV: groups of
// four rows per lane in flight in the 16-byte path (two CTAs per SM leave a 64-register budget: UV = 1).
template <class R, int UV, class Stash>
__device__ __forceinline__ void tri_rows_pass(R *__restrict__ A, long long lda, bool vec, int k, int n, int rstart,
                                              int RS, const R *__restrict__ vo, const R *__restrict__ po,
                                              const R *__restrict__ v, R *cs, R *p, Stash stash) {
    constexpr int NW = kTT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int r0 = rstart + RS * wid; r0 < n; r0 += 4 * RS * NW) {
        R *row[4];
        R vr[4], pr[4], vq[4], acc[4];
        int rq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = r0 + q * RS * NW;
            const bool ok = r < n;
            rq[q] = ok ? r : -1;   // columns c <= rq[q] belong to row q
            row[q] = A + (long long)(ok ? r : r0) * lda;
            vr[q] = ok ? vo[r] : (R)0;
            pr[q] = ok ? po[r] : (R)0;
            vq[q] = ok ? v[r] : (R)0;
            acc[q] = 0;
        }
        const int nr = min(4, (n - 1 - r0) / (RS * NW) + 1);
        const int hi = rq[nr - 1];   // the group's longest row
        auto col = [&](int c) {      // one column of the (up to) four rows
            const R poc = po[c], voc = vo[c], vc = v[c];
            R cl = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nr && c <= rq[q]) {
                    const R x = row[q][c] - vr[q] * poc - pr[q] * voc;
                    row[q][c] = x;
                    acc[q] = fma(x, vc, acc[q]);
                    if (c < rq[q]) cl = fma(x, vq[q], cl);
                    if (c == k + 1) stash(rq[q], x);
                }
            if (c < hi) atomicAdd(cs + c, cl);
        };
        bool vdone = false;
        if constexpr (sizeof(R) == 4) {
            if (vec) {
                // 16-byte column groups [cb, ce) inside [k + 1, hi], UV groups of four rows per lane in flight;
                // the ragged head [k + 1, cb) and tail [max(ce, cb), hi] (three columns at most each) column by
                // column.  A group that reaches past a shorter row stores that row's elements back unchanged.
                const int cb = min((k + 4) & ~3, hi + 1), ce = (hi + 1) & ~3;
                if (lane < 3 && k + 1 + lane < cb) col(k + 1 + lane);
                if (lane < 3 && max(ce, cb) + lane <= hi) col(max(ce, cb) + lane);
                const int nch = ce > cb ? (ce - cb) >> 2 : 0;
                for (int j0 = lane; j0 < nch; j0 += 32 * UV) {
                    float4 a[UV][4];
#pragma unroll
                    for (int u = 0; u < UV; ++u) {
                        const int j = j0 + 32 * u;
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (q < nr && j < nch && cb + 4 * j <= rq[q])
                                a[u][q] = *reinterpret_cast<const float4 *>(row[q] + cb + 4 * j);
                    }
#pragma unroll
                    for (int u = 0; u < UV; ++u) {
                        const int j = j0 + 32 * u;
                        if (j >= nch) break;
                        const int c = cb + 4 * j;
                        const float4 poc = *reinterpret_cast<const float4 *>(po + c);
                        const float4 voc = *reinterpret_cast<const float4 *>(vo + c);
                        const float4 vc = *reinterpret_cast<const float4 *>(v + c);
                        float4 cl = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (q < nr && c <= rq[q]) {
                                float4 x = a[u][q];
                                const int lim = rq[q] - c;   // elements c + e with e <= lim belong to the row
                                x.x = x.x - vr[q] * poc.x - pr[q] * voc.x;
                                acc[q] = fma(x.x, vc.x, acc[q]);
                                if (lim > 0) cl.x = fma(x.x, vq[q], cl.x);
                                if (lim >= 1) {
                                    x.y = x.y - vr[q] * poc.y - pr[q] * voc.y;
                                    acc[q] = fma(x.y, vc.y, acc[q]);
                                    if (lim > 1) cl.y = fma(x.y, vq[q], cl.y);
                                }
                                if (lim >= 2) {
                                    x.z = x.z - vr[q] * poc.z - pr[q] * voc.z;
                                    acc[q] = fma(x.z, vc.z, acc[q]);
                                    if (lim > 2) cl.z = fma(x.z, vq[q], cl.z);
                                }
                                if (lim >= 3) {
                                    x.w = x.w - vr[q] * poc.w - pr[q] * voc.w;
                                    acc[q] = fma(x.w, vc.w, acc[q]);
                                    if (lim > 3) cl.w = fma(x.w, vq[q], cl.w);
                                }
                                *reinterpret_cast<float4 *>(row[q] + c) = x;
                                if (c == k + 1) stash(rq[q], x.x);
                            }
                        // columns at or beyond the longest row's diagonal take no column sum
                        if (c < hi) atomicAdd(cs + c, cl.x);
                        if (c + 1 < hi) atomicAdd(cs + c + 1, cl.y);
                        if (c + 2 < hi) atomicAdd(cs + c + 2, cl.z);
                        if (c + 3 < hi) atomicAdd(cs + c + 3, cl.w);
                    }
                }
                vdone = true;
            }
        }
        if (!vdone) {
            for (int c = k + 1 + lane; c <= hi; c += 32) col(c);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (q >= nr) break;
            const R sum = warp_sum_t(acc[q]);
            if (lane == 0) p[rq[q]] = sum;   // the row sum; the column sums are added below
        }
    }
}

// ---------------------------------------------------------------------- 1. Householder tridiagonalisation
// A (n x n, lda; both triangles stored on input) overwritten; d, e (n), tau (n); reflector k stored in row k,
// columns k+1 .. n-1 (H_k = I - tau_k v v^T).  Only the lower triangle of the trailing matrix is read and written:
// the symmetric product A v takes every below-diagonal element twice, for its row sum (p_r) and for its column
// sum (p_c), which halves the memory traffic of the reduction.  Step k: (a) warp 0 of the owner of row k applies
// the pending update of step k-1 to column k of the trailing matrix (stashed by the previous pass; row 0 read
// directly at step 0) and forms v_k from it; (b) one pass over rows r > k, columns k+1 .. r, applies the pending
// update, accumulates the row sums of A v_k and scatters the column sums (one shared-memory add per column and
// group of four rows), and stashes column k+1; (c) p = tau (row + column sums), p -= (tau/2)(p.v) v; (v_k, p)
// become the pending update A <- A - v p^T - p v^T.  The upper part of row k holds the reflector: no later step
// reads it.
template <class R, int CL, int MINB>
__global__ void __launch_bounds__(kTT, MINB) k_tridiag(const TriDescT<R> *__restrict__ descs) {
    static_assert(CL == 1 || CL == 2, "one CTA or a pair of CTAs per matrix");
    const unsigned rank = CL == 2 ? cg::this_cluster().block_rank() : 0u;
    const TriDescT<R> D = descs[blockIdx.x / CL];
    const int n = D.n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ns = (n + 3) & ~3;   // vector stride: 16-byte aligned starts
    R *v = reinterpret_cast<R *>(smem_raw), *p = v + ns, *vo = p + ns, *po = vo + ns;   // global indices
    R *nx = po + ns;   // column k + 1 of the trailing matrix as pass (b) of step k leaves it (rows >= k + 1)
    R *cs = nx + ns;   // column sums of A v over this CTA's rows
    R *cq = cs + ns;   // (pair of CTAs) the peer's column sums for this CTA's rows
    __shared__ R part[kTT / 32];   // in the working precision: FP64 conversions and adds are slow on GB300
    __shared__ R s_beta[2], s_kc, s_pv[2];
    // cluster of two: the peer CTA's copy of a shared-memory location
    auto remote = [&](R *x) -> R * {
        if constexpr (CL == 2) return cg::this_cluster().map_shared_rank(x, rank ^ 1u);
        return x;
    };
    auto cluster_sync = [&]() {
        if constexpr (CL == 2) cg::this_cluster().sync();
    };
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int NW = kTT / 32;
    R *A = D.A;
    const long long lda = D.lda;
    const bool vec = (lda & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;   // 16-byte aligned rows
    for (int i = tid; i < n; i += kTT) {
        vo[i] = 0;
        po[i] = 0;
        cs[i] = 0;
    }
    __syncthreads();
    cluster_sync();   // both CTAs resident before the first remote store
    for (int k = 0; k + 2 < n; ++k) {
        // (a) column k with the pending update; reflector from its entries below the diagonal (formed by the CTA
        // that owns row k and copied into the peer's shared memory)
        if (wid == 0 && (CL == 1 || (unsigned)(k & 1) == rank)) {
            R *vr_ = remote(v);
            R *row = A + (long long)k * lda;
            const R vk = vo[k], pk = po[k];
            R ss = 0;
            for (int c = k + 1 + lane; c < n; c += 32) {
                const R x = (k == 0 ? row[c] : nx[c]) - vk * po[c] - pk * vo[c];
                v[c] = x;
                if (CL == 2 && c > k + 1) vr_[c] = x;
                ss = fma(x, x, ss);
            }
            ss = warp_sum_t(ss);
            if (lane == 0) {
                D.d[k] = (k == 0 ? row[0] : nx[k]) - 2 * vk * pk;
                const R x0 = v[k + 1];
                const R alpha = sqrt(ss);
                R beta = 0;
                if (alpha == (R)0) {
                    D.e[k] = 0;
                } else {
                    const R sgn = x0 >= (R)0 ? (R)1 : (R)-1;
                    v[k + 1] = x0 + sgn * alpha;
                    D.e[k] = -sgn * alpha;
                    beta = (R)1 / (alpha * (alpha + fabs(x0)));
                }
                D.tau[k] = beta;
                s_beta[k & 1] = beta;
                if constexpr (CL == 2) {
                    vr_[k + 1] = v[k + 1];
                    *remote(&s_beta[k & 1]) = beta;
                }
            }
            __syncwarp();
            for (int c = k + 1 + lane; c < n; c += 32) row[c] = v[c];   // reflector into row k
        }
        __syncthreads();
        cluster_sync();
        const R beta = s_beta[k & 1];
        // (b) pending update of the lower triangle of rows r > k fused with the row and column sums of A v; a warp
        // takes four rows at a time so that several independent loads are in flight per lane (rows r = rank
        // (mod CL): warp w takes the rows rstart + CL (w + NW q), q < 4, per pass)
        const int rstart = k + 1 + (int)((rank ^ (unsigned)(k + 1)) & (CL - 1));
        {
            R *nxr = remote(nx);
            tri_rows_pass<R, MINB == 2 ? 1 : 3>(A, lda, vec, k, n, rstart, CL, vo, po, v, cs, p, [&](int r, R x) {
                nx[r] = x;
                if (CL == 2) nxr[r] = x;
            });
        }
        __syncthreads();
        // (c) the peer's column sums for this CTA's rows, then p = beta (row + column sums) for this CTA's rows
        // (copied into the peer), p.v, and p -= (beta/2)(p.v) v over the whole vector
        if constexpr (CL == 2) {
            R *cqr = remote(cq);
            for (int c = k + 1 + tid; c < n; c += kTT)
                if ((unsigned)(c & 1) != rank) cqr[c] = cs[c];
            cluster_sync();
        }
        R pv = 0;
        {
            R *pr_ = remote(p);
            for (int c = k + 1 + tid; c < n; c += kTT) {
                if (CL == 1 || (unsigned)(c & 1) == rank) {
                    const R pc = beta * (p[c] + cs[c] + (CL == 2 ? cq[c] : (R)0));
                    p[c] = pc;
                    if (CL == 2) pr_[c] = pc;
                    pv = fma(pc, v[c], pv);
                }
                cs[c] = 0;   // ready for the next pass (the peer has its copy)
            }
        }
        pv = warp_sum_t(pv);
        if (lane == 0) part[wid] = pv;
        __syncthreads();
        if (wid == 0) {
            const R t = warp_sum_t(lane < NW ? part[lane] : (R)0);
            if (lane == 0) {
                if constexpr (CL == 2) {
                    s_pv[rank] = t;
                    *remote(&s_pv[rank]) = t;
                } else {
                    s_kc = (R)0.5 * beta * t;
                }
            }
        }
        __syncthreads();
        cluster_sync();
        const R kc = CL == 2 ? (R)0.5 * beta * (s_pv[0] + s_pv[1]) : s_kc;
        for (int r = k + 1 + tid; r < n; r += kTT) p[r] -= kc * v[r];
        __syncthreads();
        R *t = vo;
        vo = v;
        v = t;
        t = po;
        po = p;
        p = t;
    }
    cluster_sync();   // no remote access after this point; the peer's last row updates are visible
    if (tid == 0 && rank == 0) {
        if (n >= 2) {
            const int a = n - 2, b = n - 1;
            D.d[a] = A[(long long)a * lda + a] - 2 * vo[a] * po[a];
            D.e[a] = A[(long long)b * lda + a] - vo[b] * po[a] - po[b] * vo[a];
            D.d[b] = A[(long long)b * lda + b] - 2 * vo[b] * po[b];
            D.tau[a] = 0;
            A[(long long)a * lda + b] = 0;   // no reflector for the last two rows
        } else if (n == 1) {
            D.d[0] = A[0];
        }
        D.e[n - 1] = 0;
        D.tau[n - 1] = 0;
    }
}

// FP32 Householder reduction by a cluster of CL CTAs per matrix (CL = 4, 8 or 16; one CTA per SM).  Fewer matrices
// are in flight at once than with one CTA or a pair per matrix, so their trailing triangles fit in L2 and the pass
// of every step streams from L2 instead of HBM.  Row r belongs to CTA r mod CL.  Every CTA keeps full copies of v,
// p, vo, po and of the stashed column and forms the reflector itself from its copy: the same operations in the same
// order on the same values, hence the same bits on every CTA, so no reflector is sent.  The exchanges are the stash
// (each row's owner writes its element into every CTA), the column sums (each CTA gathers its peers' partial sums for
// its own rows), p (the owner of each entry writes it into every CTA) and the partial dot products p.v: two cluster
// barriers per step.  The stash is double-buffered by the parity of k, since a CTA may start the next pass while a
// peer still reads the previous column.  Results equal those of k_tridiag up to the order of the column sums.
template <int CL>
__global__ void __launch_bounds__(kTT, 1) k_tridiag_cl(const TriDescT<float> *__restrict__ descs) {
    using R = float;
    static_assert(CL == 4 || CL == 8 || CL == 16, "clusters of 4, 8 or 16 CTAs");
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    const TriDescT<R> D = descs[blockIdx.x / CL];
    const int n = D.n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ns = (n + 3) & ~3;
    R *v = reinterpret_cast<R *>(smem_raw), *p = v + ns, *vo = p + ns, *po = vo + ns;
    R *nxb = po + ns;        // two stashes: column k + 1 as pass (b) of step k leaves it, in nxb + (k & 1) ns
    R *cs = nxb + 2 * ns;    // column sums of A v over this CTA's rows
    __shared__ R part[kTT / 32];
    __shared__ R s_pv[CL];   // every CTA's partial p.v
    __shared__ R s_beta;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int NW = kTT / 32;
    // the same shared-memory location in CTA q of the cluster
    auto at = [&](R *x, unsigned q) -> R * { return cluster.map_shared_rank(x, q); };
    R *A = D.A;
    const long long lda = D.lda;
    const bool vec = (lda & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    for (int i = tid; i < n; i += kTT) {
        vo[i] = 0;
        po[i] = 0;
        cs[i] = 0;
    }
    __syncthreads();
    cluster.sync();   // every CTA resident and initialised before the first remote store
    for (int k = 0; k + 2 < n; ++k) {
        const bool own_k = (unsigned)(k & (CL - 1)) == rank;
        R *nx = nxb + (k & 1) * ns, *nxp = nxb + ((k + 1) & 1) * ns;   // written now, written by the last step
        // (a) column k with the pending update, from the stash (row 0 from memory at step 0), and the reflector;
        // every CTA alike, the owner of row k writes d, e and tau
        if (wid == 0) {
            const R *row = A + (long long)k * lda;
            const R vk = vo[k], pk = po[k];
            R ss = 0;
            for (int c = k + 1 + lane; c < n; c += 32) {
                const R x = (k == 0 ? row[c] : nxp[c]) - vk * po[c] - pk * vo[c];
                v[c] = x;
                ss = fma(x, x, ss);
            }
            ss = warp_sum_t(ss);
            if (lane == 0) {
                const R dk = (k == 0 ? row[0] : nxp[k]) - 2 * vk * pk;
                const R x0 = v[k + 1];
                const R alpha = sqrt(ss);
                R beta = 0, ek = 0;
                if (alpha != (R)0) {
                    const R sgn = x0 >= (R)0 ? (R)1 : (R)-1;
                    v[k + 1] = x0 + sgn * alpha;
                    ek = -sgn * alpha;
                    beta = (R)1 / (alpha * (alpha + fabs(x0)));
                }
                s_beta = beta;
                if (own_k) {
                    D.d[k] = dk;
                    D.e[k] = ek;
                    D.tau[k] = beta;
                }
            }
        }
        __syncthreads();
        const R beta = s_beta;
        // (b) this CTA's rows: pending update, row and column sums of A v, the new stash
        const int rstart = k + 1 + (((int)rank - (k + 1)) & (CL - 1));
        tri_rows_pass<R, 3>(A, lda, vec, k, n, rstart, CL, vo, po, v, cs, p, [&](int r, R x) { nx[r] = x; });
        __syncthreads();
        for (int r = rstart + CL * tid; r < n; r += CL * kTT) {
            const R x = nx[r];
#pragma unroll
            for (unsigned q = 1; q < CL; ++q) *at(nx + r, (rank + q) & (CL - 1)) = x;
        }
        cluster.sync();   // the column sums and the stash complete in every CTA; every (a) of step k done
        // (c) the owner of row k writes the reflector (no CTA reads row k any more); p = beta (row + column sums)
        // for this CTA's rows, into every CTA; the partial p.v into every CTA
        if (own_k)
            for (int c = k + 1 + tid; c < n; c += kTT) A[(long long)k * lda + c] = v[c];
        R pv = 0;
        for (int c = rstart + CL * tid; c < n; c += CL * kTT) {
            R t = p[c] + cs[c];
#pragma unroll
            for (unsigned q = 1; q < CL; ++q) t += *at(cs + c, (rank + q) & (CL - 1));
            const R pc = beta * t;
            p[c] = pc;
#pragma unroll
            for (unsigned q = 1; q < CL; ++q) *at(p + c, (rank + q) & (CL - 1)) = pc;
            pv = fma(pc, v[c], pv);
        }
        pv = warp_sum_t(pv);
        if (lane == 0) part[wid] = pv;
        __syncthreads();
        if (wid == 0) {
            const R t = warp_sum_t(lane < NW ? part[lane] : (R)0);
            if (lane < CL) *at(s_pv + rank, (unsigned)lane) = t;
        }
        cluster.sync();   // p and the partial dot products complete in every CTA; no peer reads cs any more
        R tpv = 0;
#pragma unroll
        for (int q = 0; q < CL; ++q) tpv += s_pv[q];   // the same order in every CTA
        const R kc = (R)0.5 * beta * tpv;
        for (int r = k + 1 + tid; r < n; r += kTT) {
            p[r] -= kc * v[r];
            cs[r] = 0;
        }
        __syncthreads();
        R *t = vo;
        vo = v;
        v = t;
        t = po;
        po = p;
        p = t;
    }
    cluster.sync();   // the last row updates of every CTA visible
    if (tid == 0 && rank == 0) {
        if (n >= 2) {
            const int a = n - 2, b = n - 1;
            D.d[a] = A[(long long)a * lda + a] - 2 * vo[a] * po[a];
            D.e[a] = A[(long long)b * lda + a] - vo[b] * po[a] - po[b] * vo[a];
            D.d[b] = A[(long long)b * lda + b] - 2 * vo[b] * po[b];
            D.tau[a] = 0;
            A[(long long)a * lda + b] = 0;
        } else if (n == 1) {
            D.d[0] = A[0];
        }
        D.e[n - 1] = 0;
        D.tau[n - 1] = 0;
    }
}

// FP32 Householder reduction with delayed updates (one CTA per matrix).  The rank-2 updates
// A <- A - v_s p_s^T - p_s v_s^T of NB consecutive steps are written into the stored lower triangle together, by the
// pass of every NB-th step (a flush pass, which applies them element by element while it forms A v).  The passes in
// between only read the stored triangle and correct its product with v for the updates still pending:
// A v = A_stored v - sum_s [v_s (p_s . v) + p_s (v_s . v)].  Every element is still read once per step but written
// once per NB steps, so the bytes moved fall to (NB + 1) / 2NB of the reduction above.  The last NB + 1 pairs
// (v_s, p_s) live in a ring in shared memory (slot s mod (NB + 1)); column k + 1 as the pass leaves it in memory is
// stashed, and step k + 1 applies to it the updates not yet written.
struct TriPend {   // the pending pairs a flush pass applies
    const float *v[4], *p[4];
};

__device__ __forceinline__ float &f4c(float4 &x, int e) { return e == 0 ? x.x : e == 1 ? x.y : e == 2 ? x.z : x.w; }

template <int UV, int NP, bool WRITE, int RW = 4>
__device__ __forceinline__ void tri_rows_pass_d(float *__restrict__ A, long long lda, bool vec, int k, int n,
                                                const TriPend &P, const float *__restrict__ v, float *cs, float *p,
                                                float *nx) {
    constexpr int NW = kTT / 32;
    constexpr int NX = NP > 0 ? NP : 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int r0 = k + 1 + wid; r0 < n; r0 += RW * NW) {
        // rows r0 + q NW, q < nr <= RW (row q's columns c <= r0 + q NW)
        float *row0 = A + (long long)r0 * lda;
        const long long rstep = (long long)NW * lda;
        const int nr = min(RW, (n - 1 - r0) / NW + 1);
        float vq[RW], acc[RW], vr[RW][NX], pr[RW][NX];
#pragma unroll
        for (int q = 0; q < RW; ++q) {
            const int r = q < nr ? r0 + q * NW : r0;
            vq[q] = q < nr ? v[r] : 0.f;
            acc[q] = 0.f;
#pragma unroll
            for (int s = 0; s < NX; ++s) {
                vr[q][s] = NP > 0 && q < nr ? P.v[s][r] : 0.f;
                pr[q][s] = NP > 0 && q < nr ? P.p[s][r] : 0.f;
            }
        }
        const int hi = r0 + (nr - 1) * NW;   // the group's longest row
        // element (row q, column c): the pending updates applied, the row and column sums taken
        auto elem = [&](float x, int q, int c, const float *pce, const float *wce, float vce, float &cl) -> float {
#pragma unroll
            for (int s = 0; s < NP; ++s) x = x - vr[q][s] * pce[s] - pr[q][s] * wce[s];
            acc[q] = fma(x, vce, acc[q]);
            if (c < r0 + q * NW) cl = fma(x, vq[q], cl);
            return x;
        };
        auto col = [&](int c) {   // one column of the (up to) four rows
            float pce[NX], wce[NX];
#pragma unroll
            for (int s = 0; s < NX; ++s) {
                pce[s] = NP > 0 ? P.p[s][c] : 0.f;
                wce[s] = NP > 0 ? P.v[s][c] : 0.f;
            }
            const float vce = v[c];
            float cl = 0.f;
#pragma unroll
            for (int q = 0; q < RW; ++q)
                if (q < nr && c <= r0 + q * NW) {
                    float *rp = row0 + q * rstep + c;
                    const float x = elem(*rp, q, c, pce, wce, vce, cl);
                    if (WRITE) *rp = x;
                    if (c == k + 1) nx[r0 + q * NW] = x;
                }
            if (c < hi) atomicAdd(cs + c, cl);
        };
        if (vec) {
            // 16-byte column groups [cb, ce) inside [k + 1, hi]; the ragged head and tail column by column
            const int cb = min((k + 4) & ~3, hi + 1), ce = (hi + 1) & ~3;
            if (lane < 3 && k + 1 + lane < cb) col(k + 1 + lane);
            if (lane < 3 && max(ce, cb) + lane <= hi) col(max(ce, cb) + lane);
            const int nch = ce > cb ? (ce - cb) >> 2 : 0;
            for (int j0 = lane; j0 < nch; j0 += 32 * UV) {
                float4 a[UV][RW];
#pragma unroll
                for (int u = 0; u < UV; ++u) {
                    const int j = j0 + 32 * u;
#pragma unroll
                    for (int q = 0; q < RW; ++q)
                        if (q < nr && j < nch && cb + 4 * j <= r0 + q * NW)
                            a[u][q] = *reinterpret_cast<const float4 *>(row0 + q * rstep + cb + 4 * j);
                }
#pragma unroll
                for (int u = 0; u < UV; ++u) {
                    const int j = j0 + 32 * u;
                    if (j >= nch) break;
                    const int c = cb + 4 * j;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {   // column c + e
                        float pce[NX], wce[NX];
#pragma unroll
                        for (int s = 0; s < NX; ++s) {
                            pce[s] = NP > 0 ? P.p[s][c + e] : 0.f;
                            wce[s] = NP > 0 ? P.v[s][c + e] : 0.f;
                        }
                        const float vce = v[c + e];
                        float cl = 0.f;
#pragma unroll
                        for (int q = 0; q < RW; ++q)
                            if (q < nr && c + e <= r0 + q * NW) f4c(a[u][q], e) = elem(f4c(a[u][q], e), q, c + e, pce, wce, vce, cl);
                        // columns at or beyond the longest row's diagonal take no column sum
                        if (c + e < hi) atomicAdd(cs + c + e, cl);
                    }
#pragma unroll
                    for (int q = 0; q < RW; ++q)
                        if (q < nr && c <= r0 + q * NW) {
                            if (WRITE) *reinterpret_cast<float4 *>(row0 + q * rstep + c) = a[u][q];
                            if (c == k + 1) nx[r0 + q * NW] = a[u][q].x;
                        }
                }
            }
        } else {
            for (int c = k + 1 + lane; c <= hi; c += 32) col(c);
        }
#pragma unroll
        for (int q = 0; q < RW; ++q) {
            if (q >= nr) break;
            const float sum = warp_sum_t(acc[q]);
            if (lane == 0) p[r0 + q * NW] = sum;   // the row sum; the column sums are added below
        }
    }
}

// Geometry of one row group of pass (b): rows r0 + q NW (q < nr), the group's longest row hi, its 16-byte column
// groups [cb, ce) (nch of them) and their chunks of 32 (one per lane: njb chunks).
struct TriGroup {
    int nr, hi, cb, ce, nch, njb;
};
__device__ __forceinline__ TriGroup tri_group(int r0, int k, int n, int rw, int nw) {
    TriGroup g;
    g.nr = min(rw, (n - 1 - r0) / nw + 1);
    g.hi = r0 + (g.nr - 1) * nw;
    g.cb = min((k + 4) & ~3, g.hi + 1);
    g.ce = (g.hi + 1) & ~3;
    g.nch = g.ce > g.cb ? (g.ce - g.cb) >> 2 : 0;
    g.njb = (g.nch + 31) >> 5;
    return g;
}

// 16-byte global -> shared copy in flight (src_bytes = 0: zero fill, nothing read)
__device__ __forceinline__ void tri_cp16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void tri_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void tri_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// tri_rows_pass_d with the 16-byte row chunks staged through shared memory: every lane copies its next NSL - 1
// chunks of the RW rows (cp.async, into an NSL-slot ring of its own) while it works on the current one, so more
// loads are in flight without registers to hold them.  The copy cursor walks the warp's row groups and chunks in the
// order of the work; a chunk being copied is never one the pass writes before it is consumed.  16-byte aligned
// rows only (vec); stage: this warp's NSL x 4 x 32 float4.
template <int NP, bool WRITE, int RW, int NSL, bool V4, int SR = 4>
__device__ __forceinline__ void tri_rows_pass_staged(float *__restrict__ A, long long lda, int k, int n,
                                                     const TriPend &P, const float *__restrict__ v, float *cs,
                                                     float *p, float *nx, float4 *stage) {
    constexpr int NW = kTT / 32;
    constexpr int NX = NP > 0 ? NP : 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gstep = RW * NW;
    // copy cursor: group pr0, chunk pjb (past the end once pr0 >= n)
    int pr0 = k + 1 + wid, pjb = 0;
    TriGroup pg = pr0 < n ? tri_group(pr0, k, n, RW, NW) : TriGroup{0, 0, 0, 0, 0, 0};
    auto skip_empty = [&]() {
        while (pr0 < n && pjb >= pg.njb) {
            pr0 += gstep;
            pjb = 0;
            if (pr0 < n) pg = tri_group(pr0, k, n, RW, NW);
        }
    };
    skip_empty();
    auto issue = [&](int slot) {   // the cursor's chunk into this lane's slot (an empty group past the end)
        if (pr0 < n) {
            const int j = pjb * 32 + lane;
#pragma unroll
            for (int q = 0; q < RW; ++q) {
                const int r = pr0 + q * NW;
                const bool ok = q < pg.nr && j < pg.nch && pg.cb + 4 * j <= r;
                tri_cp16(stage + (slot * SR + q) * 32 + lane, ok ? A + (long long)r * lda + pg.cb + 4 * j : A,
                         ok ? 16 : 0);
            }
            ++pjb;
            skip_empty();
        }
        tri_cp_commit();
    };
    int slot = 0, islot = NSL - 1;   // the slot consumed next, the slot filled next
#pragma unroll
    for (int t = 0; t < NSL - 1; ++t) issue(t);
    for (int r0 = k + 1 + wid; r0 < n; r0 += gstep) {
        const TriGroup g = tri_group(r0, k, n, RW, NW);
        float *row0 = A + (long long)r0 * lda;
        const long long rstep = (long long)NW * lda;
        const int nr = g.nr, hi = g.hi;
        float vq[RW], acc[RW], vr[RW][NX], pr[RW][NX];
#pragma unroll
        for (int q = 0; q < RW; ++q) {
            const int r = q < nr ? r0 + q * NW : r0;
            vq[q] = q < nr ? v[r] : 0.f;
            acc[q] = 0.f;
#pragma unroll
            for (int s = 0; s < NX; ++s) {
                vr[q][s] = NP > 0 && q < nr ? P.v[s][r] : 0.f;
                pr[q][s] = NP > 0 && q < nr ? P.p[s][r] : 0.f;
            }
        }
        auto elem = [&](float x, int q, int c, const float *pce, const float *wce, float vce, float &cl) -> float {
#pragma unroll
            for (int s = 0; s < NP; ++s) x = x - vr[q][s] * pce[s] - pr[q][s] * wce[s];
            acc[q] = fma(x, vce, acc[q]);
            if (c < r0 + q * NW) cl = fma(x, vq[q], cl);
            return x;
        };
        auto col = [&](int c) {   // one column of the (up to) RW rows, straight from memory
            float pce[NX], wce[NX];
#pragma unroll
            for (int s = 0; s < NX; ++s) {
                pce[s] = NP > 0 ? P.p[s][c] : 0.f;
                wce[s] = NP > 0 ? P.v[s][c] : 0.f;
            }
            const float vce = v[c];
            float cl = 0.f;
#pragma unroll
            for (int q = 0; q < RW; ++q)
                if (q < nr && c <= r0 + q * NW) {
                    float *rp = row0 + q * rstep + c;
                    const float x = elem(*rp, q, c, pce, wce, vce, cl);
                    if (WRITE) *rp = x;
                    if (c == k + 1) nx[r0 + q * NW] = x;
                }
            if (c < hi) atomicAdd(cs + c, cl);
        };
        // the ragged head [k + 1, cb) and tail [max(ce, cb), hi] column by column (outside every staged chunk)
        if (lane < 3 && k + 1 + lane < g.cb) col(k + 1 + lane);
        if (lane < 3 && max(g.ce, g.cb) + lane <= hi) col(max(g.ce, g.cb) + lane);
        for (int jb = 0; jb < g.njb; ++jb) {
            issue(islot);       // the slot consumed one chunk ago
            islot = islot + 1 == NSL ? 0 : islot + 1;
            tri_cp_wait<NSL - 1>();   // this lane's copies of the current chunk have landed
            const int j = jb * 32 + lane;
            if (j < g.nch) {
                const int c = g.cb + 4 * j;
                float4 a[RW];
#pragma unroll
                for (int q = 0; q < RW; ++q) a[q] = stage[(slot * SR + q) * 32 + lane];
                // V4: the group's four entries of v and of the pending pairs as one 16-byte load each (lanes' groups
                // are 16 bytes apart: no bank conflicts; column-wise scalar loads would collide four ways)
                float4 v4, p4[NX], w4[NX];
                if constexpr (V4) {
                    v4 = *reinterpret_cast<const float4 *>(v + c);
#pragma unroll
                    for (int s = 0; s < NX; ++s) {
                        p4[s] = NP > 0 ? *reinterpret_cast<const float4 *>(P.p[s] + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                        w4[s] = NP > 0 ? *reinterpret_cast<const float4 *>(P.v[s] + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {   // column c + e
                    float pce[NX], wce[NX];
#pragma unroll
                    for (int s = 0; s < NX; ++s) {
                        pce[s] = NP > 0 ? (V4 ? f4c(p4[s], e) : P.p[s][c + e]) : 0.f;
                        wce[s] = NP > 0 ? (V4 ? f4c(w4[s], e) : P.v[s][c + e]) : 0.f;
                    }
                    const float vce = V4 ? f4c(v4, e) : v[c + e];
                    float cl = 0.f;
#pragma unroll
                    for (int q = 0; q < RW; ++q)
                        if (q < nr && c + e <= r0 + q * NW) f4c(a[q], e) = elem(f4c(a[q], e), q, c + e, pce, wce, vce, cl);
                    // columns at or beyond the longest row's diagonal take no column sum
                    if (c + e < hi) atomicAdd(cs + c + e, cl);
                }
#pragma unroll
                for (int q = 0; q < RW; ++q)
                    if (q < nr && c <= r0 + q * NW) {
                        if (WRITE) *reinterpret_cast<float4 *>(row0 + q * rstep + c) = a[q];
                        if (c == k + 1) nx[r0 + q * NW] = a[q].x;
                    }
            }
            slot = slot + 1 == NSL ? 0 : slot + 1;
        }
#pragma unroll
        for (int q = 0; q < RW; ++q) {
            if (q >= nr) break;
            const float sum = warp_sum_t(acc[q]);
            if (lane == 0) p[r0 + q * NW] = sum;   // the row sum; the column sums are added below
        }
    }
    tri_cp_wait<0>();   // nothing in flight past the pass
}

template <int NB, int MINB, int NSL = 0, int RWS = 4>
__global__ void __launch_bounds__(kTT, MINB) k_tridiag_delayed(const TriDescT<float> *__restrict__ descs) {
    static_assert(NB >= 2 && NB <= 4, "two to four updates per flush");
    constexpr int NS = NB + 1;                     // ring slots
    constexpr int UVF = 1, UVR = MINB == 2 ? 1 : (NB == 4 ? 2 : 3);   // register budgets without spills (NB = 2, one CTA per SM)
    const TriDescT<float> D = descs[blockIdx.x];
    const int n = D.n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ns = (n + 3) & ~3;
    float *Vr = reinterpret_cast<float *>(smem_raw);   // v_s of the ring
    float *Pr = Vr + NS * ns;                          // p_s of the ring
    float *nx = Pr + NS * ns;                          // column k + 1 as the pass of step k leaves it in memory
    float *cs = nx + ns;                               // column sums of A v
    // (NSL > 0) each warp's ring of row chunks, NSL x RWS x 32 float4
    float4 *stage = reinterpret_cast<float4 *>(cs + ns) + (threadIdx.x >> 5) * (NSL * RWS * 32);
    {
        // launched with less dynamic shared memory than the ring needs: report a non-finite tridiagonal instead of
        // touching memory past the allocation (the whole block returns before any barrier)
        unsigned dsm;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsm));
        if ((size_t)dsm < (size_t)(2 * NS + 2) * ns * sizeof(float) + (size_t)(kTT / 32) * NSL * RWS * 32 * 16) {
            if (threadIdx.x == 0) D.d[0] = __int_as_float(0x7fc00000);
            return;
        }
    }
    __shared__ float part[kTT / 32][2 * NB];
    __shared__ float s_dot[2 * NB];
    __shared__ float s_beta, s_kc;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int NW = kTT / 32;
    auto vs = [&](int s) -> float * { return Vr + (((s % NS) + NS) % NS) * ns; };
    auto ps = [&](int s) -> float * { return Pr + (((s % NS) + NS) % NS) * ns; };
    float *A = D.A;
    const long long lda = D.lda;
    const bool vec = (lda & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    for (int i = tid; i < (2 * NS + 2) * ns; i += kTT) Vr[i] = 0.f;   // the ring, the stash and the column sums
    __syncthreads();
    for (int k = 0; k + 2 < n; ++k) {
        float *v = vs(k), *p = ps(k);
        const int mc = k == 0 ? 0 : (k - 1) % NB + 1;   // updates of steps k - mc .. k - 1 not yet in the stash
        // (a) column k with the updates not yet written, and its reflector (warp 0)
        if (wid == 0) {
            float *row = A + (long long)k * lda;
            float ss = 0.f;
            for (int c = k + 1 + lane; c < n; c += 32) {
                float x = k == 0 ? row[c] : nx[c];
                for (int t = 1; t <= mc; ++t) {
                    const float *vv = vs(k - t), *pp = ps(k - t);
                    x = x - vv[k] * pp[c] - pp[k] * vv[c];
                }
                v[c] = x;
                ss = fma(x, x, ss);
            }
            ss = warp_sum_t(ss);
            if (lane == 0) {
                float dk = k == 0 ? row[0] : nx[k];
                for (int t = 1; t <= mc; ++t) dk -= 2.f * vs(k - t)[k] * ps(k - t)[k];
                D.d[k] = dk;
                const float x0 = v[k + 1];
                const float alpha = sqrtf(ss);
                float beta = 0.f;
                if (alpha == 0.f) {
                    D.e[k] = 0.f;
                } else {
                    const float sgn = x0 >= 0.f ? 1.f : -1.f;
                    v[k + 1] = x0 + sgn * alpha;
                    D.e[k] = -sgn * alpha;
                    beta = 1.f / (alpha * (alpha + fabsf(x0)));
                }
                D.tau[k] = beta;
                s_beta = beta;
            }
            __syncwarp();
            for (int c = k + 1 + lane; c < n; c += 32) row[c] = v[c];   // reflector into row k
        }
        __syncthreads();
        const float beta = s_beta;
        const bool flush = k % NB == 0;
        const int m = flush ? 0 : k % NB;   // updates of steps k - m .. k - 1 missing from the stored triangle
        // (b) one pass over the rows r > k: a flush applies and writes the updates of steps k - NB .. k - 1
        if (flush) {
            TriPend P{};
#pragma unroll
            for (int s = 0; s < NB; ++s) {
                P.v[s] = vs(k - 1 - s);
                P.p[s] = ps(k - 1 - s);
            }
            if (NSL > 0 && vec)
                tri_rows_pass_staged<NB, true, MINB == 2 ? 2 : (RWS > 4 ? 4 : RWS), NSL, MINB == 1, RWS>(A, lda, k, n, P, v, cs, p, nx,
                                                                                       stage);
            else tri_rows_pass_d<UVF, NB, true, MINB == 2 ? 2 : 4>(A, lda, vec, k, n, P, v, cs, p, nx);
        } else {
            const TriPend P{};
            if (NSL > 0 && vec) tri_rows_pass_staged<0, false, RWS, NSL, MINB == 1, RWS>(A, lda, k, n, P, v, cs, p, nx, stage);
            else tri_rows_pass_d<UVR, 0, false>(A, lda, vec, k, n, P, v, cs, p, nx);
            // the dot products p_s . v and v_s . v of the missing updates
            float dl[2 * NB];
#pragma unroll
            for (int t = 0; t < 2 * NB; ++t) dl[t] = 0.f;
            for (int c = k + 1 + tid; c < n; c += kTT) {
                const float vc = v[c];
#pragma unroll
                for (int t = 0; t < NB; ++t)
                    if (t < m) {
                        dl[2 * t] = fma(ps(k - 1 - t)[c], vc, dl[2 * t]);
                        dl[2 * t + 1] = fma(vs(k - 1 - t)[c], vc, dl[2 * t + 1]);
                    }
            }
#pragma unroll
            for (int t = 0; t < 2 * NB; ++t) {
                const float x = warp_sum_t(dl[t]);
                if (lane == 0) part[wid][t] = x;
            }
        }
        __syncthreads();
        if (!flush) {
            if (wid == 0)
                for (int t = 0; t < 2 * m; ++t) {
                    const float x = warp_sum_t(lane < NW ? part[lane][t] : 0.f);
                    if (lane == 0) s_dot[t] = x;
                }
            __syncthreads();
        }
        // (c) p = beta (A v) with the correction for the missing updates, p.v, p -= (beta/2)(p.v) v
        float pv = 0.f;
        for (int c = k + 1 + tid; c < n; c += kTT) {
            float y = p[c] + cs[c];
            for (int t = 0; t < m; ++t) y -= vs(k - 1 - t)[c] * s_dot[2 * t] + ps(k - 1 - t)[c] * s_dot[2 * t + 1];
            const float pc = beta * y;
            p[c] = pc;
            pv = fma(pc, v[c], pv);
            cs[c] = 0.f;   // ready for the next pass
        }
        pv = warp_sum_t(pv);
        if (lane == 0) part[wid][0] = pv;
        __syncthreads();
        if (wid == 0) {
            const float t = warp_sum_t(lane < NW ? part[lane][0] : 0.f);
            if (lane == 0) s_kc = 0.5f * beta * t;
        }
        __syncthreads();
        const float kc = s_kc;
        for (int r = k + 1 + tid; r < n; r += kTT) p[r] -= kc * v[r];
        __syncthreads();
    }
    // the last two rows: their stored values and the updates not yet written (steps kl - kl % NB .. kl, kl = n - 3)
    if (tid == 0) {
        if (n >= 2) {
            const int a = n - 2, b = n - 1;
            float da = A[(long long)a * lda + a], ea = A[(long long)b * lda + a], db = A[(long long)b * lda + b];
            if (n >= 3) {
                const int kl = n - 3;
                for (int s = kl - kl % NB; s <= kl; ++s) {
                    const float *vv = vs(s), *pp = ps(s);
                    da -= 2.f * vv[a] * pp[a];
                    ea -= vv[b] * pp[a] + pp[b] * vv[a];
                    db -= 2.f * vv[b] * pp[b];
                }
            }
            D.d[a] = da;
            D.e[a] = ea;
            D.d[b] = db;
            D.tau[a] = 0.f;
            A[(long long)a * lda + b] = 0.f;   // no reflector for the last two rows
        } else if (n == 1) {
            D.d[0] = A[0];
        }
        D.e[n - 1] = 0.f;
        D.tau[n - 1] = 0.f;
    }
}

// ------------------------------------------------------------------------------------- 2. multisection
// Number of eigenvalues below x: sign changes of the leading principal minors p_i = det(T_0..i - x), computed by
// the three-term recurrence p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (no division).  Every four steps both
// carried minors are rescaled by an exact power of two, which keeps them finite without changing any sign.
// pivmin stands in for an exactly zero minor.
__device__ __forceinline__ int sturm_below(const double *d, const double *e2, int n, double x, double pivmin) {
    double pm = 1.0, pc = d[0] - x;
    if (pc == 0.0) pc = -pivmin;
    int cnt = pc < 0.0;
    for (int i = 1; i < n; ++i) {
        double pn = fma(d[i] - x, pc, -e2[i - 1] * pm);
        if (pn == 0.0) pn = (pc < 0.0 ? pivmin : -pivmin) * fabs(pc);   // treat as a tiny value of opposite sign
        cnt += (pn < 0.0) != (pc < 0.0);
        pm = pc;
        pc = pn;
        if ((i & 3) == 0) {
            const double a = fabs(pc);
            if (a > 0x1p+600) {
                pc *= 0x1p-600;
                pm *= 0x1p-600;
            } else if (a < 0x1p-600) {
                pc *= 0x1p+600;
                pm *= 0x1p+600;
            }
        }
    }
    return cnt;
}

// The cnt largest eigenvalues of each tridiagonal (decreasing, into w).  Warp j of the grid's y-range finds the
// j-th largest: each round the 32 lanes count at 32 interior points of the current bracket, and the bracket
// shrinks to the sub-interval where the count passes the target (33x per round).
constexpr int kMsWarps = 8;
template <class R>
__global__ void __launch_bounds__(kMsWarps * 32) k_tri_multisect(const TriDescT<R> *__restrict__ descs, int cnt) {
    const TriDescT<R> D = descs[blockIdx.x];
    const int n = D.n;
    extern __shared__ double shd[];
    double *d = shd, *e2 = shd + n;
    __shared__ double s_lo, s_hi;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        d[i] = (double)D.d[i];
        const double ei = (double)D.e[i];
        e2[i] = ei * ei;
    }
    __syncthreads();
    if (threadIdx.x < 32) {   // Gershgorin bracket
        double lo = DBL_MAX, hi = -DBL_MAX;
        for (int i = threadIdx.x; i < n; i += 32) {
            const double r = (i > 0 ? fabs((double)D.e[i - 1]) : 0.0) + (i + 1 < n ? fabs((double)D.e[i]) : 0.0);
            lo = fmin(lo, d[i] - r);
            hi = fmax(hi, d[i] + r);
        }
        lo = -warp_max(-lo);
        hi = warp_max(hi);
        if (threadIdx.x == 0) {
            const double span = fmax(hi - lo, fmax(fabs(lo), fabs(hi)));
            s_lo = lo - 2.0 * DBL_EPSILON * span - 1e-300;
            s_hi = hi + 2.0 * DBL_EPSILON * span + 1e-300;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.y * kMsWarps + (threadIdx.x >> 5);
    if (j >= cnt || j >= n) return;
    const int kk = n - 1 - j;   // j-th largest = kk-th smallest (0-based)
    const double pivmin = 1e-30;
    double lo = s_lo, hi = s_hi;
    for (int round = 0; round < 48; ++round) {
        const double width = hi - lo;
        if (!(width > 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 1e-300)) break;
        const double x = fma(width, (double)(lane + 1) / 33.0, lo);
        const unsigned below = __ballot_sync(0xffffffffu, sturm_below(d, e2, n, x, pivmin) <= kk);
        // lanes 0..f-1 have count <= kk (x <= lambda), lane f the first with count > kk
        const int f = below == 0xffffffffu ? 32 : __ffs(~below) - 1;
        const double nlo = f > 0 ? fma(width, (double)f / 33.0, lo) : lo;
        const double nhi = f < 32 ? fma(width, (double)(f + 1) / 33.0, lo) : hi;
        if (!(nlo > lo || nhi < hi)) break;   // no progress left at this precision
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) D.w[j] = (R)(0.5 * (lo + hi));
}

// FP32 counterpart for the FP32 tridiagonal (the first stage of the mixed path only needs FP32-accurate
// eigenvalues): d and e^2 are pre-scaled by the Gershgorin bound so every factor is <= 1 in magnitude, and the
// carried minors are rescaled by 2^+-40 at every step (exact, sign-preserving) to stay inside FP32 range.
__device__ __forceinline__ int sturm_below_f32(const float *d, const float *e2, int n, float x, float pivmin) {
    float pm = 1.f, pc = d[0] - x;
    if (pc == 0.f) pc = -pivmin;
    int cnt = pc < 0.f;
    for (int i = 1; i < n; ++i) {
        float pn = fmaf(d[i] - x, pc, -e2[i - 1] * pm);
        if (pn == 0.f) pn = (pc < 0.f ? pivmin : -pivmin) * fabsf(pc);
        cnt += (pn < 0.f) != (pc < 0.f);
        pm = pc;
        pc = pn;
        const float a = fabsf(pc);
        if (a > 0x1p+40f) {
            pc *= 0x1p-40f;
            pm *= 0x1p-40f;
        } else if (a < 0x1p-40f) {
            pc *= 0x1p+40f;
            pm *= 0x1p+40f;
        }
    }
    return cnt;
}

__global__ void __launch_bounds__(kMsWarps * 32) k_tri_multisect32(const TriDesc32 *__restrict__ descs, int cnt) {
    const TriDesc32 D = descs[blockIdx.x];
    const int n = D.n;
    extern __shared__ float shf[];
    float *d = shf, *e2 = shf + n;
    __shared__ float s_lo, s_hi, s_scale;
    if (threadIdx.x < 32) {   // Gershgorin bracket and scale
        float lo = FLT_MAX, hi = -FLT_MAX;
        for (int i = threadIdx.x; i < n; i += 32) {
            const float r = (i > 0 ? fabsf(D.e[i - 1]) : 0.f) + (i + 1 < n ? fabsf(D.e[i]) : 0.f);
            lo = fminf(lo, D.d[i] - r);
            hi = fmaxf(hi, D.d[i] + r);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (threadIdx.x == 0) {
            const float sc = fmaxf(fmaxf(fabsf(lo), fabsf(hi)), 1e-30f);
            s_scale = sc;
            s_lo = lo / sc - 4.f * FLT_EPSILON;
            s_hi = hi / sc + 4.f * FLT_EPSILON;
        }
    }
    __syncthreads();
    const float inv = 1.f / s_scale;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        d[i] = D.d[i] * inv;
        const float ei = D.e[i] * inv;
        e2[i] = ei * ei;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.y * kMsWarps + (threadIdx.x >> 5);
    if (j >= cnt || j >= n) return;
    const int kk = n - 1 - j;
    float lo = s_lo, hi = s_hi;
    for (int round = 0; round < 24; ++round) {
        const float width = hi - lo;
        if (!(width > 2.f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi)) + 1e-30f)) break;
        const float x = fmaf(width, (float)(lane + 1) / 33.f, lo);
        const unsigned below = __ballot_sync(0xffffffffu, sturm_below_f32(d, e2, n, x, 1e-30f) <= kk);
        const int f = below == 0xffffffffu ? 32 : __ffs(~below) - 1;
        const float nlo = f > 0 ? fmaf(width, (float)f / 33.f, lo) : lo;
        const float nhi = f < 32 ? fmaf(width, (float)(f + 1) / 33.f, lo) : hi;
        if (!(nlo > lo || nhi < hi)) break;
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) D.w[j] = 0.5f * (lo + hi) * s_scale;
}

// ------------------------------------------------------------ pivoted tridiagonal solve (one thread)
// Solves (Tri - shift) x = rhs.  Work arrays u0,u1,u2 (U rows: diagonal, first and second super-diagonal) and
// the right-hand side / solution x live in global memory at stride `st` (interleaved across threads).
template <class R>
__device__ void tri_solve(const R *d, const R *e, int n, R shift, R *x, R *u0, R *u1, R *u2, long long st,
                          R pivmin) {
    // current row i as (p, q) on columns i, i+1 (no fill yet), rhs in x
    // the eliminated rhs entry of row i is carried in xi (row i + 1 is still the original when it is read)
    R p = d[0] - shift, q = n > 1 ? e[0] : (R)0;
    R xi = x[0];
    for (int i = 0; i + 1 < n; ++i) {
        const R l = e[i];                        // entry (i+1, i)
        const R a = d[i + 1] - shift;            // (i+1, i+1)
        const R b = i + 2 < n ? e[i + 1] : (R)0; // (i+1, i+2)
        const R xn = x[(long long)(i + 1) * st];
        if (fabs(p) >= fabs(l)) {
            if (fabs(p) < pivmin) p = p < (R)0 ? -pivmin : pivmin;
            const R mlt = l / p;
            u0[(long long)i * st] = p;
            u1[(long long)i * st] = q;
            u2[(long long)i * st] = 0;
            x[(long long)i * st] = xi;
            xi = xn - mlt * xi;
            p = a - mlt * q;
            q = b;
        } else {
            const R mlt = p / l;
            u0[(long long)i * st] = l;
            u1[(long long)i * st] = a;
            u2[(long long)i * st] = b;
            x[(long long)i * st] = xn;
            xi = xi - mlt * xn;
            p = q - mlt * a;
            q = -mlt * b;
        }
    }
    if (fabs(p) < pivmin) p = p < (R)0 ? -pivmin : pivmin;
    u0[(long long)(n - 1) * st] = p;
    // back substitution
    R x1 = xi / p, x2 = 0;
    x[(long long)(n - 1) * st] = x1;
    for (int i = n - 2; i >= 0; --i) {
        const R xi = (x[(long long)i * st] - u1[(long long)i * st] * x1 - u2[(long long)i * st] * x2) /
                     u0[(long long)i * st];
        x[(long long)i * st] = xi;
        x2 = x1;
        x1 = xi;
    }
}

template <class R>
__device__ R tri_pivmin(const R *d, const R *e, int n) {
    R tnorm = 0;
    for (int i = 0; i < n; ++i) tnorm = fmax(tnorm, fabs(d[i]) + fabs(e[i]) + (i ? fabs(e[i - 1]) : (R)0));
    return fmax(tnorm, Lim<R>::tiny) * Lim<R>::eps * (R)1e-3;
}

// Per-CTA staging of the solves below: the tridiagonal (d, e) in shared memory and, when the launcher passes
// work == nullptr, each thread's four length-n work columns too (stride blockDim.x), so that the dependent
// chain of a solve waits on shared-memory latency instead of L2.  Returns d; e follows it.
template <class R>
__device__ R *stage_tri(const TriDescT<R> &D, R *sm) {
    for (int i = threadIdx.x; i < D.n; i += blockDim.x) {
        sm[i] = D.d[i];
        sm[D.n + i] = D.e[i];
    }
    __syncthreads();
    return sm;
}

// work columns of thread t: x, u0, u1, u2 and their stride
template <class R>
struct TriWork {
    R *x, *u0, *u1, *u2;
    long long st;
};
template <class R>
__device__ TriWork<R> tri_work(R *sm, int n, R *work, int b, int nmax, int mu) {
    if (work) {
        R *base = work + (long long)b * 4 * n * nmax + mu;
        return {base, base + (long long)n * nmax, base + 2LL * n * nmax, base + 3LL * n * nmax, nmax};
    }
    const int T = blockDim.x;
    R *base = sm + 2 * n + threadIdx.x;
    return {base, base + (long long)n * T, base + 2LL * n * T, base + 3LL * n * T, T};
}

// ------------------------------------------------------------------------ 3. inverse iteration (kept)
// Thread (matrix b, vector mu < n_k): three inverse-iteration solves from a pseudo-random start; the result (not
// yet orthogonalised) goes to Y row mu (Y: nmax x n per matrix, row-major).
template <class R>
__global__ void __launch_bounds__(64) k_tri_invit(const TriDescT<R> *__restrict__ descs,
                                                  const int *__restrict__ nkeep, R *__restrict__ Y,
                                                  R *__restrict__ work, int nmax) {
    const int b = blockIdx.x;
    const TriDescT<R> D = descs[b];
    const int n = D.n;
    const int mu = blockIdx.y * blockDim.x + threadIdx.x;
    const int nk = nkeep[b];
    extern __shared__ __align__(16) unsigned char tri_raw[];
    const R *ds = stage_tri(D, reinterpret_cast<R *>(tri_raw)), *es = ds + n;
    if (mu >= nk) return;
    const TriWork<R> W = tri_work(reinterpret_cast<R *>(tri_raw), n, work, b, nmax, mu);
    const long long st = W.st;
    R *x = W.x, *u0 = W.u0, *u1 = W.u1, *u2 = W.u2;
    const R pivmin = tri_pivmin(ds, es, n);
    const R lam = D.w[mu];
    unsigned h = 2166136261u ^ (unsigned)(mu * 7919 + 17);
    for (int i = 0; i < n; ++i) {
        h = (h ^ (unsigned)i) * 16777619u;
        x[(long long)i * st] = (R)(0.5 + (double)(h % 1000003u) / 1000003.0);
    }
    for (int rep = 0; rep < 3; ++rep) {
        tri_solve<R>(ds, es, n, lam, x, u0, u1, u2, st, pivmin);
        R s0 = 0, s1 = 0;
        for (int i = 0; i + 1 < n; i += 2) {
            s0 = fma(x[(long long)i * st], x[(long long)i * st], s0);
            s1 = fma(x[(long long)(i + 1) * st], x[(long long)(i + 1) * st], s1);
        }
        if (n & 1) s0 = fma(x[(long long)(n - 1) * st], x[(long long)(n - 1) * st], s0);
        const R inv = (R)1 / sqrt(s0 + s1);
        for (int i = 0; i < n; ++i) x[(long long)i * st] *= inv;
    }
    R *y = Y + ((long long)b * nmax + mu) * n;
    for (int i = 0; i < n; ++i) y[i] = x[(long long)i * st];
}

// Shifted solves of the OSV relaxation: X row mu = (Tri - s_mu)^{-1} (-R row mu) for mu < n_k, zero otherwise.
template <class R>
__global__ void __launch_bounds__(64) k_tri_shift_solve(const TriDescT<R> *__restrict__ descs,
                                                        const int *__restrict__ nkeep, const R *__restrict__ Rin,
                                                        R *__restrict__ X, R *__restrict__ work, int nmax,
                                                        const double *__restrict__ shift, int shift_ld) {
    const int b = blockIdx.x;
    const TriDescT<R> D = descs[b];
    const int n = D.n;
    const int mu = blockIdx.y * blockDim.x + threadIdx.x;
    extern __shared__ __align__(16) unsigned char tri_raw[];
    const R *ds = stage_tri(D, reinterpret_cast<R *>(tri_raw)), *es = ds + n;
    if (mu >= nmax) return;
    const int nk = nkeep[b];
    R *xo = X + ((long long)b * nmax + mu) * n;
    if (mu >= nk) {
        for (int i = 0; i < n; ++i) xo[i] = 0;
        return;
    }
    const TriWork<R> W = tri_work(reinterpret_cast<R *>(tri_raw), n, work, b, nmax, mu);
    const long long st = W.st;
    R *x = W.x, *u0 = W.u0, *u1 = W.u1, *u2 = W.u2;
    const R pivmin = tri_pivmin(ds, es, n);
    const R *r = Rin + ((long long)b * nmax + mu) * n;
    for (int i = 0; i < n; ++i) x[(long long)i * st] = -r[i];
    const R s = shift ? (R)shift[(long long)b * shift_ld + mu] : D.w[mu];
    tri_solve<R>(ds, es, n, s, x, u0, u1, u2, st, pivmin);
    for (int i = 0; i < n; ++i) xo[i] = x[(long long)i * st];
}

// ------------------------------------------------------------------------------ CGS2 helpers (per CTA)
template <class R>
__device__ __forceinline__ R warp_dot(const R *a, const R *b, int n) {
    R s0 = 0, s1 = 0;
    const int lane = threadIdx.x & 31;
    int i = lane;
    for (; i + 32 < n; i += 64) {
        s0 = fma(a[i], b[i], s0);
        s1 = fma(a[i + 32], b[i + 32], s1);
    }
    if (i < n) s0 = fma(a[i], b[i], s0);
    return warp_sum_t(s0 + s1);
}

// Orthonormalise rows 0..n_k-1 of Y (per matrix) in order with two Gram-Schmidt passes each.
template <class R>
__global__ void __launch_bounds__(kT) k_orthonormalise(const int *__restrict__ nkeep, R *__restrict__ Y, int n,
                                                       int nmax) {
    const int b = blockIdx.x;
    const int nk = nkeep[b];
    R *Yb = Y + (long long)b * nmax * n;
    __shared__ R coef[128];
    __shared__ double red[kT / 32];
    const int wid = threadIdx.x >> 5, nw = kT / 32, lane = threadIdx.x & 31;
    for (int mu = 0; mu < nk; ++mu) {
        R *y = Yb + (long long)mu * n;
        for (int pass = 0; pass < 2; ++pass) {
            for (int nu = wid; nu < mu; nu += nw) {
                const R c = warp_dot<R>(y, Yb + (long long)nu * n, n);
                if (lane == 0) coef[nu] = c;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += kT) {
                R s = y[i];
                for (int nu = 0; nu < mu; ++nu) s -= coef[nu] * Yb[(long long)nu * n + i];
                y[i] = s;
            }
            __syncthreads();
        }
        double ss = 0.0;
        for (int i = threadIdx.x; i < n; i += kT) ss += (double)y[i] * (double)y[i];
        ss = block_sum(ss, red);
        const R inv = ss > 0.0 ? (R)(1.0 / sqrt(ss)) : (R)0;
        for (int i = threadIdx.x; i < n; i += kT) y[i] *= inv;
        __syncthreads();
    }
}

// X rows mu < nx of each matrix -= projection onto rows 0..n_k-1 of Y (two passes; Y orthonormal).
template <class R>
__global__ void __launch_bounds__(kT) k_project_out(const int *__restrict__ nkeep, const R *__restrict__ Y,
                                                    R *__restrict__ X, int n, int nmax) {
    const int b = blockIdx.x;
    const int nk = nkeep[b];
    const R *Yb = Y + (long long)b * nmax * n;
    R *Xb = X + (long long)b * nmax * n;
    const int wid = threadIdx.x >> 5, nw = kT / 32, lane = threadIdx.x & 31;
    for (int pass = 0; pass < 2; ++pass) {
        for (int mu = wid; mu < nk; mu += nw) {
            R *x = Xb + (long long)mu * n;
            // coefficients against every kept y, then one update (classical Gram-Schmidt, repeated)
            R cbuf[4];
            for (int nu0 = 0; nu0 < nk; nu0 += 4) {
                const int cnt = min(4, nk - nu0);
                for (int t = 0; t < cnt; ++t) cbuf[t] = warp_dot<R>(x, Yb + (long long)(nu0 + t) * n, n);
                __syncwarp();
                for (int i = lane; i < n; i += 32) {
                    R s = x[i];
                    for (int t = 0; t < cnt; ++t) s -= cbuf[t] * Yb[(long long)(nu0 + t) * n + i];
                    x[i] = s;
                }
                __syncwarp();
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------- 4. reflector products
// rows mu < nrow(b) of V (nmax x n per matrix): forward = 0 applies H = H_0 ... H_{n-3} (q = H y),
// forward = 1 applies H^T (y = H^T g).  Reflector k: row k of A, columns k+1..n-1, scalar tau[k].
// CTA (matrix b, group of G rows): the G rows live in shared memory for the whole reflector sequence (one warp
// per row: a dot product and an update per reflector), and the next reflector is copied into a second buffer
// with cp.async while the current one is applied.
__device__ __forceinline__ void cp_async_elem(void *dst, const void *src, int bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <class R>
__global__ void __launch_bounds__(kT) k_reflect(const TriDescT<R> *__restrict__ descs, const int *__restrict__ nrow,
                                                R *__restrict__ V, int nmax, int forward, int G) {
    const int b = blockIdx.x;
    const TriDescT<R> D = descs[b];
    const int n = D.n;
    const int nr = nrow ? nrow[b] : nmax;
    const int g0 = blockIdx.y * G;
    if (g0 >= nr || n < 3) return;
    const int rows = min(G, nr - g0);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *Vs = reinterpret_cast<R *>(smem_raw);   // rows x n
    R *vb = Vs + (long long)G * n;               // 2 x n: current and next reflector
    R *ts = vb + 2 * n;                          // tau
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    R *Vg = V + ((long long)b * nmax + g0) * n;
    for (int i = tid; i < rows * n; i += kT) Vs[i] = Vg[i];
    for (int i = tid; i < n; i += kT) ts[i] = D.tau[i];
    auto fetch = [&](int s, R *dst) {   // reflector of step s -> dst[0 .. m)
        const int k = forward ? s : n - 3 - s, m = n - k - 1;
        const R *src = D.A + (long long)k * D.lda + k + 1;
        for (int i = tid; i < m; i += kT) cp_async_elem(dst + i, src + i, (int)sizeof(R));
    };
    fetch(0, vb);
    cp_async_wait_all();
    __syncthreads();
    for (int s = 0; s + 2 < n; ++s) {
        const int k = forward ? s : n - 3 - s, m = n - k - 1;
        const R *v = vb + (s & 1) * n;
        if (s + 3 < n) fetch(s + 1, vb + ((s + 1) & 1) * n);
        const R beta = ts[k];
        if (beta != (R)0 && wid < rows) {
            R *y = Vs + (long long)wid * n + k + 1;
            R a0 = 0, a1 = 0;
            int i = lane;
            for (; i + 32 < m; i += 64) {
                a0 = fma(y[i], v[i], a0);
                a1 = fma(y[i + 32], v[i + 32], a1);
            }
            if (i < m) a0 = fma(y[i], v[i], a0);
            const R c = beta * warp_sum_t(a0 + a1);
            for (int j = lane; j < m; j += 32) y[j] -= c * v[j];
        }
        cp_async_wait_all();
        __syncthreads();
    }
    for (int i = tid; i < rows * n; i += kT) Vg[i] = Vs[i];
}

// rows per CTA of k_reflect for order n: as many as fit next to the two reflector buffers (at most 8)
template <class R>
int reflect_rows(int n) {
    const long long cap = 200 * 1024, per = (long long)n * sizeof(R);
    const long long g = (cap - 3 * per) / per;
    return (int)std::max<long long>(1, std::min<long long>(8, g));
}

// -------------------------------------------------------------------------------- small dense Jacobi
// Cyclic parallel Jacobi for symmetric matrices of order <= kJacobiMax held in shared memory (A and V, padded to
// even order).  Eigenvalues decreasing into w, eigenvectors as rows of Zt.  n_dev (optional) gives the order.
__global__ void __launch_bounds__(kT) k_jacobi_small(const EighDesc *__restrict__ descs, int *err) {
    const EighDesc D = descs[blockIdx.x];
    const int n = D.n_dev ? min(*D.n_dev, D.n) : D.n;
    if (n <= 0) return;
    const int ne = (n + 1) & ~1;       // even order (the extra index never couples)
    const int ld = ne + 1;
    extern __shared__ double sh[];
    double *A = sh, *V = sh + (long long)ne * ld;
    double *cs = V + (long long)ne * ld, *sn = cs + ne / 2;
    int *pp = reinterpret_cast<int *>(sn + ne / 2), *qq = pp + ne / 2, *rank = qq + ne / 2;
    __shared__ double red[kT / 32];
    __shared__ int s_flag;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < ne * ne; idx += kT) {
        const int r = idx / ne, c = idx % ne;
        A[r * ld + c] = (r < n && c < n) ? D.A[(long long)r * D.lda + c] : 0.0;
        V[r * ld + c] = r == c ? 1.0 : 0.0;
    }
    __syncthreads();
    const bool conv = jacobi_sweeps<double>(A, V, ne, ld, cs, sn, pp, qq, red, &s_flag, 40, 1e-28);
    if (!conv && tid == 0) raise_err(err, kDevEighNoConv);
    diag_rank<double>(A, n, ld, rank);
    for (int i = tid; i < n; i += kT) D.w[rank[i]] = A[i * ld + i];
    for (int idx = tid; idx < n * n; idx += kT) {
        const int c = idx / n, r = idx % n;    // eigenvector c, component r
        D.Zt[(long long)rank[c] * D.ldz + r] = V[r * ld + c];
    }
}

// Mixed-precision variant for the pair eigenproblems (order <= kJacobiMixedMax): FP32 Jacobi sweeps to the FP32
// floor give V0; then, in double-float arithmetic on the FP32 pipe (common.cuh; an FP64 operation issues at 1/64
// of the FP32 rate on GB300): two Newton-Schulz steps V <- V (3I - V^T V)/2 (orthonormality 1e-6 -> 1e-12 ->
// 1e-16), A1 = V^T A V, and Jacobi polishing sweeps on A1, which is diagonal to ~1e-7 relative and converges
// quadratically (one sweep, two with close eigenvalues).  Shared memory: four n x n double-float buffers (the
// FP32 A and V of the first stage alias the first).

// C = op(A) op(B) for ne x ne double-float matrices in shared memory (leading dimension ld), 5 x 5 outputs per
// thread; op = transpose when TA / TB.
template <bool TA, bool TB>
__device__ void df_gemm_sm(int ne, int ld, const float2 *A, const float2 *B, float2 *C) {
    const int t5 = (ne + 4) / 5;
    for (int t = threadIdx.x; t < t5 * t5; t += blockDim.x) {
        const int r0 = (t / t5) * 5, c0 = (t % t5) * 5;
        float h[5][5] = {}, l[5][5] = {};
        for (int k = 0; k < ne; ++k) {
            float2 a[5], b[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                const int r = min(r0 + i, ne - 1), c = min(c0 + i, ne - 1);
                a[i] = TA ? A[k * ld + r] : A[r * ld + k];
                b[i] = TB ? B[c * ld + k] : B[k * ld + c];
            }
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j) df_fma(h[i][j], l[i][j], a[i], b[j]);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (r0 + i < ne && c0 + j < ne) C[(r0 + i) * ld + c0 + j] = df_renorm(h[i][j], l[i][j]);
    }
}

// zwork holds D.n x D.n doubles: room for the ne x ne FP32 first-stage vectors unless n = 1
__device__ __forceinline__ bool jacobi_z_fits(const EighDesc &D, int n) {
    const long long ne = (n + 1) & ~1;
    return D.zwork != nullptr && ne * ne <= 2LL * D.n * D.n;
}

// First stage of the mixed small Jacobi on its own (small shared memory, several CTAs per SM): FP32 sweeps on
// A from the identity; the vectors (columns) go to zwork as ne x ne floats.
__global__ void __launch_bounds__(kT) k_jacobi32(const EighDesc *__restrict__ descs) {
    const EighDesc D = descs[blockIdx.x];
    const int n = D.n_dev ? min(*D.n_dev, D.n) : D.n;
    if (n <= 0 || !jacobi_z_fits(D, n)) return;
    const int ne = (n + 1) & ~1, ld = ne + 1;
    extern __shared__ __align__(16) float j32[];
    float *A32 = j32, *V32 = A32 + (long long)ne * ld, *cs = V32 + (long long)ne * ld, *sn = cs + ne / 2;
    int *pp = reinterpret_cast<int *>(sn + ne / 2), *qq = pp + ne / 2;
    __shared__ double red[kT / 32];
    __shared__ int s_flag;
    for (int idx = threadIdx.x; idx < ne * ne; idx += kT) {
        const int r = idx / ne, c = idx % ne;
        A32[r * ld + c] = (r < n && c < n) ? (float)D.A[(long long)r * D.lda + c] : 0.f;
        V32[r * ld + c] = r == c ? 1.f : 0.f;
    }
    __syncthreads();
    jacobi_sweeps<float>(A32, V32, ne, ld, cs, sn, pp, qq, red, &s_flag, 20, 1e-10);
    float *Vz = reinterpret_cast<float *>(D.zwork);
    for (int idx = threadIdx.x; idx < ne * ne; idx += kT) Vz[idx] = V32[(idx / ne) * ld + idx % ne];
}

__global__ void __launch_bounds__(kTJ) k_jacobi_mixed(const EighDesc *__restrict__ descs, int *err) {
    const EighDesc D = descs[blockIdx.x];
    const int n = D.n_dev ? min(*D.n_dev, D.n) : D.n;
    if (n <= 0) return;
    const int ne = (n + 1) & ~1;
    const int ld = ne + 1;
    const long long sq = (long long)ne * ld;
    extern __shared__ double sh[];
    float2 *B0 = reinterpret_cast<float2 *>(sh), *B1 = B0 + sq, *B2 = B1 + sq, *B3 = B2 + sq;
    float2 *cs = B3 + sq, *sn = cs + ne / 2;
    double *dg = reinterpret_cast<double *>(sn + ne / 2);
    float *cs32 = reinterpret_cast<float *>(dg + ne), *sn32 = cs32 + ne / 2;
    int *pp = reinterpret_cast<int *>(sn32 + ne / 2), *qq = pp + ne / 2, *rank = qq + ne / 2;
    float *A32 = reinterpret_cast<float *>(B0), *V32 = A32 + sq;
    __shared__ double red[kTJ / 32];
    __shared__ int s_flag;
    const int tid = threadIdx.x;
    auto Ag = [&](int r, int c) -> double { return (r < n && c < n) ? D.A[(long long)r * D.lda + c] : 0.0; };
    if (jacobi_z_fits(D, n)) {   // first stage done by k_jacobi32
        const float *Vz = reinterpret_cast<const float *>(D.zwork);
        for (int idx = tid; idx < ne * ne; idx += kTJ) {
            const int r = idx / ne, c = idx % ne;
            B3[r * ld + c] = split_df(Ag(r, c));   // A as double-float for A1 = V^T A V
            B1[r * ld + c] = make_float2(Vz[idx], 0.f);
        }
    } else {
        for (int idx = tid; idx < ne * ne; idx += kTJ) {
            const int r = idx / ne, c = idx % ne;
            const double a = Ag(r, c);
            A32[r * ld + c] = (float)a;
            V32[r * ld + c] = r == c ? 1.f : 0.f;
            B3[r * ld + c] = split_df(a);   // A as double-float for A1 = V^T A V
        }
        __syncthreads();
        jacobi_sweeps<float>(A32, V32, ne, ld, cs32, sn32, pp, qq, red, &s_flag, 20, 1e-10);
        for (int idx = tid; idx < ne * ne; idx += kTJ) {
            const int r = idx / ne, c = idx % ne;
            B1[r * ld + c] = make_float2(V32[r * ld + c], 0.f);
        }
    }
    __syncthreads();
    // two Newton-Schulz steps: V in B1 -> B0 -> B1
    float2 *Vin = B1, *Vout = B0;
    for (int step = 0; step < 2; ++step) {
        df_gemm_sm<true, false>(ne, ld, Vin, Vin, B2);   // G = V^T V
        __syncthreads();
        for (int idx = tid; idx < ne * ne; idx += kTJ) {   // M = (3I - G)/2
            const int r = idx / ne, c = idx % ne;
            const float2 g = B2[r * ld + c];
            if (r == c) {   // 1.5 - g/2 with an exact two-sum (g ~ 1: a plain FP32 subtraction would round)
                float h = 1.5f, l = -0.5f * g.y;
                df_add(h, l, -0.5f * g.x);
                B2[r * ld + c] = df_renorm(h, l);
            } else {
                B2[r * ld + c] = make_float2(-0.5f * g.x, -0.5f * g.y);
            }
        }
        __syncthreads();
        df_gemm_sm<false, false>(ne, ld, Vin, B2, Vout);   // V M
        __syncthreads();
        float2 *t = Vin;
        Vin = Vout;
        Vout = t;
    }
    // V in B1: T = A V (B0), A1 = V^T T (B2, symmetrised)
    df_gemm_sm<false, false>(ne, ld, B3, B1, B0);
    __syncthreads();
    df_gemm_sm<true, false>(ne, ld, B1, B0, B2);
    __syncthreads();
    for (int idx = tid; idx < ne * ne; idx += kTJ) {   // symmetrise: (x + y) / 2 with a two-sum
        const int r = idx / ne, c = idx % ne;
        if (r < c) {
            const float2 x = B2[r * ld + c], y = B2[c * ld + r];
            float h = x.x, l = __fadd_rn(x.y, y.y);
            df_add(h, l, y.x);
            const float2 m = df_renorm(0.5f * h, 0.5f * l);
            B2[r * ld + c] = m;
            B2[c * ld + r] = m;
        }
    }
    __syncthreads();
    for (int idx = tid; idx < ne * ne; idx += kTJ) {   // polish rotations accumulate from the identity
        const int r = idx / ne, c = idx % ne;
        B3[r * ld + c] = make_float2(r == c ? 1.f : 0.f, 0.f);
    }
    __syncthreads();
    const bool conv = jacobi_sweeps_df(B2, B3, ne, ld, cs, sn, pp, qq, red, &s_flag, 20, 1e-28);
    if (!conv && tid == 0) raise_err(err, kDevEighNoConv);
    for (int i = tid; i < ne; i += kTJ) dg[i] = df_val(B2[i * ld + i].x, B2[i * ld + i].y);
    __syncthreads();
    df_gemm_sm<false, false>(ne, ld, B1, B3, B0);   // eigenvectors V V'
    for (int i = tid; i < n; i += kTJ) {
        const double di = dg[i];
        int rk = 0;
        for (int j = 0; j < n; ++j) rk += (dg[j] > di) || (dg[j] == di && j < i);
        rank[i] = rk;
    }
    __syncthreads();
    for (int i = tid; i < n; i += kTJ) D.w[rank[i]] = dg[i];
    for (int idx = tid; idx < n * n; idx += kTJ) {
        const int c = idx / n, r = idx % n;    // eigenvector c, component r
        const float2 z = B0[r * ld + c];
        D.Zt[(long long)rank[c] * D.ldz + r] = df_val(z.x, z.y);
    }
}

template <class K>
cudaError_t smem_attr(K kernel, size_t sh) {
    if (sh > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    return cudaSuccess;
}

// Block size, shared memory and work pointer of the tridiagonal solves for order n: 16 threads with their work
// columns in shared memory when they fit (work pointer nullptr), else 64 threads on the global work array.
template <class R>
R *tri_solve_launch(int n, R *work, int &T, size_t &sh) {
    const size_t smem = (2 * (size_t)n + 4 * (size_t)n * 16) * sizeof(R);
    if (smem <= 220 * 1024) {
        T = 16;
        sh = smem;
        return nullptr;
    }
    T = 64;
    sh = 2 * (size_t)n * sizeof(R);
    return work;
}

}  // namespace

size_t jacobi_smem_bytes(int n) {
    const int ne = (n + 1) & ~1;
    return (size_t)2 * ne * (ne + 1) * sizeof(double) + (size_t)ne * sizeof(double) + (size_t)3 * (ne / 2 + 1) * sizeof(int) +
           (size_t)ne * sizeof(int) + 64;
}

// k_tridiag_delayed<NB, MINB>: the ring of NB + 1 pairs (v_s, p_s), the stash and the column sums in shared memory
template <int NB, int MINB, int NSL = 0, int RWS = 4>
cudaError_t launch_tridiag_delayed(const TriDescT<float> *d, int batch, int n, cudaStream_t s) {
    const size_t sh = (size_t)(2 * (NB + 1) + 2) * ((n + 3) & ~3) * sizeof(float) +
                      (size_t)(kTT / 32) * NSL * RWS * 32 * sizeof(float4);
    if (sh > 227 * 1024) return cudaErrorNotSupported;   // the ring does not fit beside the vectors at this order
    cudaError_t e = smem_attr(k_tridiag_delayed<NB, MINB, NSL, RWS>, sh);
    if (e != cudaSuccess) return e;
    count_launch();
    k_tridiag_delayed<NB, MINB, NSL, RWS><<<batch, kTT, sh, s>>>(d);
    return cudaGetLastError();
}

template <class R>
cudaError_t osv_tridiag(const TriDescT<R> *d, int batch, int n, cudaStream_t s, int variant) {
    if (batch <= 0) return cudaSuccess;
    cudaError_t e;
    if constexpr (sizeof(R) == 4) {
        if (variant == 1) {
            // FP32, one CTA per matrix and two CTAs per SM (no cluster barriers; more warps per SM)
            const size_t sh = 6 * (size_t)((n + 3) & ~3) * sizeof(R);
            if ((e = smem_attr(k_tridiag<R, 1, 2>, sh)) != cudaSuccess) return e;
            count_launch();
            k_tridiag<R, 1, 2><<<batch, kTT, sh, s>>>(d);
            return cudaGetLastError();
        }
        if (variant == 8) return launch_tridiag_delayed<2, 2, 2>(d, batch, n, s);
        if (variant == 9) return launch_tridiag_delayed<2, 1, 2>(d, batch, n, s);
        if (variant == 10) return launch_tridiag_delayed<2, 1, 3>(d, batch, n, s);
        if (variant == 11) return launch_tridiag_delayed<2, 1, 4>(d, batch, n, s);
        if (variant == 12) return launch_tridiag_delayed<2, 1, 2, 8>(d, batch, n, s);
        if (variant >= 5 && variant <= 7) {
            // FP32, one CTA per matrix, the updates of two (variants 5, 6) or four (7) steps written together;
            // variant 6 two CTAs per SM
            if (variant == 5) return launch_tridiag_delayed<2, 1>(d, batch, n, s);
            if (variant == 6) return launch_tridiag_delayed<2, 2>(d, batch, n, s);
            return launch_tridiag_delayed<4, 1>(d, batch, n, s);
        }
        if (variant >= 2 && variant <= 4) {
            // FP32, a cluster of 4, 8 or 16 CTAs per matrix, one CTA per SM (16 is a non-portable cluster size)
            const int cl = 2 << variant;
            const size_t sh = 7 * (size_t)((n + 3) & ~3) * sizeof(R);
            void (*kern)(const TriDescT<float> *) =
                cl == 4 ? k_tridiag_cl<4> : cl == 8 ? k_tridiag_cl<8> : k_tridiag_cl<16>;
            if ((e = smem_attr(kern, sh)) != cudaSuccess) return e;
            if (cl == 16 && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
                                cudaSuccess)
                return e;
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = dim3((unsigned)cl * (unsigned)batch);
            cfg.blockDim = dim3(kTT);
            cfg.dynamicSmemBytes = sh;
            cfg.stream = s;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = (unsigned)cl;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if ((e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg)) != cudaSuccess) return e;
            if (nclusters < 1) return cudaErrorNotSupported;   // this GPU cannot hold one such cluster
            count_launch();
            return cudaLaunchKernelEx(&cfg, kern, d);
        }
        // FP32: a pair of CTAs (thread-block cluster) per matrix, each owning every other row; v, p, vo, po, the
        // column stash, the column sums and the peer's column sums in shared memory
        const size_t sh = 7 * (size_t)((n + 3) & ~3) * sizeof(R);
        if ((e = smem_attr(k_tridiag<R, 2, 1>, sh)) != cudaSuccess) return e;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(2 * (unsigned)batch);
        cfg.blockDim = dim3(kTT);
        cfg.dynamicSmemBytes = sh;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        count_launch();
        return cudaLaunchKernelEx(&cfg, k_tridiag<R, 2, 1>, d);
    } else {
        (void)variant;
        const size_t sh = 6 * (size_t)((n + 3) & ~3) * sizeof(R);
        if ((e = smem_attr(k_tridiag<R, 1, 1>, sh)) != cudaSuccess) return e;
        count_launch();
        k_tridiag<R, 1, 1><<<batch, kTT, sh, s>>>(d);
        return cudaGetLastError();
    }
}

template <class R>
cudaError_t osv_tri_eigvals(const TriDescT<R> *d, int batch, int n, int cnt, cudaStream_t s) {
    if (batch <= 0 || cnt <= 0) return cudaSuccess;
    cnt = cnt < n ? cnt : n;
    const dim3 grid(batch, (cnt + kMsWarps - 1) / kMsWarps);
    cudaError_t e;
    if constexpr (sizeof(R) == 4) {
        const size_t sh = 2 * (size_t)n * sizeof(float);
        if ((e = smem_attr(k_tri_multisect32, sh)) != cudaSuccess) return e;
        count_launch();
        k_tri_multisect32<<<grid, kMsWarps * 32, sh, s>>>(d, cnt);
    } else {
        const size_t sh = 2 * (size_t)n * sizeof(double);
        if ((e = smem_attr(k_tri_multisect<R>, sh)) != cudaSuccess) return e;
        count_launch();
        k_tri_multisect<R><<<grid, kMsWarps * 32, sh, s>>>(d, cnt);
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t osv_tri_kept_vectors(const TriDescT<R> *d, int batch, int n, int nmax, const int *nkeep, R *Y, R *work,
                                 cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    if (nmax > 128) return cudaErrorInvalidValue;
    int T;
    size_t sh;
    R *wk = tri_solve_launch<R>(n, work, T, sh);
    cudaError_t e;
    if ((e = smem_attr(k_tri_invit<R>, sh)) != cudaSuccess) return e;
    count_launch();
    k_tri_invit<R><<<dim3(batch, (nmax + T - 1) / T), T, sh, s>>>(d, nkeep, Y, wk, nmax);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_launch();
    k_orthonormalise<R><<<batch, kT, 0, s>>>(nkeep, Y, n, nmax);
    return cudaGetLastError();
}

template <class R>
cudaError_t osv_reflect(const TriDescT<R> *d, int batch, int n, int nmax, const int *nrow, R *V, int forward,
                        cudaStream_t s) {
    if (batch <= 0 || nmax <= 0) return cudaSuccess;
    const int G = reflect_rows<R>(n);
    const size_t sh = (size_t)(G + 3) * n * sizeof(R);
    cudaError_t e;
    if ((e = smem_attr(k_reflect<R>, sh)) != cudaSuccess) return e;
    count_launch();
    k_reflect<R><<<dim3(batch, (nmax + G - 1) / G), kT, sh, s>>>(d, nrow, V, nmax, forward, G);
    return cudaGetLastError();
}

template <class R>
cudaError_t osv_project_out(const int *nkeep, const R *Y, R *X, int batch, int n, int nmax, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    count_launch();
    k_project_out<R><<<batch, kT, 0, s>>>(nkeep, Y, X, n, nmax);
    return cudaGetLastError();
}

template <class R>
cudaError_t osv_tri_shift_solve(const TriDescT<R> *d, int batch, int n, int nmax, const int *nkeep, const R *Rin,
                                R *X, R *work, const double *shift, int shift_ld, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    int T;
    size_t sh;
    R *wk = tri_solve_launch<R>(n, work, T, sh);
    cudaError_t e;
    if ((e = smem_attr(k_tri_shift_solve<R>, sh)) != cudaSuccess) return e;
    count_launch();
    k_tri_shift_solve<R><<<dim3(batch, (nmax + T - 1) / T), T, sh, s>>>(d, nkeep, Rin, X, wk, nmax, shift, shift_ld);
    return cudaGetLastError();
}

#define OSV_EIG_INST(R)                                                                                            \
    template cudaError_t osv_tridiag<R>(const TriDescT<R> *, int, int, cudaStream_t, int);                         \
    template cudaError_t osv_tri_eigvals<R>(const TriDescT<R> *, int, int, int, cudaStream_t);                     \
    template cudaError_t osv_tri_kept_vectors<R>(const TriDescT<R> *, int, int, int, const int *, R *, R *,        \
                                                 cudaStream_t);                                                    \
    template cudaError_t osv_reflect<R>(const TriDescT<R> *, int, int, int, const int *, R *, int, cudaStream_t);  \
    template cudaError_t osv_project_out<R>(const int *, const R *, R *, int, int, int, cudaStream_t);             \
    template cudaError_t osv_tri_shift_solve<R>(const TriDescT<R> *, int, int, int, const int *, const R *, R *,   \
                                                R *, const double *, int, cudaStream_t);
OSV_EIG_INST(double)
OSV_EIG_INST(float)
#undef OSV_EIG_INST

size_t jacobi_mixed_smem_bytes(int n) {
    const int ne = (n + 1) & ~1;
    return (size_t)4 * ne * (ne + 1) * sizeof(float2) + (size_t)ne * sizeof(float2) + (size_t)ne * sizeof(double) +
           (size_t)ne * sizeof(float) + (size_t)3 * (ne / 2 + 1) * sizeof(int) + (size_t)ne * sizeof(int) + 64;
}

cudaError_t eigh_small_jacobi_mixed(const EighDesc *d, int batch, int n_max, int *err, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    if (n_max > kJacobiMixedMax) return cudaErrorInvalidValue;
    const int ne = (n_max + 1) & ~1;
    const size_t sh32 = (2 * (size_t)ne * (ne + 1) + ne) * sizeof(float) + (size_t)ne * sizeof(int);
    const size_t sh = jacobi_mixed_smem_bytes(n_max);
    cudaError_t e;
    if ((e = smem_attr(k_jacobi32, sh32)) != cudaSuccess) return e;
    if ((e = smem_attr(k_jacobi_mixed, sh)) != cudaSuccess) return e;
    count_launch(2);
    k_jacobi32<<<batch, kT, sh32, s>>>(d);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_jacobi_mixed<<<batch, kTJ, sh, s>>>(d, err);
    return cudaGetLastError();
}

cudaError_t eigh_small_jacobi(const EighDesc *d, int batch, int n_max, int *err, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    const size_t sh = jacobi_smem_bytes(n_max);
    cudaError_t e;
    if ((e = smem_attr(k_jacobi_small, sh)) != cudaSuccess) return e;
    count_launch();
    k_jacobi_small<<<batch, kT, sh, s>>>(d, err);
    return cudaGetLastError();
}

}  // namespace osv
