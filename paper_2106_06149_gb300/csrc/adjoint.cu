// Adjoint of the MBE(3)-OSV-MP2 energy (dE/dB, dE/df_occ), FP64.
//
// The amplitudes are variational (Sec. 2.1, text around Eq. 9), so dE is the partial derivative of
// E = sum_c w_c E^c_H at frozen cluster amplitudes.  With T = V T~ V^T in each pair's OSV basis and
// Tb = 2T - T^T, the per-cluster partials with respect to the pair blocks of Eq. 7 are, in the pseudo-canonical
// basis of each pair (Lambda = diag(e), m = 2 for i != j from the ordered pairs ij and ji, m = 1 for ii):
//   d/dS_(ij,ij):  m [Tb Lambda T^T + T^T Lambda Tb - (f_ii + f_jj)(Tb T^T + T^T Tb)]
//   d/dF_(ij,ij):  m [T^T Tb + Tb T^T]
//   d/dS_(ij,kl):  -m f [Tb S T'^T + Tb^T S T']            (one per coupling term of Eq. 4)
//   d/dK_(ij,ij):  2 m Tb_collective                         (linear: only the MBE-combined amplitudes)
//   d/df_xy:       -<S T' S^T, Tb> per term, -<T, Tb> for the diagonal f of D
// (these are the OSV-space densities D, D' and N_ij of Eqs. 14-16 in the orthonormal pair basis, MBE-combined
// as in Eqs. 33-34).  They are mapped back with V, split into LMO-pair blocks s_ab = Q_a^T Q_b,
// phi_ab = Q_a^T eps Q_b and K sub-blocks W^(i)_a W^(j)T_b, chained to W (recomputed in the forward and kept),
// Q and B, and the OSV gradient is relaxed through the discarded eigenvectors of T_kk (Eq. 8):
//   x_mu = sum_nu q'_nu q'_nu^T g_mu / (omega_mu - omega'_nu) (restricted resolvent, no discarded vectors formed),
//   G_T = sym(sum_mu x_mu q_mu^T),
//   dE/dB_k += 2 (G_T / Delta) B_k,  dE/df_kk += 2 sum_ab G_T,ab T_ab / Delta_ab.
#include "ctx.h"
#include "launch.h"

namespace osv {

namespace {

constexpr int kThreads = 256;

// C (M x N) (+)= alpha * op(A) diag(dk) op(B) with dk optional (scales the k index).
template <class R>
__device__ void sgemm_d(int M, int N, int K, const R *__restrict__ A, long long lda, bool ta,
                        const R *__restrict__ dk, const R *__restrict__ B, long long ldb, bool tb,
                        R *C, long long ldc, R alpha, bool accumulate) {
    const int mt = (M + 3) >> 2, nt = (N + 3) >> 2;
    for (int t = threadIdx.x; t < mt * nt; t += blockDim.x) {
        const int bm = (t / nt) << 2, bn = (t % nt) << 2;
        R acc[4][4] = {};
        for (int k = 0; k < K; ++k) {
            const R sk = dk ? dk[k] : R(1);
            R a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int m = bm + i;
                a[i] = m < M ? sk * (ta ? A[(long long)k * lda + m] : A[(long long)m * lda + k]) : R(0);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = bn + j;
                b[j] = n < N ? (tb ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n]) : R(0);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = bm + i;
            if (m >= M) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = bn + j;
                if (n >= N) continue;
                R *c = C + (long long)m * ldc + n;
                *c = accumulate ? *c + alpha * acc[i][j] : alpha * acc[i][j];
            }
        }
    }
}

struct AdjArgs {
    const ClusterInfo *clusters;
    const Slot *slots;
    const Term *terms;
    const PairInfo *pairs;
    const int *rdim;
    const double *focc;
    const void *e, *Tslot, *Stil;  // R-typed: pair energies, slot amplitudes, coupling blocks
    int n_occ, ncl;
    double *GS, *GF, *GSc, *dF;   // FP64 accumulators (pair off / coupling offset / n_occ^2)
    void *scratch;                // R-typed per-CTA scratch
    long long sstride, pstride;   // per-CTA scratch, one matrix slot
};

// Per-cluster partials of the weighted Hylleraas functional (products in precision R, FP64 accumulation).
template <class R>
__global__ void __launch_bounds__(kThreads) k_cluster_adjoint(AdjArgs A) {
    __shared__ double red[kThreads / 32];
    R *Tb = (R *)A.scratch + (long long)blockIdx.x * A.sstride;
    R *M1 = Tb + A.pstride, *M2 = M1 + A.pstride, *U1 = M2 + A.pstride, *U2 = U1 + A.pstride;
    const R *Ts = (const R *)A.Tslot, *Ss = (const R *)A.Stil, *Ee = (const R *)A.e;
    const int tid = threadIdx.x;
    for (int c = blockIdx.x; c < A.ncl; c += gridDim.x) {
        const ClusterInfo C = A.clusters[c];
        if (C.weight == 0) continue;
        const double w = (double)C.weight;
        for (int s = C.slot0; s < C.slot1; ++s) {
            const Slot S = A.slots[s];
            const PairInfo P = A.pairs[S.pair];
            const int r = A.rdim[S.pair], np = P.np;
            const R *T = Ts + S.t_off;
            const R *e = Ee + P.e_off;
            const double fii = A.focc[(long long)P.i * A.n_occ + P.i], fjj = A.focc[(long long)P.j * A.n_occ + P.j];
            double tt = 0.0;
            for (int idx = tid; idx < r * r; idx += kThreads) {
                const int a = idx / r, b = idx % r;
                const R tb = R(2) * T[(long long)a * np + b] - T[(long long)b * np + a];
                Tb[(long long)a * np + b] = tb;
                tt += (double)T[(long long)a * np + b] * (double)tb;
            }
            tt = block_sum(tt, red);   // also orders the Tb writes before the products below
            const double wm = w * S.mult;
            if (tid == 0) {
                atomicAdd(&A.dF[(long long)P.i * A.n_occ + P.i], -wm * tt);
                atomicAdd(&A.dF[(long long)P.j * A.n_occ + P.j], -wm * tt);
            }
            // M1 = Tb L T^T + T^T L Tb ;  M2 = Tb T^T + T^T Tb
            sgemm_d<R>(r, r, r, Tb, np, false, e, T, np, true, M1, np, R(1), false);
            sgemm_d<R>(r, r, r, Tb, np, false, nullptr, T, np, true, M2, np, R(1), false);
            __syncthreads();
            sgemm_d<R>(r, r, r, T, np, true, e, Tb, np, false, M1, np, R(1), true);
            sgemm_d<R>(r, r, r, T, np, true, nullptr, Tb, np, false, M2, np, R(1), true);
            __syncthreads();
            for (int idx = tid; idx < r * r; idx += kThreads) {
                const long long o = (long long)(idx / r) * np + idx % r;
                atomicAdd(&A.GS[P.off + o], wm * ((double)M1[o] - (fii + fjj) * (double)M2[o]));
                atomicAdd(&A.GF[P.off + o], wm * (double)M2[o]);
            }
            __syncthreads();
        }
        for (int t = C.term0; t < C.term1; ++t) {
            const Term T = A.terms[t];
            const Slot Sd = A.slots[T.dst], Ssl = A.slots[T.src];
            const PairInfo Pd = A.pairs[Sd.pair], Ps = A.pairs[Ssl.pair];
            const int rp = A.rdim[Sd.pair], rq = A.rdim[Ssl.pair];
            const int np = Pd.np, nq = Ps.np;
            const double f = A.focc[(long long)T.fx * A.n_occ + T.fy];
            const R *Sb = Ss + T.sblk;
            const long long lds = T.s_trans ? np : nq;
            const R *Tq = Ts + Ssl.t_off;
            const R *Tp = Ts + Sd.t_off;
            const double wm = w * Sd.mult;
            // Tb of the destination pair
            for (int idx = tid; idx < rp * rp; idx += kThreads) {
                const int a = idx / rp, b = idx % rp;
                Tb[(long long)a * np + b] = R(2) * Tp[(long long)a * np + b] - Tp[(long long)b * np + a];
            }
            __syncthreads();
            // U1 = Tb S (rp x rq), U2 = Tb^T S
            sgemm_d<R>(rp, rq, rp, Tb, np, false, nullptr, Sb, lds, T.s_trans, U1, nq, R(1), false);
            sgemm_d<R>(rp, rq, rp, Tb, np, true, nullptr, Sb, lds, T.s_trans, U2, nq, R(1), false);
            __syncthreads();
            // M2 = U1 T'^T (+ U2 T' below), rp x rq;  X = <S T', Tb S> = tr(T'^T S^T Tb S) = <S, U1 T'^T>
            sgemm_d<R>(rp, rq, rq, U1, nq, false, nullptr, Tq, nq, !T.t_trans, M2, nq, R(1), false);
            __syncthreads();
            double x = 0.0;
            for (int idx = tid; idx < rp * rq; idx += kThreads) {
                const int a = idx / rq, b = idx % rq;
                const double sab = T.s_trans ? (double)Sb[(long long)b * lds + a] : (double)Sb[(long long)a * lds + b];
                x += sab * (double)M2[(long long)a * nq + b];
            }
            x = block_sum(x, red);   // also orders every read of M2 above before the accumulation below
            if (tid == 0) {
                atomicAdd(&A.dF[(long long)T.fx * A.n_occ + T.fy], -w * x);
                if (Pd.i != Pd.j) atomicAdd(&A.dF[(long long)T.fy * A.n_occ + T.fx], -w * x);
            }
            sgemm_d<R>(rp, rq, rq, U2, nq, false, nullptr, Tq, nq, T.t_trans, M2, nq, R(1), true);
            __syncthreads();
            double *G = A.GSc + T.sblk;
            for (int idx = tid; idx < rp * rq; idx += kThreads) {
                const int a = idx / rq, b = idx % rq;
                const double v = -wm * f * (double)M2[(long long)a * nq + b];
                if (T.s_trans) atomicAdd(&G[(long long)b * np + a], v);   // stored as (src pair) x (dst pair)
                else atomicAdd(&G[(long long)a * nq + b], v);
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------------ double-float (FP32 pair) version
// The same partials in "double-float" arithmetic on the FP32 pipe (on GB300 an FP64 multiply-add issues at 1/64
// of the FP32 rate): every operand is split once into a pair of FP32 numbers (hi + lo, ~48 significant bits),
// a product is formed exactly (hi*hi and its FMA error term) plus the cross terms, and sums are kept as
// (hi, lo) pairs with an error-free two-sum.  ~12 FP32 operations per FP64 multiply-add, relative error
// ~2^-44 per partial (the FP64 version: 2^-53; the gradient bar is ~1e-7 relative).
// Shared memory: four np_max x ld buffers of float2: slot phase B0 = T, B1 = Tb, B2 = Tb L', B3 = L' T (L' =
// diag(e) - f_ii - f_jj); term phase B0 = S~, B1 = Tb_p then T~'_q, B2 = U1 = Tb S~, B3 = U2 = Tb^T S~.
constexpr int kAT = 512;   // one CTA per SM (its shared memory): 16 warps to hide the double-float latency

__global__ void __launch_bounds__(kAT, 1) k_cluster_adjoint_df(AdjArgsS A) {
    extern __shared__ __align__(16) float2 smf[];
    const int ld = A.ld;
    const long long sq = (long long)ld * ld;
    float2 *B0 = smf, *B1 = smf + sq, *B2 = smf + 2 * sq, *B3 = smf + 3 * sq;
    __shared__ double red[kAT / 32];
    const int tid = threadIdx.x;
    for (int q = blockIdx.x; q < A.ncl; q += gridDim.x) {
        const int c = A.order[q];
        const ClusterInfo C = A.clusters[c];
        if (C.weight == 0) continue;
        const double w = (double)C.weight;
        for (int s = C.slot0; s < C.slot1; ++s) {
            const Slot S = A.slots[s];
            const PairInfo P = A.pairs[S.pair];
            const int r = A.rdim[S.pair], np = P.np;
            const double *T = A.Tslot + S.t_off;
            const double *e = A.e + P.e_off;
            const double fii = A.focc[(long long)P.i * A.n_occ + P.i], fjj = A.focc[(long long)P.j * A.n_occ + P.j];
            // T lands raw (FP64) in B3's slots by asynchronous copies, all in flight together; then B0..B2, then B3
            double tt = 0.0;
            for (int idx = tid; idx < r * r; idx += kAT) {
                const int a = idx / r, b = idx % r;
                cpa_elem(B3 + a * ld + b, T + (long long)a * np + b, 8);
            }
            cpa_wait();
            __syncthreads();
            const double *Tr = reinterpret_cast<const double *>(B3);
            for (int idx = tid; idx < r * r; idx += kAT) {
                const int a = idx / r, b = idx % r;
                const double t = Tr[a * ld + b], tb = 2.0 * t - Tr[b * ld + a];
                B0[a * ld + b] = split_df(t);
                B1[a * ld + b] = split_df(tb);
                B2[a * ld + b] = split_df(tb * (e[b] - fii - fjj));   // Tb L'
                tt += t * tb;
            }
            __syncthreads();
            for (int idx = tid; idx < r * r; idx += kAT) {
                const int a = idx / r, b = idx % r;
                B3[a * ld + b] = split_df((e[a] - fii - fjj) * Tr[a * ld + b]);   // L' T (own element, in place)
            }
            tt = block_sum(tt, red);   // also orders the staging writes before the products
            const double wm = w * S.mult;
            if (tid == 0) {
                atomicAdd(&A.dF[(long long)P.i * A.n_occ + P.i], -wm * tt);
                atomicAdd(&A.dF[(long long)P.j * A.n_occ + P.j], -wm * tt);
            }
            // M2 = Tb T^T + T^T Tb and M1' = M1 - (f_ii + f_jj) M2 = (Tb L') T^T + (L' T)^T Tb, L' = diag(e) -
            // (f_ii + f_jj) (staged in B2, B3); two passes over k keep the register tiles small
            const int tr = (r + 3) >> 2;
            for (int t = tid; t < tr * tr; t += kAT) {
                const int a0 = (t / tr) << 2, b0 = (t % tr) << 2;
                double m2[4][4];
                {
                    float h[4][4] = {}, l[4][4] = {};
                    for (int k = 0; k < r; ++k) {
                        float2 x[4], y[4], u[4], v[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int a = min(a0 + i, r - 1), b = min(b0 + i, r - 1);
                            x[i] = B1[a * ld + k];   // Tb(a, k)
                            y[i] = B0[b * ld + k];   // T(b, k)
                            u[i] = B0[k * ld + a];   // T(k, a)
                            v[i] = B1[k * ld + b];   // Tb(k, b)
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                df_fma(h[i][j], l[i][j], x[i], y[j]);
                                df_fma(h[i][j], l[i][j], u[i], v[j]);
                            }
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) m2[i][j] = df_val(h[i][j], l[i][j]);
                }
                float h[4][4] = {}, l[4][4] = {};
                for (int k = 0; k < r; ++k) {
                    float2 xl[4], y[4], ul[4], v[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int a = min(a0 + i, r - 1), b = min(b0 + i, r - 1);
                        xl[i] = B2[a * ld + k];   // (Tb L')(a, k)
                        y[i] = B0[b * ld + k];    // T(b, k)
                        ul[i] = B3[k * ld + a];   // (L' T)(k, a)
                        v[i] = B1[k * ld + b];    // Tb(k, b)
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            df_fma(h[i][j], l[i][j], xl[i], y[j]);
                            df_fma(h[i][j], l[i][j], ul[i], v[j]);
                        }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int a = a0 + i, b = b0 + j;
                        if (a >= r || b >= r) continue;
                        const long long o = (long long)a * np + b;
                        atomicAdd(&A.GS[P.off + o], wm * df_val(h[i][j], l[i][j]));
                        atomicAdd(&A.GF[P.off + o], wm * m2[i][j]);
                    }
            }
            __syncthreads();
        }
        for (int t = C.term0; t < C.term1; ++t) {
            const Term Tm = A.terms[t];
            const Slot Sd = A.slots[Tm.dst], Ssl = A.slots[Tm.src];
            const PairInfo Pd = A.pairs[Sd.pair], Ps = A.pairs[Ssl.pair];
            const int rp = A.rdim[Sd.pair], rq = A.rdim[Ssl.pair];
            const int np = Pd.np, nq = Ps.np;
            const double f = A.focc[(long long)Tm.fx * A.n_occ + Tm.fy];
            const double *Sb = A.Stil + Tm.sblk;
            const long long lds = Tm.s_trans ? np : nq;
            const double *Tq = A.Tslot + Ssl.t_off, *Tp = A.Tslot + Sd.t_off;
            const double wm = w * Sd.mult;
            // B0 = S~ (rp x rq), B1 = Tb_p: S~ into B0's slots and T_p into B2's (raw FP64, asynchronous copies all
            // in flight together), then split in place / combined into B1
            for (int idx = tid; idx < rp * rq; idx += kAT) {
                const int a = idx / rq, b = idx % rq;
                cpa_elem(B0 + a * ld + b, Tm.s_trans ? Sb + (long long)b * lds + a : Sb + (long long)a * lds + b, 8);
            }
            for (int idx = tid; idx < rp * rp; idx += kAT) {
                const int a = idx / rp, b = idx % rp;
                cpa_elem(B2 + a * ld + b, Tp + (long long)a * np + b, 8);
            }
            cpa_wait();
            for (int idx = tid; idx < rp * rq; idx += kAT) {   // own elements
                const int a = idx / rq, b = idx % rq;
                B0[a * ld + b] = split_df(*reinterpret_cast<const double *>(B0 + a * ld + b));
            }
            __syncthreads();
            {
                const double *Tpr = reinterpret_cast<const double *>(B2);
                for (int idx = tid; idx < rp * rp; idx += kAT) {
                    const int a = idx / rp, b = idx % rp;
                    B1[a * ld + b] = split_df(2.0 * Tpr[a * ld + b] - Tpr[b * ld + a]);
                }
            }
            __syncthreads();
            // U1 = Tb S (B2), U2 = Tb^T S (B3): one 4 x 4 tile of one of them per job
            const int ta = (rp + 3) >> 2, tq = (rq + 3) >> 2;
            for (int job = tid; job < 2 * ta * tq; job += kAT) {
                const bool second = job >= ta * tq;
                const int t2 = second ? job - ta * tq : job;
                const int a0 = (t2 / tq) << 2, b0 = (t2 % tq) << 2;
                float uh[4][4] = {}, ul[4][4] = {};
                for (int k = 0; k < rp; ++k) {
                    float2 x[4], y[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int a = min(a0 + i, rp - 1), b = min(b0 + i, rq - 1);
                        x[i] = second ? B1[k * ld + a] : B1[a * ld + k];
                        y[i] = B0[k * ld + b];
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) df_fma(uh[i][j], ul[i][j], x[i], y[j]);
                }
                float2 *U = second ? B3 : B2;
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (a0 + i < rp && b0 + j < rq) {   // renormalised pairs
                            const float h = __fadd_rn(uh[i][j], ul[i][j]);
                            U[(a0 + i) * ld + b0 + j] = make_float2(h, __fsub_rn(ul[i][j], __fsub_rn(h, uh[i][j])));
                        }
            }
            __syncthreads();
            // B1 = T~'_q (rq x rq): asynchronous copies, then each thread splits its own elements
            for (int idx = tid; idx < rq * rq; idx += kAT) {
                const int a = idx / rq, b = idx % rq;
                cpa_elem(B1 + a * ld + b, Tm.t_trans ? Tq + (long long)b * nq + a : Tq + (long long)a * nq + b, 8);
            }
            cpa_wait();
            for (int idx = tid; idx < rq * rq; idx += kAT) {
                const int a = idx / rq, b = idx % rq;
                B1[a * ld + b] = split_df(*reinterpret_cast<const double *>(B1 + a * ld + b));
            }
            __syncthreads();
            // M2 = M2a + M2b with M2a = U1 T'^T, M2b = U2 T';  x = <S T', U1> = tr(T'^T S^T Tb S) = <S, M2a>
            double xs = 0.0;
            double *G = A.GSc + Tm.sblk;
            for (int t2 = tid; t2 < ta * tq; t2 += kAT) {
                const int a0 = (t2 / tq) << 2, b0 = (t2 % tq) << 2;
                double ma[4][4];
                {
                    float h[4][4] = {}, l[4][4] = {};
                    for (int k = 0; k < rq; ++k) {
                        float2 p1[4], tw[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int a = min(a0 + i, rp - 1), b = min(b0 + i, rq - 1);
                            p1[i] = B2[a * ld + k];   // U1(a, k)
                            tw[i] = B1[b * ld + k];   // T'(b, k)
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) df_fma(h[i][j], l[i][j], p1[i], tw[j]);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) ma[i][j] = df_val(h[i][j], l[i][j]);
                }
                float h[4][4] = {}, l[4][4] = {};
                for (int k = 0; k < rq; ++k) {
                    float2 p2[4], tv[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int a = min(a0 + i, rp - 1), b = min(b0 + i, rq - 1);
                        p2[i] = B3[a * ld + k];   // U2(a, k)
                        tv[i] = B1[k * ld + b];   // T'(k, b)
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) df_fma(h[i][j], l[i][j], p2[i], tv[j]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int a = a0 + i, b = b0 + j;
                        if (a >= rp || b >= rq) continue;
                        const float2 sab = B0[a * ld + b];
                        xs += df_val(sab.x, sab.y) * ma[i][j];
                        const double v = -wm * f * (ma[i][j] + df_val(h[i][j], l[i][j]));
                        if (Tm.s_trans) atomicAdd(&G[(long long)b * np + a], v);   // stored as (src pair) x (dst pair)
                        else atomicAdd(&G[(long long)a * nq + b], v);
                    }
            }
            xs = block_sum(xs, red);
            if (tid == 0) {
                atomicAdd(&A.dF[(long long)Tm.fx * A.n_occ + Tm.fy], -w * xs);
                if (Pd.i != Pd.j) atomicAdd(&A.dF[(long long)Tm.fy * A.n_occ + Tm.fx], -w * xs);
            }
            __syncthreads();
        }
    }
}

// dE/dK~ per pair: 2 m (2 Tc - Tc^T) (collective amplitudes)
__global__ void k_gk_tilde(const PairInfo *__restrict__ pairs, const double *__restrict__ Tc,
                           double *__restrict__ out) {
    const PairInfo P = pairs[blockIdx.x];
    const double m = P.i == P.j ? 1.0 : 2.0;
    const int np = P.np;
    for (long long idx = threadIdx.x; idx < (long long)np * np; idx += blockDim.x) {
        const int a = int(idx / np), b = int(idx % np);
        out[P.off + idx] = 2.0 * m * (2.0 * Tc[P.off + idx] - Tc[P.off + (long long)b * np + a]);
    }
}

// G = sym(G_T) / Delta in place, and df_kk += 2 sum_ab sym(G_T)_ab T_ab / Delta_ab.
__global__ void k_relax_sym(double *__restrict__ GT, const double *__restrict__ Tkk, const double *__restrict__ eps,
                            const double *__restrict__ focc, int n_occ, int nv, double *__restrict__ dF) {
    const int k = blockIdx.y;
    __shared__ double red[kThreads / 32];
    const double fkk = focc[(long long)k * n_occ + k];
    double *G = GT + (long long)k * nv * nv;
    const double *T = Tkk + (long long)k * nv * nv;
    double acc = 0.0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)nv * nv;
         idx += (long long)gridDim.x * blockDim.x) {
        const int a = int(idx / nv), b = int(idx % nv);
        if (b < a) continue;
        const double g = 0.5 * (G[(long long)a * nv + b] + G[(long long)b * nv + a]);
        const double den = eps[a] + eps[b] - 2.0 * fkk;
        const double gm = g / den;
        G[(long long)a * nv + b] = gm;
        G[(long long)b * nv + a] = gm;
        acc += (a == b ? 2.0 : 4.0) * gm * T[(long long)a * nv + b];
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) atomicAdd(&dF[(long long)k * n_occ + k], acc);
}

template <class T>
__global__ void k_out_b(const double *__restrict__ src, T *__restrict__ dst, long long n, double scale) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (T)((double)dst[i] + scale * src[i]);
}

}  // namespace

void AdjointPlan::release() {
    for (void *p : allocs) cudaFree(p);
    allocs.clear();
    for (GemmBatch *g : {&gb_kc1, &gb_kc2, &gb_f1, &gb_f2, &gb_k1, &gb_k2, &gb_c1, &gb_c2, &gb_z, &gb_db, &gb_dq,
                         &gb_gt, &gb_rb, &gb_at}) {
        gemm_batch_free(*g);
        g->h.clear();
    }
    for (TcTiles *t : {&oz_z, &oz_db, &oz_dq, &oz_gt, &oz_rb}) tc_tiles_free(*t);
    bc_hs.h.clear();
    bc_hs.d = nullptr;
    planned = false;
}

namespace {

template <class T>
cudaError_t adj_alloc(AdjointPlan &a, T *&p, size_t count) {
    p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e == cudaSuccess) a.allocs.push_back((void *)p);
    return e;
}

}  // namespace

cudaError_t AdjointPlan::plan(osv_ctx &c) {
    release();
    cudaError_t e;
    const int n = c.n_occ, nv = c.n_vir, nm = c.nmax;
    const long long npairs = (long long)c.pairs.size();
#define AL(p, cnt) if ((e = adj_alloc(*this, p, (size_t)(cnt))) != cudaSuccess) return e
    AL(GS, c.pair_mat);
    AL(GF, c.pair_mat);
    AL(GK, c.pair_mat);
    AL(GSo, c.pair_mat);
    AL(GFo, c.pair_mat);
    AL(GKo, c.pair_mat);
    AL(ptmp, c.pair_mat);
    AL(GSc, c.coup_mat);
    AL(GSco, c.coup_mat);
    AL(ctmp, c.coup_mat);
    AL(HS, npairs * nm * nm);
    AL(HF, npairs * nm * nm);
    AL(Z, c.w_off[n]);
    AL(dQ, (long long)n * nm * nv);
    AL(dB64, c.aux_ptr[n] * (long long)nv);
    AL(dF64, (long long)n * n);
    AL(A1, (long long)n * nv * nm);
    if (2 * nm <= kAdjTcMaxOrder) {   // (either precision: the plan outlives a change of mode)
        AL(TbS, std::max<long long>(c.slot_mat, 1));
        AL(ebS, std::max<size_t>(c.slots.h.size(), 1));
    }
    grid = (int)std::min<size_t>(c.cl.size(), 152 * 4);
    pstride = 4LL * nm * nm;
    AL(scratch, (long long)std::max(grid, 1) * 5 * pstride);
#undef AL
    // V G~ V^T for pair and coupling accumulators, and the K gradient
    auto vgv = [&](GemmBatch &b1, GemmBatch &b2, const double *G, double *tmp, double *out, const PairInfo &Pa,
                   const PairInfo &Pb, long long off) {
        // tmp = G V_b^T (na x nb), out = V_a tmp
        b1.add(gemm(Pa.np, Pb.np, Pb.np, G + off, Pb.np, 0, c.V + Pb.off, Pb.np, 1, tmp + off, Pb.np));
        b2.add(gemm(Pa.np, Pb.np, Pa.np, c.V + Pa.off, Pa.np, 0, tmp + off, Pb.np, 0, out + off, Pb.np));
    };
    for (size_t p = 0; p < c.pairs.size(); ++p) {
        const PairInfo &P = c.pinfo.h[p];
        vgv(gb_kc1, gb_kc2, GS, ptmp, GSo, P, P, P.off);
    }
    // the GF and GK transforms reuse ptmp: they go into separate batches run one after the other
    for (size_t p = 0; p < c.pairs.size(); ++p) {
        const PairInfo &P = c.pinfo.h[p];
        gb_f1.add(gemm(P.np, P.np, P.np, GF + P.off, P.np, 0, c.V + P.off, P.np, 1, ptmp + P.off, P.np));
        gb_f2.add(gemm(P.np, P.np, P.np, c.V + P.off, P.np, 0, ptmp + P.off, P.np, 0, GFo + P.off, P.np));
        gb_k1.add(gemm(P.np, P.np, P.np, GK + P.off, P.np, 0, c.V + P.off, P.np, 1, ptmp + P.off, P.np));
        gb_k2.add(gemm(P.np, P.np, P.np, c.V + P.off, P.np, 0, ptmp + P.off, P.np, 0, GKo + P.off, P.np));
    }
    for (size_t q = 0; q < c.couplings.size(); ++q) {
        const PairInfo &Pa = c.pinfo.h[c.couplings[q].first], &Pb = c.pinfo.h[c.couplings[q].second];
        vgv(gb_c1, gb_c2, GSc, ctmp, GSco, Pa, Pb, c.coup_off[q]);
    }
    // scatter OSV-basis blocks into LMO-pair accumulators HS (overlap) and HF (Fock)
    auto scatter = [&](const double *src, long long ld, int x_lmo, int y_lmo, double *H) {
        BlockCopy b{};
        const int q = c.pid(x_lmo, y_lmo);
        b.dst = H + (long long)q * nm * nm;
        b.ldd = nm;
        b.src = src;
        b.lds = ld;
        b.rows = b.cols = nm;
        b.trans = x_lmo > y_lmo ? 1 : 0;
        b.accumulate = 1;
        b.scale = 1.0;
        bc_hs.h.push_back(b);
    };
    for (size_t p = 0; p < c.pairs.size(); ++p) {
        const PairInfo &P = c.pinfo.h[p];
        const int d[2] = {P.i, P.j}, nd = P.i == P.j ? 1 : 2;
        for (int x = 0; x < nd; ++x)
            for (int y = 0; y < nd; ++y) {
                const long long o = P.off + (long long)x * nm * P.np + (long long)y * nm;
                scatter(GSo + o, P.np, d[x], d[y], HS);
                scatter(GFo + o, P.np, d[x], d[y], HF);
            }
    }
    for (size_t q = 0; q < c.couplings.size(); ++q) {
        const PairInfo &Pa = c.pinfo.h[c.couplings[q].first], &Pb = c.pinfo.h[c.couplings[q].second];
        const int da[2] = {Pa.i, Pa.j}, db[2] = {Pb.i, Pb.j};
        const int na = Pa.i == Pa.j ? 1 : 2, nb_ = Pb.i == Pb.j ? 1 : 2;
        for (int x = 0; x < na; ++x)
            for (int y = 0; y < nb_; ++y)
                scatter(GSco + c.coup_off[q] + (long long)x * nm * Pb.np + (long long)y * nm, Pb.np, da[x], db[y], HS);
    }
    e = [&]() {
        if (bc_hs.h.empty()) return cudaSuccess;
        cudaError_t ee = adj_alloc(*this, bc_hs.d, bc_hs.h.size());
        if (ee != cudaSuccess) return ee;
        return cudaMemcpy(bc_hs.d, bc_hs.h.data(), bc_hs.h.size() * sizeof(BlockCopy), cudaMemcpyHostToDevice);
    }();
    if (e != cudaSuccess) return e;
    // Z^(i) from the K gradient (common fitting domain gathers as in the forward K blocks)
    const bool full = [&]() {
        for (int i = 0; i < n; ++i)
            if (c.a_of(i) != c.n_aux) return false;
        return true;
    }();
    std::map<long long, std::pair<const int *, const int *>> kmap;
    std::map<long long, int> klen;
    if (!full) {
        // the forward's gb_k descriptors carry the common-domain lists: reuse them
        for (const GemmDesc &g : c.gb_k.h)
            if (g.k_idx_a) {
                // find the pair from the destination pointer
                const long long off = g.C - c.Kp;
                for (size_t p = 0; p < c.pairs.size(); ++p) {
                    const PairInfo &P = c.pinfo.h[p];
                    if (off >= P.off && off < P.off + (long long)P.np * P.np) {
                        kmap[(long long)P.i * n + P.j] = {g.k_idx_a, g.k_idx_b};
                        klen[(long long)P.i * n + P.j] = g.K;
                        break;
                    }
                }
            }
    }
    std::vector<int> zr_h;
    {
        long long offdiag = 0;
        for (size_t p = 0; p < c.pairs.size(); ++p) offdiag += c.pinfo.h[p].i != c.pinfo.h[p].j;
        if ((e = adj_alloc(*this, zrows, (size_t)(offdiag * 4 * nm))) != cudaSuccess) return e;
        zr_h.reserve((size_t)offdiag * 4 * nm);
    }
    for (size_t p = 0; p < c.pairs.size(); ++p) {
        const PairInfo &P = c.pinfo.h[p];
        const int i = P.i, j = P.j;
        const long long ai = c.a_of(i), aj = c.a_of(j);
        if (i == j) {
            const long long o = c.w_off[i] + (long long)c.slot_of(i, i) * nm * ai;
            for (int tr = 0; tr < 2; ++tr) {
                GemmDesc g = gemm(nm, (int)ai, nm, GKo + P.off, P.np, tr, c.W + o, ai, 0, Z + o, ai);
                g.atomic = 1;
                gb_z.add(g);
            }
            continue;
        }
        const int d[2] = {i, j};
        // dW^(i)_x += sum_y G_xy W^(j)_y and dW^(j)_y += sum_x G_xy^T W^(i)_x (columns on the common domain): the
        // two terms of each sum stacked along K (G rows or columns of the pair block; W rows through a row map)
        const long long zo = (long long)zr_h.size();
        for (int y = 0; y < 2; ++y)
            for (int t = 0; t < nm; ++t) zr_h.push_back(c.slot_of(j, d[y]) * nm + t);
        for (int x = 0; x < 2; ++x)
            for (int t = 0; t < nm; ++t) zr_h.push_back(c.slot_of(i, d[x]) * nm + t);
        for (int x = 0; x < 2; ++x) {
            const long long oi = c.w_off[i] + (long long)c.slot_of(i, d[x]) * nm * ai;
            GemmDesc g1 = gemm(nm, full ? c.n_aux : 0, 2 * nm, GKo + P.off + (long long)x * nm * P.np, P.np, 0,
                               c.W + c.w_off[j], aj, 0, Z + oi, ai);
            g1.k_idx_b = zrows + zo;
            g1.atomic = 1;
            if (!full) {
                const auto &m = kmap[(long long)i * n + j];
                g1.N = klen[(long long)i * n + j];
                g1.n_idx_b = m.second;
                g1.n_idx_c = m.first;
            }
            gb_z.add(g1);
        }
        for (int y = 0; y < 2; ++y) {
            const long long oj = c.w_off[j] + (long long)c.slot_of(j, d[y]) * nm * aj;
            GemmDesc g2 = gemm(nm, full ? c.n_aux : 0, 2 * nm, GKo + P.off + (long long)y * nm, P.np, 1,
                               c.W + c.w_off[i], ai, 0, Z + oj, aj);
            g2.k_idx_b = zrows + zo + 2 * nm;
            g2.atomic = 1;
            if (!full) {
                const auto &m = kmap[(long long)i * n + j];
                g2.N = klen[(long long)i * n + j];
                g2.n_idx_b = m.first;
                g2.n_idx_c = m.second;
            }
            gb_z.add(g2);
        }
    }
    if (!zr_h.empty() &&
        (e = cudaMemcpy(zrows, zr_h.data(), zr_h.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    // dB_i = sum_a Q_a Z^(i)_a  (Q rows gathered with the forward's row maps)
    {
        size_t at = 0;
        for (int i = 0; i < n; ++i) {
            const long long ai = c.a_of(i);
            const int kk = (int)c.nb[i].size() * nm;
            GemmDesc g = gemm(nv, (int)ai, kk, c.Q, nv, 1, Z + c.w_off[i], ai, 0, dB64 + c.b_off(i), ai);
            g.k_idx_a = c.rows_w.d + at;
            at += kk;
            gb_db.add(g);
        }
    }
    // dQ_a (rows) += Z^(i)_a B_i^T ;  HS/HF chains
    for (int i = 0; i < n; ++i) {
        const long long ai = c.a_of(i);
        for (int a : c.nb[i]) {
            const long long o = c.w_off[i] + (long long)c.slot_of(i, a) * nm * ai;
            GemmDesc g = gemm(nm, nv, (int)ai, Z + o, ai, 0, c.B64 + c.b_off(i), ai, 1, dQ + (long long)a * nm * nv, nv);
            g.atomic = 1;
            gb_dq.add(g);
        }
    }
    for (size_t p = 0; p < c.pairs.size(); ++p) {
        const int a = c.pairs[p].first, b = c.pairs[p].second;
        const double *Hs = HS + (long long)p * nm * nm, *Hf = HF + (long long)p * nm * nm;
        double *dQa = dQ + (long long)a * nm * nv, *dQb = dQ + (long long)b * nm * nv;
        const double *Qa = c.Q + (long long)a * nm * nv, *Qb = c.Q + (long long)b * nm * nv;
        const double *Qea = c.Qe + (long long)a * nm * nv, *Qeb = c.Qe + (long long)b * nm * nv;
        GemmDesc g[4] = {gemm(nm, nv, nm, Hs, nm, 0, Qb, nv, 0, dQa, nv), gemm(nm, nv, nm, Hs, nm, 1, Qa, nv, 0, dQb, nv),
                         gemm(nm, nv, nm, Hf, nm, 0, Qeb, nv, 0, dQa, nv), gemm(nm, nv, nm, Hf, nm, 1, Qea, nv, 0, dQb, nv)};
        for (auto &x : g) {
            x.atomic = 1;
            gb_dq.add(x);
        }
    }
    // relaxation: G_T = X^T Q with X the kept x discarded resolvent applied to dE/dQ (rows), then dB += 2 (G_T/Delta) B
    const long long nv2 = (long long)nv * nv;
    for (int k = 0; k < n; ++k) {
        gb_gt.add(gemm(nv, nv, nm, A1 + (long long)k * nm * nv, nv, 1, c.Q + (long long)k * nm * nv, nv, 0, c.Zc + k * nv2, nv));
        gb_rb.add(gemm(nv, (int)c.a_of(k), nv, c.Zc + k * nv2, nv, 0, c.B64 + c.b_off(k), c.a_of(k), 0,
                       dB64 + c.b_off(k), c.a_of(k), 2.0, 1.0));
        if (c.osv_mixed)
            gb_at.add(gemm(nm, nv, nv, A1 + (long long)k * nm * nv, nv, 0, c.Tkk + k * nv2, nv, 0,
                           c.refine.AT + (long long)k * nm * nv, nv));
    }
    for (GemmBatch *g : {&gb_kc1, &gb_kc2, &gb_f1, &gb_f2, &gb_k1, &gb_k2, &gb_c1, &gb_c2, &gb_z, &gb_db, &gb_dq,
                         &gb_gt, &gb_rb, &gb_at})
        if ((e = gemm_batch_upload(*g)) != cudaSuccess) return e;
    if ((e = bf16x4_batch_prepare(gb_z, oz_z)) != cudaSuccess ||
        (e = bf16x4_batch_prepare(gb_db, oz_db)) != cudaSuccess || (e = bf16x4_batch_prepare(gb_dq, oz_dq)) != cudaSuccess ||
        (e = bf16x4_batch_prepare(gb_gt, oz_gt)) != cudaSuccess || (e = bf16x4_batch_prepare(gb_rb, oz_rb)) != cudaSuccess)
        return e;
    if (c.prm.precision == OSV_MIXED_BF16X4) {
        long long need = 0;
        for (const TcTiles *t : {&oz_z, &oz_db, &oz_dq, &oz_gt, &oz_rb}) need = std::max(need, t->scratch_bytes);
        if ((e = c.oz_reserve((size_t)need)) != cudaSuccess) return e;
    }
    planned = true;
    return cudaSuccess;
}

cudaError_t AdjointPlan::run(osv_ctx &c, double scale, void *dB, double *dF, std::string &msg) {
    cudaError_t e;
    msg = "gradient_backward";
    if (!planned && (e = plan(c)) != cudaSuccess) {
        msg = "gradient_backward plan";
        return e;
    }
    cudaStream_t s = c.stream;
    const int n = c.n_occ, nv = c.n_vir, nm = c.nmax;
#define CK(x) \
    do { \
        if ((e = (x)) != cudaSuccess) return e; \
    } while (0)
    CK(cudaMemsetAsync(GS, 0, c.pair_mat * sizeof(double), s));
    CK(cudaMemsetAsync(GF, 0, c.pair_mat * sizeof(double), s));
    CK(cudaMemsetAsync(GSc, 0, c.coup_mat * sizeof(double), s));
    CK(cudaMemsetAsync(HS, 0, c.pairs.size() * nm * nm * sizeof(double), s));
    CK(cudaMemsetAsync(HF, 0, c.pairs.size() * nm * nm * sizeof(double), s));
    CK(cudaMemsetAsync(Z, 0, c.w_off[n] * sizeof(double), s));
    CK(cudaMemsetAsync(dQ, 0, (size_t)n * nm * nv * sizeof(double), s));
    CK(cudaMemsetAsync(dF64, 0, (size_t)n * n * sizeof(double), s));
    AdjArgs a{};
    a.clusters = c.cinfo.d;
    a.slots = c.slots.d;
    a.terms = c.terms.d;
    a.pairs = c.pinfo.d;
    a.rdim = c.rdim;
    a.e = c.pe;
    a.Tslot = c.Tslot;
    a.Stil = c.Stil;
    a.focc = c.focc;
    a.n_occ = n;
    a.ncl = (int)c.cl.size();
    a.GS = GS;
    a.GF = GF;
    a.GSc = GSc;
    a.dF = dF64;
    a.scratch = scratch;
    a.sstride = 5 * pstride;
    a.pstride = pstride;
    {
        StageTimer t(c, "adj_clusters");
        // FP64 in every mode: FP32 products here cost ~7e-7 relative in dE/dB, too much for a 1e-6 bar
        const int ld = 2 * nm + 1;
        const size_t sh = 4 * (size_t)ld * ld * sizeof(float2);
        const AdjArgsS as{c.cinfo.d, c.order.d, c.slots.d, c.terms.d, c.pinfo.d, c.rdim, c.focc, c.pe, c.Tslot,
                          c.Stil, n, (int)c.cl.size(), ld, GS, GF, GSc, dF64, TbS, ebS};
        if (c.osv_mixed && !c.cl.empty() && 2 * nm <= kAdjTcMaxOrder && TbS && ebS) {
            // mixed modes, pair orders <= 80: exact BF16 slices on the tensor cores
            CK(launch_cluster_adjoint_tc(as, (int)c.cl.size(), c.derr, c.wait_budget, s));
        } else if (c.osv_mixed && !c.cl.empty() && sh <= 216 * 1024) {
            // mixed modes: double-float products on the FP32 pipe
            CK(cudaFuncSetAttribute(k_cluster_adjoint_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
            count_launch();
            k_cluster_adjoint_df<<<(int)std::min<size_t>(c.cl.size(), 152), kAT, sh, s>>>(as);
        } else if (grid > 0) {
            count_launch();
            k_cluster_adjoint<double><<<grid, kThreads, 0, s>>>(a);
        }
        CK(cudaGetLastError());
    }
    {
        StageTimer t(c, "adj_pair_blocks");
        if (!c.pairs.empty()) { count_launch(); k_gk_tilde<<<(unsigned)c.pairs.size(), kThreads, 0, s>>>(c.pinfo.d, c.Tc, GK); }
        CK(cudaGetLastError());
        for (GemmBatch *g : {&gb_kc1, &gb_kc2, &gb_f1, &gb_f2, &gb_k1, &gb_k2, &gb_c1, &gb_c2}) CK(c.run_small(*g));
        CK(launch_block_copy(bc_hs.d, (int)bc_hs.h.size(), s));
    }
    {
        StageTimer t(c, "adj_half_transform");
        CK(c.run_dense(gb_z, oz_z));
        CK(c.run_dense(gb_db, oz_db));
        CK(c.run_dense(gb_dq, oz_dq));
    }
    StageTimer trelax(c, "adj_osv_relax");
    // A1 = (omega_mu - T)^{-1} P_perp dE/dQ on the discarded space.  FP64: P_perp -> tridiagonal basis ->
    // (Tri - omega_mu)^{-1} -> P_perp -> back to the virtual basis.  Mixed: the same chain in FP32 as a
    // preconditioner of FP64 residual corrections.
    if (c.osv_mixed && osv_project_rows_fits(nv, nm)) CK(osv_project_rows<double>(c.nosv, c.Q, dQ, n, nv, nm, s));
    else CK(osv_project_out<double>(c.nosv, c.Q, dQ, n, nv, nm, s));
    if (c.osv_mixed) {
        CK(osv_mixed_relax(c.refine, gb_at, n, nv, nm, c.Q, c.nosv, dQ, A1, s));
    } else {
        CK(osv_reflect<double>(c.tri_osv.d, n, nv, nm, c.nosv, dQ, 1, s));
        CK(osv_tri_shift_solve<double>(c.tri_osv.d, n, nv, nm, c.nosv, dQ, A1, c.tri_work, nullptr, 0, s));
        CK(osv_project_out<double>(c.nosv, c.Ytri, A1, n, nv, nm, s));
        CK(osv_reflect<double>(c.tri_osv.d, n, nv, nm, c.nosv, A1, 0, s));
    }
    CK(c.run_dense(gb_gt, oz_gt));
    {
        const int bx = (int)std::min<long long>(((long long)nv * nv + kThreads - 1) / kThreads, 64);
        count_launch();
        k_relax_sym<<<dim3(bx, n), kThreads, 0, s>>>(c.Zc, c.Tkk, c.eps, c.focc, n, nv, dF64);
        CK(cudaGetLastError());
    }
    CK(c.run_dense(gb_rb, oz_rb));
    const long long nb = c.aux_ptr[n] * (long long)nv;
    if (dB) {
        const int blocks = (int)std::min<long long>((nb + 255) / 256, 152LL * 16);
        if (c.B_dtype == 0) { count_launch(); k_out_b<double><<<blocks, 256, 0, s>>>(dB64, (double *)dB, nb, scale); }
        else { count_launch(); k_out_b<float><<<blocks, 256, 0, s>>>(dB64, (float *)dB, nb, scale); }
        CK(cudaGetLastError());
    }
    if (dF) {
        count_launch();
        k_out_b<double><<<1, 256, 0, s>>>(dF64, dF, (long long)n * n, scale);
        CK(cudaGetLastError());
    }
#undef CK
    return cudaSuccess;
}

}  // namespace osv
