// Cluster residual solver (Eq. 4 per cluster, Sec. 2.2.1), MBE(3) combination (Eqs. 28-32) and the
// Hylleraas energy (Eq. 3).  Plain FP64 solve, or FP32 iterations with FP64 iterative refinement (mixed modes).
//
// Each pair ij of a cluster works in the orthonormal pseudo-canonical basis Phi_ij = (Q_i Q_j) V_ij of its own
// domain (V^T S_(ij,ij) V = 1, V^T F_(ij,ij) V = diag(e)).  Projected on it, Eq. 4 reads
//   R~_ij = K~_ij + (e_a + e_b - f_ii - f_jj) T~_ij - sum_{k != j} f_kj S~ T~_ik S~^T - sum_{k != i} f_ik S~ T~_kj S~^T
// with S~ = Phi_ij^T Phi_(other pair) and k running over the cluster's LMOs; the Jacobi update is
// T~ -= R~ / (e_a + e_b - f_ii - f_jj).  One CTA owns one cluster for all its iterations; the small
// products run as block-cooperative register-tiled FP64 GEMMs.
#include <type_traits>

#include "kernels.cuh"
#include "launch.h"

namespace osv {

namespace {

constexpr int kThreads = 256;

// C (M x N) = alpha * op(A) op(B) (+ C if accumulate).  op(A)(m,k) = ta ? A[k*lda+m] : A[m*lda+k],
// op(B)(k,n) = tb ? B[n*ldb+k] : B[k*ldb+n].  Block-cooperative, 4 x 4 outputs per thread and tile.
template <class R>
__device__ void blk_gemm(int M, int N, int K, const R *__restrict__ A, long long lda, bool ta,
                         const R *__restrict__ B, long long ldb, bool tb, R *C, long long ldc, R alpha,
                         bool accumulate) {
    const int mt = (M + 3) >> 2, nt = (N + 3) >> 2;
    for (int t = threadIdx.x; t < mt * nt; t += blockDim.x) {
        const int bm = (t / nt) << 2, bn = (t % nt) << 2;
        R acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = R(0);
        for (int k = 0; k < K; ++k) {
            R a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int m = bm + i;
                a[i] = m < M ? (ta ? A[(long long)k * lda + m] : A[(long long)m * lda + k]) : R(0);
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

// Per-precision view of the operands of one residual evaluation.
template <class R>
struct View {
    const R *e;      // pair pseudo-canonical energies (pair e_off)
    const R *rhs;    // right-hand side: K~ by pair (rhs_by_slot = false) or a per-slot array
    bool rhs_by_slot;
    const R *S;      // coupling blocks
    R *T, *Rr, *G1;  // per-slot amplitudes, residuals; per-CTA scratch
    float *sm;       // mixed kernel: shared-memory staging (3 x ld^2 floats or 2 x ld^2 float pairs)
    int ld;
    bool df;         // FP64 evaluation in double-float arithmetic (mixed kernel)
};

// One coupling term of an FP64-accurate evaluation in double-float arithmetic on the FP32 pipe:
//   G1 = S~ T~'_q (written to the per-CTA FP64 scratch), then R~_p -= f G1 S~^T.
// Shared memory: sS[c][a] = S~(a, c) and sX[c][.] = T~'(c, .), later G1(., c), as (hi, lo) pairs.
__device__ void term_df(int rp, int rq, const double *__restrict__ Sb, long long lds, bool s_trans,
                        const double *__restrict__ Tq, long long ldt, bool t_trans, double f, double *Rp,
                        long long ldr, double *G1, long long ldg, float2 *sm, int ld) {
    float2 *sS = sm, *sX = sm + (long long)ld * ld;
    const int tid = threadIdx.x, nt = blockDim.x;
    // the FP64 operands land in the 8-byte slots of their (hi, lo) pairs by asynchronous copies; each thread then
    // splits the elements it copied
    auto stage = [&](bool conv) {
        for (int idx = tid; idx < rp * rq; idx += nt) {
            int a, c;
            if (s_trans) { c = idx / rp; a = idx % rp; } else { a = idx / rq; c = idx % rq; }
            float2 *dst = sS + c * ld + a;
            if (conv) *dst = split_df(*reinterpret_cast<const double *>(dst));
            else cpa_elem(dst, s_trans ? Sb + (long long)c * lds + a : Sb + (long long)a * lds + c, 8);
        }
        for (int idx = tid; idx < rq * rq; idx += nt) {
            int c, b;
            if (t_trans) { b = idx / rq; c = idx % rq; } else { c = idx / rq; b = idx % rq; }
            float2 *dst = sX + c * ld + b;
            if (conv) *dst = split_df(*reinterpret_cast<const double *>(dst));
            else cpa_elem(dst, t_trans ? Tq + (long long)b * ldt + c : Tq + (long long)c * ldt + b, 8);
        }
    };
    stage(false);
    cpa_wait();
    stage(true);
    __syncthreads();
    const int ta = (rp + 4) / 5, tq = (rq + 4) / 5;
    // G1 = S~ T~'.  When every tile has its own thread, the tiles stay in registers across one barrier and go to
    // sX (in place of T~') as (hi, lo) pairs; otherwise through the FP64 scratch.
    auto g1_tile = [&](int t, float (&hh)[5][5], float (&ll)[5][5]) {
        const int a0 = (t / tq) * 5, b0 = (t % tq) * 5;
        for (int c = 0; c < rq; ++c) {
            float2 x[5], y[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                x[i] = sS[c * ld + min(a0 + i, rp - 1)];
                y[i] = sX[c * ld + min(b0 + i, rq - 1)];
            }
            df_tile5(hh, ll, x, y);
        }
    };
    if (ta * tq <= nt) {
        float hh[5][5] = {}, ll[5][5] = {};
        const bool mine = tid < ta * tq;
        if (mine) g1_tile(tid, hh, ll);
        __syncthreads();
        if (mine) {
            const int a0 = (tid / tq) * 5, b0 = (tid % tq) * 5;
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j)
                    if (a0 + i < rp && b0 + j < rq) {
                        const float h = __fadd_rn(hh[i][j], ll[i][j]);
                        sX[(b0 + j) * ld + a0 + i] = make_float2(h, __fsub_rn(ll[i][j], __fsub_rn(h, hh[i][j])));
                    }
        }
        __syncthreads();
    } else {
        for (int t = tid; t < ta * tq; t += nt) {
            float hh[5][5] = {}, ll[5][5] = {};
            g1_tile(t, hh, ll);
            const int a0 = (t / tq) * 5, b0 = (t % tq) * 5;
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j)
                    if (a0 + i < rp && b0 + j < rq) G1[(long long)(a0 + i) * ldg + b0 + j] = df_val(hh[i][j], ll[i][j]);
        }
        __syncthreads();
        for (int idx = tid; idx < rp * rq; idx += nt) {   // sX[c][a] = G1(a, c)
            const int a = idx / rq, c = idx % rq;
            sX[c * ld + a] = split_df(G1[(long long)a * ldg + c]);
        }
        __syncthreads();
    }
    for (int t = tid; t < ta * ta; t += nt) {   // R~_p -= f G1 S~^T
        const int a0 = (t / ta) * 5, b0 = (t % ta) * 5;
        float hh[5][5] = {}, ll[5][5] = {};
        for (int c = 0; c < rq; ++c) {
            float2 x[5], y[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                x[i] = sX[c * ld + min(a0 + i, rp - 1)];
                y[i] = sS[c * ld + min(b0 + i, rp - 1)];
            }
            df_tile5(hh, ll, x, y);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (a0 + i < rp && b0 + j < rp) {
                    double *rp_ = Rp + (long long)(a0 + i) * ldr + b0 + j;
                    *rp_ = fma(-f, df_val(hh[i][j], ll[i][j]), *rp_);
                }
    }
    __syncthreads();
}

// One coupling term in FP32 with its operands staged in shared memory:
//   R~_p(a, b) -= f sum_c G1(a, c) S~(b, c),  G1 = S~ T~'_q,  S~ = op(Sb) (rp x rq), T~'_q = op(Tq) (rq x rq).
// sS[c][a] = S~(a, c), sT[c][b] = T~'(c, b), sG[c][a] = G1(a, c); 5 x 5 outputs per thread.
__device__ void term_f32(int rp, int rq, const float *__restrict__ Sb, long long lds, bool s_trans,
                         const float *__restrict__ Tq, long long ldt, bool t_trans, float f, float *Rp, long long ldr,
                         float *sm, int ld) {
    float *sS = sm, *sT = sm + (long long)ld * ld, *sG = sm + 2LL * ld * ld;
    const int tid = threadIdx.x, nt = blockDim.x;
    // asynchronous element copies into the transposed staging layouts (all in flight together)
    if (s_trans) {
        for (int idx = tid; idx < rp * rq; idx += nt) {
            const int c = idx / rp, a = idx % rp;
            cpa_elem(sS + c * ld + a, Sb + (long long)c * lds + a, 4);
        }
    } else {
        for (int idx = tid; idx < rp * rq; idx += nt) {
            const int a = idx / rq, c = idx % rq;
            cpa_elem(sS + c * ld + a, Sb + (long long)a * lds + c, 4);
        }
    }
    if (t_trans) {
        for (int idx = tid; idx < rq * rq; idx += nt) {
            const int b = idx / rq, c = idx % rq;
            cpa_elem(sT + c * ld + b, Tq + (long long)b * ldt + c, 4);
        }
    } else {
        for (int idx = tid; idx < rq * rq; idx += nt) {
            const int c = idx / rq, b = idx % rq;
            cpa_elem(sT + c * ld + b, Tq + (long long)c * ldt + b, 4);
        }
    }
    cpa_wait();
    __syncthreads();
    const int ta = (rp + 4) / 5, tq = (rq + 4) / 5;
    for (int t = tid; t < ta * tq; t += nt) {   // G1 = S~ T~'
        const int a0 = (t / tq) * 5, b0 = (t % tq) * 5;
        float acc[5][5] = {};
        for (int c = 0; c < rq; ++c) {
            float x[5], y[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                x[i] = sS[c * ld + a0 + i];
                y[i] = sT[c * ld + b0 + i];
            }
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j) acc[i][j] = fmaf(x[i], y[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (a0 + i < rp && b0 + j < rq) sG[(b0 + j) * ld + a0 + i] = acc[i][j];
    }
    __syncthreads();
    for (int t = tid; t < ta * ta; t += nt) {   // R~_p -= f G1 S~^T
        const int a0 = (t / ta) * 5, b0 = (t % ta) * 5;
        float acc[5][5] = {};
        for (int c = 0; c < rq; ++c) {
            float x[5], y[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                x[i] = sG[c * ld + a0 + i];
                y[i] = sS[c * ld + b0 + i];
            }
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j) acc[i][j] = fmaf(x[i], y[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (a0 + i < rp && b0 + j < rp) Rp[(long long)(a0 + i) * ldr + b0 + j] -= f * acc[i][j];
    }
    __syncthreads();
}

// R~ = rhs + D o T~ - sum_terms f S~ T~' S~^T for every slot of cluster C (Eq. 4 projected on the
// pseudo-canonical pair bases); returns max over slots of ||R~||_F.
template <class R>
__device__ double residual_eval(const SolveArgs &A, const ClusterInfo &C, const View<R> &v, double *red) {
    const int tid = threadIdx.x;
    for (int s = C.slot0; s < C.slot1; ++s) {
        const Slot S = A.slots[s];
        const PairInfo P = A.pairs[S.pair];
        const int r = A.rdim[S.pair], np = P.np;
        const R fii = (R)A.focc[(long long)P.i * A.n_occ + P.i], fjj = (R)A.focc[(long long)P.j * A.n_occ + P.j];
        const R *__restrict__ e = v.e + P.e_off;
        const R *__restrict__ rhs = v.rhs + (v.rhs_by_slot ? S.t_off : P.off);
        const R *__restrict__ Ts = v.T + S.t_off;
        R *__restrict__ Rs = v.Rr + S.t_off;
#pragma unroll 4
        for (int idx = tid; idx < r * r; idx += kThreads) {
            const int a = idx / r, b = idx % r;
            const long long o = (long long)a * np + b;
            Rs[o] = rhs[o] + (e[a] + e[b] - fii - fjj) * Ts[o];
        }
    }
    __syncthreads();
    for (int t = C.term0; t < C.term1; ++t) {
        const Term T = A.terms[t];
        const Slot Sd = A.slots[T.dst], Ss = A.slots[T.src];
        const PairInfo Pd = A.pairs[Sd.pair], Ps = A.pairs[Ss.pair];
        const int rp = A.rdim[Sd.pair], rq = A.rdim[Ss.pair];
        const R f = (R)A.focc[(long long)T.fx * A.n_occ + T.fy];
        const R *Sb = v.S + T.sblk;
        // stored block is (smaller pair id) x (larger pair id)
        const long long lds = T.s_trans ? Pd.np : Ps.np;
        if constexpr (std::is_same<R, float>::value) {
            term_f32(rp, rq, Sb, lds, T.s_trans, v.T + Ss.t_off, Ps.np, T.t_trans, f, v.Rr + Sd.t_off, Pd.np, v.sm, v.ld);
        } else if (v.df) {
            term_df(rp, rq, Sb, lds, T.s_trans, v.T + Ss.t_off, Ps.np, T.t_trans, f, v.Rr + Sd.t_off, Pd.np, v.G1, Ps.np,
                    reinterpret_cast<float2 *>(v.sm), v.ld);
        } else {
            // G1 = S~_pq T~'_q   (rp x rq)
            blk_gemm<R>(rp, rq, rq, Sb, lds, T.s_trans, v.T + Ss.t_off, Ps.np, T.t_trans, v.G1, Ps.np, R(1), false);
            __syncthreads();
            // R~_p -= f G1 S~_pq^T
            blk_gemm<R>(rp, rp, rq, v.G1, Ps.np, false, Sb, lds, !T.s_trans, v.Rr + Sd.t_off, Pd.np, -f, true);
            __syncthreads();
        }
    }
    double rmax = 0.0;
    for (int s = C.slot0; s < C.slot1; ++s) {
        const Slot S = A.slots[s];
        const int r = A.rdim[S.pair], np = A.pairs[S.pair].np;
        double ss = 0.0;
        for (int idx = tid; idx < r * r; idx += kThreads) {
            const double x = (double)v.Rr[S.t_off + (long long)(idx / r) * np + idx % r];
            ss += x * x;
        }
        rmax = fmax(rmax, sqrt(block_sum(ss, red)));
    }
    return rmax;
}

// Jacobi update T~ -= R~ / (e_a + e_b - f_ii - f_jj) on every slot of cluster C.
template <class R>
__device__ void jacobi_update(const SolveArgs &A, const ClusterInfo &C, const View<R> &v) {
    for (int s = C.slot0; s < C.slot1; ++s) {
        const Slot S = A.slots[s];
        const PairInfo P = A.pairs[S.pair];
        const int r = A.rdim[S.pair], np = P.np;
        const R fii = (R)A.focc[(long long)P.i * A.n_occ + P.i], fjj = (R)A.focc[(long long)P.j * A.n_occ + P.j];
        const R *__restrict__ e = v.e + P.e_off;
        R *__restrict__ Ts = v.T + S.t_off;
        const R *__restrict__ Rs = v.Rr + S.t_off;
#pragma unroll 4
        for (int idx = threadIdx.x; idx < r * r; idx += kThreads) {
            const int a = idx / r, b = idx % r;
            const long long o = (long long)a * np + b;
            Ts[o] -= Rs[o] / (e[a] + e[b] - fii - fjj);
        }
    }
    __syncthreads();
}

// Cluster Hylleraas energy: sum over ordered pairs of <K~ + R~, 2T~ - T~^T> (FP64).
__device__ double hylleraas(const SolveArgs &A, const ClusterInfo &C, double *red) {
    double E = 0.0;
    for (int s = C.slot0; s < C.slot1; ++s) {
        const Slot S = A.slots[s];
        const PairInfo P = A.pairs[S.pair];
        const int r = A.rdim[S.pair], np = P.np;
        double acc = 0.0;
        for (int idx = threadIdx.x; idx < r * r; idx += kThreads) {
            const int a = idx / r, b = idx % r;
            const long long o = (long long)a * np + b;
            const double tbar = 2.0 * A.T[S.t_off + o] - A.T[S.t_off + (long long)b * np + a];
            acc += (A.Kt[P.off + o] + A.R[S.t_off + o]) * tbar;
        }
        E += S.mult * block_sum(acc, red);
    }
    return E;
}

// Plain FP64 cluster solve: Jacobi iterations from T~ = 0 until max ||R~||_F <= tol.
__device__ void solve_cluster_fp64(const SolveArgs &A, int c) {
    const ClusterInfo C = A.clusters[c];
    __shared__ double red[kThreads / 32];
    View<double> v{A.e, A.Kt, false, A.sblk, A.T, A.R, A.G1 + (long long)blockIdx.x * A.gstride, nullptr, 0, false};
    bool conv = false;
    int it = 0;
    for (;; ++it) {
        const double rmax = residual_eval<double>(A, C, v, red);
        if (!(rmax > A.tol)) {   // converged (a NaN norm also stops here and is caught by energy())
            conv = rmax <= A.tol;
            break;
        }
        if (it >= A.max_iter) break;
        jacobi_update<double>(A, C, v);
    }
    const double E = hylleraas(A, C, red);
    if (threadIdx.x == 0) {
        A.E_cluster[c] = E;
        A.iters[c] = conv ? it : -1;
        if (A.evals64) A.evals64[c] = it + 1;
        if (A.evals32) A.evals32[c] = 0;
    }
}

// FP32 Jacobi solve of L(x) = -rhs from x = 0 until max ||R~||_F <= tol32 or the norm stops falling (by 10 %
// per iteration: the FP32 floor); returns the number of updates.  *fresh: the residual buffer belongs to the
// final x (false when the update cap ended the loop).
__device__ int solve32(const SolveArgs &A, const ClusterInfo &C, const View<float> &v, double tol32, int max_it,
                       double *red, bool *fresh = nullptr, int *nevals = nullptr) {
    double prev = INFINITY;
    int it = 0;
    bool ev = false;
    for (; it < max_it; ++it) {
        const double r = residual_eval<float>(A, C, v, red);
        ev = true;
        if (!(r > tol32) || r > 0.9 * prev) break;
        prev = r;
        jacobi_update<float>(A, C, v);
        ev = false;
    }
    if (fresh) *fresh = ev;
    if (nevals) *nevals += ev ? it + 1 : it;
    return it;
}

// A.R (FP64) <- A.R32 on every slot of cluster C; returns max over slots of ||R~||_F.
__device__ double promote_residual(const SolveArgs &A, const ClusterInfo &C, double *red) {
    double rmax = 0.0;
    for (int s = C.slot0; s < C.slot1; ++s) {
        const Slot S = A.slots[s];
        const int r = A.rdim[S.pair], np = A.pairs[S.pair].np;
        double ss = 0.0;
        for (int idx = threadIdx.x; idx < r * r; idx += kThreads) {
            const long long o = S.t_off + (long long)(idx / r) * np + idx % r;
            const double x = (double)A.R32[o];
            A.R[o] = x;
            ss += x * x;
        }
        rmax = fmax(rmax, sqrt(block_sum(ss, red)));
    }
    return rmax;
}

// Mixed cluster solve: FP32 Jacobi to the FP32 floor, then FP64 iterative refinement (FP64 residual, FP32
// correction solve with the FP64 residual as right-hand side, FP64 update) until max ||R~||_F <= tol in FP64.
// The energy uses the last FP64 residual, so its error is second order in the amplitude error (Eq. 3).
__device__ void solve_cluster_mixed(const SolveArgs &A, int c, float *stage32) {
    const ClusterInfo C = A.clusters[c];
    __shared__ double red[kThreads / 32];
    const int ld = A.np_max + 1;
    View<float> v32{A.e32, A.Kt32, false, A.sblk32, A.T32, A.R32, A.G1_32 + (long long)blockIdx.x * A.gstride, stage32, ld,
                    false};
    View<double> v64{A.e, A.Kt, false, A.sblk, A.T, A.R, A.G1 + (long long)blockIdx.x * A.gstride, stage32, ld, true};
    const int tid = threadIdx.x;
    auto zero32 = [&](float *x) {
        for (int s = C.slot0; s < C.slot1; ++s) {
            const Slot S = A.slots[s];
            const long long nn = (long long)A.pairs[S.pair].np * A.pairs[S.pair].np;
            for (long long i = tid; i < nn; i += kThreads) x[S.t_off + i] = 0.f;
        }
        __syncthreads();
    };
    zero32(A.T32);
    int ev32 = 0;
    int total = solve32(A, C, v32, fmax(A.tol, 1e-6), A.max_iter, red, nullptr, &ev32);
    // T64 = T32
    for (int s = C.slot0; s < C.slot1; ++s) {
        const Slot S = A.slots[s];
        const long long nn = (long long)A.pairs[S.pair].np * A.pairs[S.pair].np;
        for (long long i = tid; i < nn; i += kThreads) A.T[S.t_off + i] = (double)A.T32[S.t_off + i];
    }
    __syncthreads();
    bool conv = false;
    int evals = 0;
    View<float> vc{A.e32, A.H32, true, A.sblk32, A.T32, A.R32, v32.G1, stage32, ld, false};
    bool have_r = false;   // A.R already holds the residual of the current T64 (by linearity, below)
    double r64 = 0.0;
    for (int round = 0; round < 8; ++round) {
        if (!have_r) {
            r64 = residual_eval<double>(A, C, v64, red);
            ++evals;
        }
        if (!(r64 > A.tol)) {
            conv = r64 <= A.tol;
            break;
        }
        if (have_r) {   // the estimate missed the tolerance: evaluate afresh before the next correction
            have_r = false;
            --round;
            continue;
        }
        if (round == 7 || total >= A.max_iter) break;
        // correction: L(d) = -R64 in FP32 (rhs = R64), then T64 += d
        for (int s = C.slot0; s < C.slot1; ++s) {
            const Slot S = A.slots[s];
            const long long nn = (long long)A.pairs[S.pair].np * A.pairs[S.pair].np;
            for (long long i = tid; i < nn; i += kThreads) {
                A.H32[S.t_off + i] = (float)A.R[S.t_off + i];
                A.T32[S.t_off + i] = 0.f;
            }
        }
        __syncthreads();
        bool fresh = false;
        total += solve32(A, C, vc, fmax(1e-7 * r64, 0.1 * A.tol), A.max_iter, red, &fresh, &ev32);
        for (int s = C.slot0; s < C.slot1; ++s) {
            const Slot S = A.slots[s];
            const long long nn = (long long)A.pairs[S.pair].np * A.pairs[S.pair].np;
            for (long long i = tid; i < nn; i += kThreads) A.T[S.t_off + i] += (double)A.T32[S.t_off + i];
        }
        __syncthreads();
        // R is affine in T: R64(T + d) = R64(T) + L(d).  The correction solve's last evaluation holds
        // fl32(R64(T)) + L32(d) at its final d; L(d) is of the size of R64(T), so its FP32 error is ~2^-24 |R64(T)|
        // and the sum is the residual of the updated T64 to far below tol.  It is taken as such; a fresh FP64
        // evaluation follows only if it misses the tolerance.
        if (fresh) {
            r64 = promote_residual(A, C, red);
            have_r = true;
        }
    }
    const double E = hylleraas(A, C, red);
    if (tid == 0) {
        A.E_cluster[c] = E;
        A.iters[c] = conv ? total + evals - 1 : -1;
        if (A.evals64) A.evals64[c] = evals;
        if (A.evals32) A.evals32[c] = ev32;
    }
}

// One persistent grouped launch over every cluster: each CTA takes the next cluster of the cost-sorted order
// (most expensive first) from a device counter until none is left, so uneven clusters balance over the resident
// CTAs without a launch per cluster.
template <bool MIXED>
__global__ void __launch_bounds__(kThreads) k_residual(SolveArgs A) {
    __shared__ int s_q;
    extern __shared__ __align__(16) float stage32[];
    for (;;) {
        __syncthreads();   // every thread has read the previous index
        if (threadIdx.x == 0) s_q = atomicAdd(A.next, 1);
        __syncthreads();
        const int q = s_q;
        if (q >= A.ncl) break;
        if constexpr (MIXED) solve_cluster_mixed(A, A.order[q], stage32);
        else solve_cluster_fp64(A, A.order[q]);
    }
}

// Collective amplitudes: T~coll_p = sum over clusters containing p of w_c T~^c_p (Eqs. 28-32).
__global__ void k_combine(const PairInfo *__restrict__ pairs, const int *__restrict__ ptr,
                          const long long *__restrict__ src, const int *__restrict__ w,
                          const double *__restrict__ T, double *__restrict__ Tc) {
    const int p = blockIdx.x;
    const PairInfo P = pairs[p];
    const long long nn = (long long)P.np * P.np;
    for (long long idx = threadIdx.x; idx < nn; idx += blockDim.x) {
        double acc = 0.0;
        for (int q = ptr[p]; q < ptr[p + 1]; ++q) acc += w[q] * T[src[q] + idx];
        Tc[P.off + idx] = acc;
    }
}

// Per-pair linear energy term mult * <K~, 2T~coll - T~coll^T>.
__global__ void k_pair_linear(const PairInfo *__restrict__ pairs, const int *__restrict__ rdim,
                              const double *__restrict__ Kt, const double *__restrict__ Tc,
                              double *__restrict__ out) {
    const int p = blockIdx.x;
    const PairInfo P = pairs[p];
    const int r = rdim[p], np = P.np;
    __shared__ double red[kThreads / 32];
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
        const int a = idx / r, b = idx % r;
        acc += Kt[P.off + (long long)a * np + b] *
               (2.0 * Tc[P.off + (long long)a * np + b] - Tc[P.off + (long long)b * np + a]);
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[p] = (P.i == P.j ? 1.0 : 2.0) * acc;
}

// E = sum_c w_c E^c and E_lin = sum_p lin_p, deterministic order.
__global__ void k_energy_final(const double *__restrict__ Ec, const ClusterInfo *__restrict__ cl, int ncl,
                               const double *__restrict__ lin, int npairs, double *__restrict__ out) {
    __shared__ double red[kThreads / 32];
    double a = 0.0, b = 0.0;
    for (int c = threadIdx.x; c < ncl; c += blockDim.x) a += cl[c].weight * Ec[c];
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) b += lin[p];
    a = block_sum(a, red);
    b = block_sum(b, red);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

// One-step posterior correction over the collective amplitudes (Sec. 3): every stored pair p is a pseudo-cluster
// whose single slot is p and whose terms run over the LMOs k of the clusters that hold both LMOs of p (the slots
// and the amplitudes are those of the pairs: t_off = the pair's offset into Tsrc / Rdst).  One CTA per pair: R~_p of
// Eq. 4 at Tsrc and its Frobenius norm, FP64 (df = false) or double-float on the FP32 pipe (df = true).
__global__ void __launch_bounds__(kThreads) k_posterior_eval(SolveArgs A, const double *__restrict__ Tsrc,
                                                             double *__restrict__ Rdst, double *__restrict__ rnorm,
                                                             bool df) {
    const int p = blockIdx.x;
    const ClusterInfo C = A.clusters[p];
    __shared__ double red[kThreads / 32];
    extern __shared__ __align__(16) float stage[];
    View<double> v{A.e, A.Kt, false, A.sblk, const_cast<double *>(Tsrc), Rdst, A.G1 + (long long)blockIdx.x * A.gstride,
                   stage, A.np_max + 1, df};
    const double rn = residual_eval<double>(A, C, v, red);
    if (threadIdx.x == 0) rnorm[p] = rn;
}

// T' = T - R~ / (e_a + e_b - f_ii - f_jj) on the r_p x r_p block of every pair (the cluster solver's preconditioned
// step); zero elsewhere.
__global__ void k_posterior_step(const PairInfo *__restrict__ pairs, const int *__restrict__ rdim,
                                 const double *__restrict__ e, const double *__restrict__ focc, int n_occ,
                                 const double *__restrict__ T, const double *__restrict__ R, double *__restrict__ T2) {
    const int p = blockIdx.x;
    const PairInfo P = pairs[p];
    const int r = rdim[p], np = P.np;
    const double fii = focc[(long long)P.i * n_occ + P.i], fjj = focc[(long long)P.j * n_occ + P.j];
    for (int idx = threadIdx.x; idx < np * np; idx += blockDim.x) {
        const int a = idx / np, b = idx % np;
        const long long o = P.off + idx;
        T2[o] = (a < r && b < r) ? T[o] - R[o] / (e[P.e_off + a] + e[P.e_off + b] - fii - fjj) : 0.0;
    }
}

// Per pair: mult_p <K~_p + R~_p, 2T~_p - T~_p^T> (Eq. 3 over the ordered pairs ij and ji, which are transposes).
__global__ void k_pair_functional(const PairInfo *__restrict__ pairs, const int *__restrict__ rdim,
                                  const double *__restrict__ Kt, const double *__restrict__ T,
                                  const double *__restrict__ R, double *__restrict__ out) {
    const int p = blockIdx.x;
    const PairInfo P = pairs[p];
    const int r = rdim[p], np = P.np;
    __shared__ double red[kThreads / 32];
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
        const int a = idx / r, b = idx % r;
        const long long o = P.off + (long long)a * np + b;
        acc += (Kt[o] + R[o]) * (2.0 * T[o] - T[P.off + (long long)b * np + a]);
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[p] = (P.i == P.j ? 1.0 : 2.0) * acc;
}

}  // namespace

cudaError_t launch_posterior(const SolveArgs &a, int npairs, const double *Tc, double *R1, double *T2, double *R2,
                             double *rnorm, double *E1, double *E2, bool df, cudaStream_t s) {
    if (npairs <= 0) return cudaSuccess;
    const int ld = a.np_max + 1;
    const size_t sh = df ? 2 * (size_t)ld * ld * sizeof(float2) : 0;
    cudaError_t e;
    if (sh > 48 * 1024 && (e = cudaFuncSetAttribute(k_posterior_eval, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)sh)) != cudaSuccess)
        return e;
    count_launch(5);
    k_posterior_eval<<<npairs, kThreads, sh, s>>>(a, Tc, R1, rnorm, df);
    k_posterior_step<<<npairs, kThreads, 0, s>>>(a.pairs, a.rdim, a.e, a.focc, a.n_occ, Tc, R1, T2);
    k_posterior_eval<<<npairs, kThreads, sh, s>>>(a, T2, R2, rnorm + npairs, df);
    k_pair_functional<<<npairs, kThreads, 0, s>>>(a.pairs, a.rdim, a.Kt, Tc, R1, E1);
    k_pair_functional<<<npairs, kThreads, 0, s>>>(a.pairs, a.rdim, a.Kt, T2, R2, E2);
    return cudaGetLastError();
}

cudaError_t launch_residual(const SolveArgs &a, int nclusters, bool mixed, cudaStream_t s) {
    if (nclusters <= 0) return cudaSuccess;
    const int ld = a.np_max + 1;
    const size_t sh = mixed ? std::max(3 * (size_t)ld * ld * sizeof(float), 2 * (size_t)ld * ld * sizeof(float2)) : 0;
    auto kern = mixed ? k_residual<true> : k_residual<false>;
    cudaError_t e;
    if (sh > 48 * 1024 && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh)) != cudaSuccess)
        return e;
    // resident CTAs: occupancy x SMs, at most one per cluster (the per-CTA scratch G1 has nclusters slots)
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, sh)) != cudaSuccess)
        return e;
    const int grid = std::max(1, std::min(nclusters, std::max(per_sm, 1) * sms));
    if ((e = cudaMemsetAsync(a.next, 0, sizeof(int), s)) != cudaSuccess) return e;
    count_launch();
    kern<<<grid, kThreads, sh, s>>>(a);
    return cudaGetLastError();
}

namespace {
__global__ void k_to_f32(const double *__restrict__ in, float *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}
}  // namespace

cudaError_t launch_to_f32(const double *in, float *out, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    k_to_f32<<<(int)std::min<long long>((n + 255) / 256, 152LL * 8), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_combine(const PairInfo *pairs, int npairs, const int *ptr, const long long *src, const int *w,
                           const double *T, double *Tc, cudaStream_t s) {
    if (npairs <= 0) return cudaSuccess;
    count_launch();
    k_combine<<<npairs, kThreads, 0, s>>>(pairs, ptr, src, w, T, Tc);
    return cudaGetLastError();
}

cudaError_t launch_energy(const PairInfo *pairs, const int *rdim, const double *Kt, const double *Tc, int npairs,
                          double *lin, const double *Ec, const ClusterInfo *cl, int ncl, double *out,
                          cudaStream_t s) {
    if (npairs > 0) { count_launch(); k_pair_linear<<<npairs, kThreads, 0, s>>>(pairs, rdim, Kt, Tc, lin); }
    count_launch();
    k_energy_final<<<1, kThreads, 0, s>>>(Ec, cl, ncl, lin, npairs, out);
    return cudaGetLastError();
}

}  // namespace osv
