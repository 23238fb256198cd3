// C ABI of libosvmbe: host planner (cluster selection, pair / coupling / slot layout, GEMM batches) and the
// launch sequence of the MBE(3)-OSV-MP2 hot path.  All device shapes are planned from the padded OSV width
// nmax, so no step waits for the device to learn the data-dependent OSV counts: padded OSV rows are zero
// and padded pair-basis columns are dropped by the overlap eigenvalue test.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "ctx.h"
#include "launch.h"

using namespace osv;

namespace {
thread_local std::string g_noctx_err;
}

namespace osv {
std::atomic<long long> g_launches{0};
void set_noctx_error(const std::string &msg) { g_noctx_err = msg; }
}

namespace {

osv_status check_params(osv_ctx *c, const osv_params *p) {
    if (!p) return c->fail(OSV_ERR_INVALID, "params is NULL");
    if (!(p->tol > 0.0) || p->max_iter < 1) return c->fail(OSV_ERR_INVALID, "tol must be > 0 and max_iter >= 1");
    if (p->n_osv_fixed <= 0 && p->n_osv_max <= 0) return c->fail(OSV_ERR_INVALID, "n_osv_max must be > 0");
    if (p->mbe_order < 0 || p->mbe_order > 3) return c->fail(OSV_ERR_INVALID, "mbe_order must be 0..3");
    if (!(p->tau_red >= 0.0) || !(p->r2b >= 0.0) || !(p->r3b >= 0.0) || !std::isfinite(p->l_osv))
        return c->fail(OSV_ERR_INVALID, "tau_red, r2b, r3b must be >= 0 and l_osv finite");
    if (p->precision == OSV_MIXED_TF32X3)
        return c->fail(OSV_ERR_INVALID, "OSV_MIXED_TF32X3 is reserved: split TF32 with FP32 accumulation misses the "
                                        "1e-6 Eh bar; use OSV_MIXED_BF16X4");
    if (p->precision != OSV_FP64 && p->precision != OSV_MIXED_BF16X4)
        return c->fail(OSV_ERR_INVALID, "unknown precision");
    return OSV_OK;
}

osv_status check_problem(osv_ctx *c, const osv_problem *pb) {
    if (!pb) return c->fail(OSV_ERR_INVALID, "problem is NULL");
    if (pb->n_occ < 1 || pb->n_vir < 1 || pb->n_aux < 1) return c->fail(OSV_ERR_INVALID, "sizes must be >= 1");
    if (pb->n_vir > 4096) return c->fail(OSV_ERR_INVALID, "n_vir > 4096 is not supported");
    if (!pb->centres || !pb->aux_ptr || !pb->aux_idx) return c->fail(OSV_ERR_INVALID, "host arrays are NULL");
    if (pb->aux_ptr[0] != 0) return c->fail(OSV_ERR_INVALID, "aux_ptr[0] must be 0");
    for (int i = 0; i < pb->n_occ; ++i) {
        const int64_t a0 = pb->aux_ptr[i], a1 = pb->aux_ptr[i + 1];
        if (a1 <= a0) return c->fail(OSV_ERR_INVALID, "every fitting domain must be non-empty");
        for (int64_t q = a0; q < a1; ++q) {
            if (pb->aux_idx[q] < 0 || pb->aux_idx[q] >= pb->n_aux)
                return c->fail(OSV_ERR_INVALID, "aux_idx out of range");
            if (q > a0 && pb->aux_idx[q] <= pb->aux_idx[q - 1])
                return c->fail(OSV_ERR_INVALID, "aux_idx lists must be strictly increasing");
        }
    }
    for (int i = 0; i < 3 * pb->n_occ; ++i)
        if (!std::isfinite(pb->centres[i])) return c->fail(OSV_ERR_INVALID, "non-finite centre");
    if (pb->B_dtype != 0 && pb->B_dtype != 1) return c->fail(OSV_ERR_INVALID, "B_dtype must be 0 or 1");
    return OSV_OK;
}

// clusters: sorted member lists.  Distance rule of clusters_build, or (s2b != NULL) the OSV-overlap rule of
// clusters_build_osv (Sec. 2.2.1, Eqs. 2bscreen and 3bscreen): pair ij kept iff s2b_ij > l2b, triple ijk kept iff
// its three pairs are kept and (s2b_ij + s2b_ik + s2b_jk) / 3 > l3b (s2b read at i < j).
void select_clusters(osv_ctx *c, const double *s2b = nullptr, double l2b = 0.0, double l3b = 0.0) {
    const int n = c->n_occ;
    const osv_params &p = c->prm;
    c->cl.clear();
    c->ncl_order[0] = c->ncl_order[1] = c->ncl_order[2] = 0;
    if (p.mbe_order == 0) {
        std::vector<int> all(n);
        std::iota(all.begin(), all.end(), 0);
        c->cl.push_back(all);
        c->ncl_order[0] = 1;
        return;
    }
    auto dist = [&](int i, int j) {
        double s = 0.0;
        for (int x = 0; x < 3; ++x) {
            const double d = c->centres[3 * i + x] - c->centres[3 * j + x];
            s += d * d;
        }
        return std::sqrt(s);
    };
    for (int i = 0; i < n; ++i) c->cl.push_back({i});
    c->ncl_order[0] = n;
    if (p.mbe_order < 2) return;
    if (s2b) {
        auto s = [&](int i, int j) { return s2b[(size_t)i * n + j]; };
        std::vector<char> kp((size_t)n * n, 0);
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j)
                if (s(i, j) > l2b) {
                    kp[(size_t)i * n + j] = 1;
                    c->cl.push_back({i, j});
                    ++c->ncl_order[1];
                }
        if (p.mbe_order < 3) return;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                if (!kp[(size_t)i * n + j]) continue;
                for (int k = j + 1; k < n; ++k)
                    if (kp[(size_t)i * n + k] && kp[(size_t)j * n + k] && (s(i, j) + s(i, k) + s(j, k)) / 3.0 > l3b) {
                        c->cl.push_back({i, j, k});
                        ++c->ncl_order[2];
                    }
            }
        return;
    }
    std::vector<char> keep((size_t)n * n, 0);
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (dist(i, j) <= p.r2b) {
                keep[(size_t)i * n + j] = 1;
                c->cl.push_back({i, j});
                ++c->ncl_order[1];
            }
    if (p.mbe_order < 3) return;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            if (!keep[(size_t)i * n + j]) continue;
            for (int k = j + 1; k < n; ++k)
                if (keep[(size_t)i * n + k] && keep[(size_t)j * n + k] && dist(i, j) <= p.r3b && dist(i, k) <= p.r3b &&
                    dist(j, k) <= p.r3b) {
                    c->cl.push_back({i, j, k});
                    ++c->ncl_order[2];
                }
        }
}

// w_c = sum over selected supersets c' of c of (-1)^(|c'|-|c|), accumulated from each selected c' over its
// selected subsets.
void mbe_weights(osv_ctx *c) {
    std::map<std::vector<int>, int> idx;
    for (size_t q = 0; q < c->cl.size(); ++q) idx[c->cl[q]] = (int)q;
    c->cl_w.assign(c->cl.size(), 0);
    for (const auto &big : c->cl) {
        const int m = (int)big.size();
        if (m > 3) {   // the single full cluster of mbe_order 0
            c->cl_w[idx[big]] += 1;
            continue;
        }
        for (int mask = 1; mask < (1 << m); ++mask) {
            std::vector<int> sub;
            for (int t = 0; t < m; ++t)
                if (mask >> t & 1) sub.push_back(big[t]);
            auto it = idx.find(sub);
            if (it != idx.end()) c->cl_w[it->second] += ((m - (int)sub.size()) % 2) ? -1 : 1;
        }
    }
}

osv_status clusters_setup(osv_ctx *c, const osv_problem *pb, const osv_params *prm, int *n_clusters,
                          const double *s2b, double l2b, double l3b) {
    if (!c) return OSV_ERR_INVALID;
    osv_status st;
    if ((st = check_params(c, prm)) != OSV_OK) return st;
    if ((st = check_problem(c, pb)) != OSV_OK) return st;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    c->release();
    c->prm = *prm;
    c->n_occ = pb->n_occ;
    c->n_vir = pb->n_vir;
    c->n_aux = pb->n_aux;
    c->centres.assign(pb->centres, pb->centres + 3 * pb->n_occ);
    c->aux_ptr.assign(pb->aux_ptr, pb->aux_ptr + pb->n_occ + 1);
    c->aux_idx.assign(pb->aux_idx, pb->aux_idx + pb->aux_ptr[pb->n_occ]);
    select_clusters(c, s2b, l2b, l3b);
    mbe_weights(c);
    const int n = c->n_occ;
    // stored pairs i <= j: every diagonal pair and every pair inside a cluster
    c->pairs.clear();
    c->pair_id.clear();
    for (int i = 0; i < n; ++i) {
        c->pair_id[(long long)i * n + i] = (int)c->pairs.size();
        c->pairs.push_back({i, i});
    }
    for (const auto &m : c->cl)
        for (size_t a = 0; a < m.size(); ++a)
            for (size_t b = a + 1; b < m.size(); ++b) {
                const long long key = (long long)m[a] * n + m[b];
                if (!c->pair_id.count(key)) {
                    c->pair_id[key] = (int)c->pairs.size();
                    c->pairs.push_back({m[a], m[b]});
                }
            }
    c->nb.assign(n, {});
    for (int i = 0; i < n; ++i) c->nb[i].push_back(i);
    for (const auto &pr : c->pairs)
        if (pr.first != pr.second) {
            c->nb[pr.first].push_back(pr.second);
            c->nb[pr.second].push_back(pr.first);
        }
    for (auto &v : c->nb) std::sort(v.begin(), v.end());
    c->have_clusters = true;
    if (n_clusters) {
        n_clusters[0] = c->ncl_order[0];
        n_clusters[1] = c->ncl_order[1];
        n_clusters[2] = c->ncl_order[2];
    }
    return OSV_OK;
}

}  // namespace

extern "C" {

const char *osv_last_error(const osv_ctx *ctx) { return ctx ? ctx->err.c_str() : g_noctx_err.c_str(); }

osv_status osv_create(osv_ctx **ctx, void *cuda_stream) {
    if (!ctx) return OSV_ERR_INVALID;
    *ctx = nullptr;
    osv_ctx *c = new (std::nothrow) osv_ctx();
    if (!c) return OSV_ERR_OOM;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        g_noctx_err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        delete c;
        return OSV_ERR_CUDA;
    }
    c->stream = (cudaStream_t)cuda_stream;
    *ctx = c;
    return OSV_OK;
}

osv_status osv_destroy(osv_ctx *ctx) {
    if (!ctx) return OSV_ERR_INVALID;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    ctx->release();
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    for (auto &e : ctx->pev) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
    delete ctx;
    return OSV_OK;
}

osv_status clusters_build(osv_ctx *c, const osv_problem *pb, const osv_params *prm, int *n_clusters) {
    return clusters_setup(c, pb, prm, n_clusters, nullptr, 0.0, 0.0);
}

osv_status clusters_build_osv(osv_ctx *c, const osv_problem *pb, const osv_params *prm, const double *s2b, double l2b,
                              double l3b, int *n_clusters) {
    if (!c) return OSV_ERR_INVALID;
    if (!s2b || !std::isfinite(l2b) || !std::isfinite(l3b))
        return c->fail(OSV_ERR_INVALID, "s2b must be non-NULL and l2b, l3b finite");
    if (pb && pb->n_occ > 0)
        for (long long q = 0; q < (long long)pb->n_occ * pb->n_occ; ++q)
            if (!std::isfinite(s2b[q])) return c->fail(OSV_ERR_INVALID, "non-finite s2b entry");
    return clusters_setup(c, pb, prm, n_clusters, s2b, l2b, l3b);
}

}  // extern "C"

namespace {

// Host plan of slots, terms, couplings and combine lists (needs nmax).
void plan_clusters(osv_ctx *c) {
    const int n = c->n_occ, nm = c->nmax;
    // pairs
    c->pinfo.h.clear();
    long long off = 0, eoff = 0;
    for (const auto &pr : c->pairs) {
        PairInfo P{};
        P.i = pr.first;
        P.j = pr.second;
        P.np = pr.first == pr.second ? nm : 2 * nm;
        P.off = off;
        P.e_off = eoff;
        off += (long long)P.np * P.np;
        eoff += P.np;
        c->pinfo.h.push_back(P);
    }
    c->pair_mat = off;
    c->pair_vec = eoff;
    // slots and terms
    c->slots.h.clear();
    c->terms.h.clear();
    c->cinfo.h.clear();
    c->couplings.clear();
    c->coupling_id.clear();
    long long toff = 0;
    for (size_t q = 0; q < c->cl.size(); ++q) {
        const auto &m = c->cl[q];
        ClusterInfo C{};
        C.slot0 = (int)c->slots.h.size();
        C.term0 = (int)c->terms.h.size();
        C.weight = c->cl_w[q];
        C.size = (int)m.size();
        std::map<int, int> slot_of_pair;
        for (size_t a = 0; a < m.size(); ++a)
            for (size_t b = a; b < m.size(); ++b) {
                const int p = c->pid(m[a], m[b]);
                Slot S{};
                S.pair = p;
                S.cluster = (int)q;
                S.t_off = toff;
                S.mult = a == b ? 1 : 2;
                toff += (long long)c->pinfo.h[p].np * c->pinfo.h[p].np;
                slot_of_pair[p] = (int)c->slots.h.size();
                c->slots.h.push_back(S);
            }
        C.slot1 = (int)c->slots.h.size();
        for (int s = C.slot0; s < C.slot1; ++s) {
            const int p = c->slots.h[s].pair;
            const int i = c->pinfo.h[p].i, j = c->pinfo.h[p].j;
            auto add = [&](int x, int y, int fx, int fy) {   // amplitude t_xy, coefficient f[fx][fy]
                const int qp = c->pid(x, y);
                Term T{};
                T.dst = s;
                T.src = slot_of_pair[qp];
                T.fx = fx;
                T.fy = fy;
                T.t_trans = x > y ? 1 : 0;
                const int pa = std::min(p, qp), pb = std::max(p, qp);
                const long long key = (long long)pa * (long long)c->pairs.size() + pb;
                auto it = c->coupling_id.find(key);
                int cid;
                if (it == c->coupling_id.end()) {
                    cid = (int)c->couplings.size();
                    c->coupling_id[key] = cid;
                    c->couplings.push_back({pa, pb});
                } else {
                    cid = it->second;
                }
                T.coupling = cid;
                T.s_trans = p > qp ? 1 : 0;
                c->terms.h.push_back(T);
            };
            for (int k : m) {
                if (k != j) add(i, k, k, j);   // -f_kj S t_ik S
                if (k != i) add(k, j, i, k);   // -f_ik S t_kj S
            }
        }
        C.term1 = (int)c->terms.h.size();
        c->cinfo.h.push_back(C);
    }
    c->slot_mat = toff;
    // coupling block offsets, then patch the terms
    c->coup_off.assign(c->couplings.size(), 0);
    long long coff = 0;
    for (size_t q = 0; q < c->couplings.size(); ++q) {
        c->coup_off[q] = coff;
        coff += (long long)c->pinfo.h[c->couplings[q].first].np * c->pinfo.h[c->couplings[q].second].np;
    }
    c->coup_mat = coff;
    for (auto &T : c->terms.h) T.sblk = c->coup_off[T.coupling];
    // processing order: most expensive clusters first
    c->order.h.resize(c->cl.size());
    std::iota(c->order.h.begin(), c->order.h.end(), 0);
    std::vector<long long> cost(c->cl.size(), 0);
    for (size_t q = 0; q < c->cl.size(); ++q)
        for (int t = c->cinfo.h[q].term0; t < c->cinfo.h[q].term1; ++t) {
            const long long a = c->pinfo.h[c->slots.h[c->terms.h[t].dst].pair].np;
            const long long b = c->pinfo.h[c->slots.h[c->terms.h[t].src].pair].np;
            cost[q] += a * b * (a + b);
        }
    std::stable_sort(c->order.h.begin(), c->order.h.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    // combine lists: for each pair, the slots holding it and their cluster weights
    std::vector<std::vector<std::pair<long long, int>>> lst(c->pairs.size());
    for (const auto &S : c->slots.h) lst[S.pair].push_back({S.t_off, c->cl_w[S.cluster]});
    c->comb_ptr.h.assign(1, 0);
    c->comb_src.h.clear();
    c->comb_w.h.clear();
    for (const auto &l : lst) {
        for (const auto &x : l) {
            c->comb_src.h.push_back(x.first);
            c->comb_w.h.push_back(x.second);
        }
        c->comb_ptr.h.push_back((int)c->comb_src.h.size());
    }
    c->gstride = 4LL * nm * nm;
    (void)n;
}

// positions of the common fitting functions of LMOs i and j in their own lists
void common_domain(const osv_ctx *c, int i, int j, std::vector<int> &pi, std::vector<int> &pj) {
    pi.clear();
    pj.clear();
    int64_t a = c->aux_ptr[i], b = c->aux_ptr[j];
    const int64_t ae = c->aux_ptr[i + 1], be = c->aux_ptr[j + 1];
    while (a < ae && b < be) {
        if (c->aux_idx[a] == c->aux_idx[b]) {
            pi.push_back(int(a - c->aux_ptr[i]));
            pj.push_back(int(b - c->aux_ptr[j]));
            ++a;
            ++b;
        } else if (c->aux_idx[a] < c->aux_idx[b]) {
            ++a;
        } else {
            ++b;
        }
    }
}

bool full_domains(const osv_ctx *c) {
    for (int i = 0; i < c->n_occ; ++i)
        if (c->a_of(i) != c->n_aux) return false;
    return true;
}

osv_status build_plan(osv_ctx *c) {
    cudaError_t e;
    const int n = c->n_occ, nv = c->n_vir, nm = c->nmax;
    const long long nv2 = (long long)nv * nv;
#define ALLOC(ptr, cnt) \
    if ((e = c->dalloc(ptr, (size_t)(cnt))) != cudaSuccess) return c->cuda_fail(e, "cudaMalloc " #ptr)
    ALLOC(c->Tkk, n * nv2);
    ALLOC(c->Zc, n * nv2);
    ALLOC(c->omega, (long long)n * nv);
    ALLOC(c->nosv, n);
    ALLOC(c->derr, 1);
    ALLOC(c->Q, (long long)n * nm * nv);
    ALLOC(c->Qe, (long long)n * nm * nv);
    const long long np_ = (long long)c->pairs.size();
    ALLOC(c->sblk, np_ * nm * nm);
    ALLOC(c->fblk, np_ * nm * nm);
    c->w_off.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) c->w_off[i + 1] = c->w_off[i] + (long long)c->nb[i].size() * nm * c->a_of(i);
    ALLOC(c->W, c->w_off[n]);
    ALLOC(c->Kp, c->pair_mat);
    ALLOC(c->Sp, c->pair_mat);
    ALLOC(c->Fp, c->pair_mat);
    ALLOC(c->X, c->pair_mat);
    ALLOC(c->Fx, c->pair_mat);
    ALLOC(c->V, c->pair_mat);
    ALLOC(c->Kt, c->pair_mat);
    ALLOC(c->ptmp, c->pair_mat);
    ALLOC(c->Tc, c->pair_mat);
    ALLOC(c->pz, c->pair_mat);
    ALLOC(c->sw, c->pair_vec);
    ALLOC(c->pe, c->pair_vec);
    ALLOC(c->pd, c->pair_vec);
    ALLOC(c->pee, c->pair_vec);
    ALLOC(c->ptau, c->pair_vec);
    ALLOC(c->rdim, np_);
    ALLOC(c->Scp, c->coup_mat);
    ALLOC(c->Stil, c->coup_mat);
    ALLOC(c->ctmp, c->coup_mat);
    ALLOC(c->Tslot, c->slot_mat);
    ALLOC(c->Rslot, c->slot_mat);
    ALLOC(c->G1, (long long)c->cl.size() * c->gstride);
    ALLOC(c->Ecl, c->cl.size());
    ALLOC(c->iters, c->cl.size());
    ALLOC(c->lin, np_);
    ALLOC(c->Eout, 2);
    ALLOC(c->e32, c->pair_vec);
    ALLOC(c->Kt32, c->pair_mat);
    ALLOC(c->S32, c->coup_mat);
    ALLOC(c->T32, c->slot_mat);
    ALLOC(c->R32, c->slot_mat);
    ALLOC(c->H32, c->slot_mat);
    ALLOC(c->G1_32, (long long)c->cl.size() * c->gstride);
    ALLOC(c->evals64, c->cl.size());
    ALLOC(c->evals32, c->cl.size());
    ALLOC(c->work_next, 1);
    if (c->B_dtype == 1) {
        ALLOC(c->B64own, c->aux_ptr[n] * (long long)nv);
        c->B64 = c->B64own;
    } else {
        c->B64 = (const double *)c->B_in;
    }
    const bool full = full_domains(c);

    // --- a1: Gram products (ka|kb) = B_k B_k^T
    for (int k = 0; k < n; ++k) {
        const long long a = c->a_of(k);
        c->gb_gram.add(gemm(nv, nv, (int)a, c->B64 + c->b_off(k), a, 0, c->B64 + c->b_off(k), a, 1,
                            c->Tkk + k * nv2, nv));
    }
    // --- a2: OSV eigenproblems.  FP64: tridiagonal route (multisection + inverse iteration of the kept vectors).
    // Mixed: the same route in FP32, then FP64 Rayleigh-Ritz refinement of the n_max leading eigenpairs.
    c->tri_osv.h.clear();
    if (!c->osv_mixed) {
        ALLOC(c->Awork, n * nv2);
        ALLOC(c->dsc, (long long)n * nv);
        ALLOC(c->esc, (long long)n * nv);
        ALLOC(c->tausc, (long long)n * nv);
        ALLOC(c->Ytri, (long long)n * nm * nv);
        ALLOC(c->tri_work, 4LL * n * nm * nv);
        for (int k = 0; k < n; ++k) {
            TriDesc D{};
            D.A = c->Awork + k * nv2;
            D.lda = nv;
            D.n = nv;
            D.d = c->dsc + (long long)k * nv;
            D.e = c->esc + (long long)k * nv;
            D.tau = c->tausc + (long long)k * nv;
            D.w = c->omega + (long long)k * nv;
            c->tri_osv.h.push_back(D);
        }
    } else {
        OsvRefine &r = c->refine;
        const long long blk = (long long)n * nm * nv;
        ALLOC(r.A32, n * nv2);
        ALLOC(r.d32, (long long)n * nv);
        ALLOC(r.e32, (long long)n * nv);
        ALLOC(r.tau32, (long long)n * nv);
        ALLOC(r.w32, (long long)n * nv);
        ALLOC(r.Y32, blk);
        ALLOC(r.work32, 4 * blk);
        ALLOC(r.X32, blk);
        ALLOC(r.Z32, blk);
        ALLOC(r.QW[0], 2 * blk);
        ALLOC(r.QW[1], 2 * blk);
        ALLOC(r.GH, 2LL * n * nm * nm);
        ALLOC(r.Ct, (long long)n * nm * nm);
        ALLOC(r.lam, (long long)n * nm);
        ALLOC(r.AT, blk);
        ALLOC(r.RS, blk);
        ALLOC(r.nm_all, n);
        // compact-WY factors only where the blocked reflector product fits shared memory (n_vir up to ~1700);
        // larger orders apply the reflectors one by one
        ALLOC(r.Twy, (long long)osv_wy_floats(n, nv));
        std::vector<int> all(n, nm);
        if ((e = cudaMemcpy(r.nm_all, all.data(), n * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
            return c->cuda_fail(e, "upload n_max");
        r.tri_h.clear();
        for (int k = 0; k < n; ++k) {
            TriDesc32 D{};
            D.A = r.A32 + k * nv2;
            D.lda = nv;
            D.n = nv;
            D.d = r.d32 + (long long)k * nv;
            D.e = r.e32 + (long long)k * nv;
            D.tau = r.tau32 + (long long)k * nv;
            D.w = r.w32 + (long long)k * nv;
            r.tri_h.push_back(D);
        }
        ALLOC(r.tri_d, n);
        if ((e = cudaMemcpy(r.tri_d, r.tri_h.data(), n * sizeof(TriDesc32), cudaMemcpyHostToDevice)) != cudaSuccess)
            return c->cuda_fail(e, "upload tri32");
        const long long per = (long long)nm * nv;
        for (int x = 0; x < 2; ++x) {
            const int y = x ^ 1;
            for (int k = 0; k < n; ++k) {
                double *qx = r.QW[x] + 2 * per * k, *qy = r.QW[y] + 2 * per * k;
                const double *ct = r.Ct + (long long)k * nm * nm;
                // W = Q T;  [G; H] = [Q; W] Q^T;  [Q; W] <- Ct [Q; W];  final Q = Ct Q
                r.gb_w[x].add(gemm(nm, nv, nv, qx, nv, 0, c->Tkk + k * nv2, nv, 0, qx + per, nv));
                r.gb_gh[x].add(gemm(2 * nm, nm, nv, qx, nv, 0, qx, nv, 1, r.GH + 2LL * k * nm * nm, nm));
                r.gb_rot[x].add(gemm(nm, nv, nm, ct, nm, 0, qx, nv, 0, qy, nv));
                r.gb_rot[x].add(gemm(nm, nv, nm, ct, nm, 0, qx + per, nv, 0, qy + per, nv));
                r.gb_fin[x].add(gemm(nm, nv, nm, ct, nm, 0, qx, nv, 0, c->Q + per * k, nv));
            }
        }
    }
    // --- a3: LMO-pair blocks s_ij = Q_i Q_j^T, phi_ij = Q_i diag(eps) Q_j^T (rows = OSVs)
    for (size_t p = 0; p < c->pairs.size(); ++p) {
        const int i = c->pairs[p].first, j = c->pairs[p].second;
        const double *Qi = c->Q + (long long)i * nm * nv;
        c->gb_sf.add(gemm(nm, nm, nv, Qi, nv, 0, c->Q + (long long)j * nm * nv, nv, 1, c->sblk + p * nm * nm, nm));
        c->gb_sf.add(gemm(nm, nm, nv, Qi, nv, 0, c->Qe + (long long)j * nm * nv, nv, 1, c->fblk + p * nm * nm, nm));
    }
    // --- a4: half transforms W^{(i)} = [Q_m]_{m in nb(i)} B_i (stacked rows), then K blocks
    c->rows_w.h.clear();
    std::vector<size_t> rows_at(n);
    for (int i = 0; i < n; ++i) {
        rows_at[i] = c->rows_w.h.size();
        for (int m : c->nb[i])
            for (int mu = 0; mu < nm; ++mu) c->rows_w.h.push_back(m * nm + mu);
    }
    c->kidx.h.clear();
    struct KRef { size_t pi, pj; int len; };
    std::map<long long, KRef> kref;
    if (!full) {
        std::vector<int> pi, pj;
        for (const auto &pr : c->pairs) {
            if (pr.first == pr.second) continue;
            common_domain(c, pr.first, pr.second, pi, pj);
            KRef r{c->kidx.h.size(), c->kidx.h.size() + pi.size(), (int)pi.size()};
            c->kidx.h.insert(c->kidx.h.end(), pi.begin(), pi.end());
            c->kidx.h.insert(c->kidx.h.end(), pj.begin(), pj.end());
            kref[(long long)pr.first * n + pr.second] = r;
        }
    }
    if ((e = c->upload(c->rows_w)) != cudaSuccess) return c->cuda_fail(e, "upload rows");
    if ((e = c->upload(c->kidx)) != cudaSuccess) return c->cuda_fail(e, "upload kidx");
    for (int i = 0; i < n; ++i) {
        const long long a = c->a_of(i);
        GemmDesc g = gemm((int)c->nb[i].size() * nm, (int)a, nv, c->Q, nv, 0, c->B64 + c->b_off(i), a, 0,
                          c->W + c->w_off[i], a);
        g.a_rows = c->rows_w.d + rows_at[i];
        c->gb_w.add(g);
    }
    for (size_t p = 0; p < c->pairs.size(); ++p) {
        const int i = c->pairs[p].first, j = c->pairs[p].second;
        const PairInfo &P = c->pinfo.h[p];
        const long long ai = c->a_of(i), aj = c->a_of(j);
        if (i == j) {
            const double *Wii = c->W + c->w_off[i] + (long long)c->slot_of(i, i) * nm * ai;
            c->gb_k.add(gemm(nm, nm, (int)ai, Wii, ai, 0, Wii, ai, 1, c->Kp + P.off, P.np));
            continue;
        }
        const int dom[2] = {i, j};
        for (int x = 0; x < 2; ++x)
            for (int y = 0; y < 2; ++y) {
                const double *Wa = c->W + c->w_off[i] + (long long)c->slot_of(i, dom[x]) * nm * ai;
                const double *Wb = c->W + c->w_off[j] + (long long)c->slot_of(j, dom[y]) * nm * aj;
                GemmDesc g = gemm(nm, nm, full ? c->n_aux : 0, Wa, ai, 0, Wb, aj, 1,
                                  c->Kp + P.off + (long long)x * nm * P.np + (long long)y * nm, P.np);
                if (!full) {
                    const KRef &r = kref[(long long)i * n + j];
                    g.K = r.len;
                    g.k_idx_a = c->kidx.d + r.pi;
                    g.k_idx_b = c->kidx.d + r.pj;
                }
                c->gb_k.add(g);
            }
    }
    // --- a5: pair bases.  S_pp / F_pp assembled from the LMO-pair blocks
    c->bc_pair.h.clear();
    auto blk = [&](double *base, int x, int y, bool fock) -> BlockCopy {
        BlockCopy b{};
        const int q = c->pid(x, y);
        b.src = (fock ? c->fblk : c->sblk) + (long long)q * nm * nm;
        b.trans = x > y ? 1 : 0;
        b.rows = b.cols = nm;
        b.lds = nm;
        b.scale = 1.0;
        b.dst = base;
        return b;
    };
    for (size_t p = 0; p < c->pairs.size(); ++p) {
        const PairInfo &P = c->pinfo.h[p];
        const int dom[2] = {P.i, P.j};
        const int nd = P.i == P.j ? 1 : 2;
        for (int x = 0; x < nd; ++x)
            for (int y = 0; y < nd; ++y)
                for (int f = 0; f < 2; ++f) {
                    BlockCopy b = blk((f ? c->Fp : c->Sp) + P.off + (long long)x * nm * P.np + (long long)y * nm,
                                      dom[x], dom[y], f);
                    b.ldd = P.np;
                    c->bc_pair.h.push_back(b);
                }
    }
    c->eig_s.h.clear();
    c->eig_f.h.clear();
    for (size_t p = 0; p < c->pairs.size(); ++p) {
        const PairInfo &P = c->pinfo.h[p];
        EighDesc D{};
        D.A = c->Sp + P.off;
        D.lda = P.np;
        D.n = P.np;
        D.w = c->sw + P.e_off;
        D.Zt = c->Sp + P.off;
        D.ldz = P.np;
        D.zwork = c->pz + P.off;
        D.d = c->pd + P.e_off;
        D.e = c->pee + P.e_off;
        D.tau = c->ptau + P.e_off;
        c->eig_s.h.push_back(D);
        D.A = c->Fx + P.off;
        D.Zt = c->Fx + P.off;
        D.w = c->pe + P.e_off;
        D.n_dev = nullptr;   // patched after rdim upload below
        c->eig_f.h.push_back(D);
    }
    for (size_t p = 0; p < c->pairs.size(); ++p) {
        const PairInfo &P = c->pinfo.h[p];
        c->eig_f.h[p].n_dev = c->rdim + p;
        // F' = X^T F X
        c->gb_fx1.add(gemm(P.np, P.np, P.np, c->Fp + P.off, P.np, 0, c->X + P.off, P.np, 0, c->ptmp + P.off, P.np));
        c->gb_fx2.add(gemm(P.np, P.np, P.np, c->X + P.off, P.np, 1, c->ptmp + P.off, P.np, 0, c->Fx + P.off, P.np));
        // V = X W  (W(k, c) = Wt[c][k])
        c->gb_v.add(gemm(P.np, P.np, P.np, c->X + P.off, P.np, 0, c->Fx + P.off, P.np, 1, c->V + P.off, P.np));
        // K~ = V^T K V
        c->gb_kt1.add(gemm(P.np, P.np, P.np, c->Kp + P.off, P.np, 0, c->V + P.off, P.np, 0, c->ptmp + P.off, P.np));
        c->gb_kt2.add(gemm(P.np, P.np, P.np, c->V + P.off, P.np, 1, c->ptmp + P.off, P.np, 0, c->Kt + P.off, P.np));
    }
    // coupling blocks S~_(pa,pb) = V_pa^T S_(pa,pb) V_pb
    c->bc_coup.h.clear();
    for (size_t q = 0; q < c->couplings.size(); ++q) {
        const PairInfo &Pa = c->pinfo.h[c->couplings[q].first], &Pb = c->pinfo.h[c->couplings[q].second];
        const int da[2] = {Pa.i, Pa.j}, db[2] = {Pb.i, Pb.j};
        const int na = Pa.i == Pa.j ? 1 : 2, nbb = Pb.i == Pb.j ? 1 : 2;
        for (int x = 0; x < na; ++x)
            for (int y = 0; y < nbb; ++y) {
                BlockCopy b = blk(c->Scp + c->coup_off[q] + (long long)x * nm * Pb.np + (long long)y * nm, da[x],
                                  db[y], false);
                b.ldd = Pb.np;
                c->bc_coup.h.push_back(b);
            }
        c->gb_c1.add(gemm(Pa.np, Pb.np, Pb.np, c->Scp + c->coup_off[q], Pb.np, 0, c->V + Pb.off, Pb.np, 0,
                          c->ctmp + c->coup_off[q], Pb.np));
        c->gb_c2.add(gemm(Pa.np, Pb.np, Pa.np, c->V + Pa.off, Pa.np, 1, c->ctmp + c->coup_off[q], Pb.np, 0,
                          c->Stil + c->coup_off[q], Pb.np));
    }
#undef ALLOC
    for (HostDev<PairInfo> *h : {&c->pinfo}) if ((e = c->upload(*h)) != cudaSuccess) return c->cuda_fail(e, "upload");
    if ((e = c->upload(c->slots)) != cudaSuccess) return c->cuda_fail(e, "upload slots");
    if ((e = c->upload(c->terms)) != cudaSuccess) return c->cuda_fail(e, "upload terms");
    if ((e = c->upload(c->cinfo)) != cudaSuccess) return c->cuda_fail(e, "upload clusters");
    if ((e = c->upload(c->order)) != cudaSuccess) return c->cuda_fail(e, "upload order");
    if ((e = c->upload(c->comb_ptr)) != cudaSuccess) return c->cuda_fail(e, "upload comb");
    if ((e = c->upload(c->comb_src)) != cudaSuccess) return c->cuda_fail(e, "upload comb");
    if ((e = c->upload(c->comb_w)) != cudaSuccess) return c->cuda_fail(e, "upload comb");
    if ((e = c->upload(c->bc_pair)) != cudaSuccess) return c->cuda_fail(e, "upload bc");
    if ((e = c->upload(c->bc_coup)) != cudaSuccess) return c->cuda_fail(e, "upload bc");
    if (!c->osv_mixed && (e = c->upload(c->tri_osv)) != cudaSuccess) return c->cuda_fail(e, "upload tri");
    if ((e = c->upload(c->eig_s)) != cudaSuccess) return c->cuda_fail(e, "upload eig");
    if ((e = c->upload(c->eig_f)) != cudaSuccess) return c->cuda_fail(e, "upload eig");
    for (GemmBatch *g : {&c->gb_gram, &c->gb_sf, &c->gb_w, &c->gb_k, &c->gb_fx1, &c->gb_fx2, &c->gb_v, &c->gb_kt1,
                         &c->gb_kt2, &c->gb_c1, &c->gb_c2})
        if ((e = gemm_batch_upload(*g)) != cudaSuccess) return c->cuda_fail(e, "upload gemm batch");
    if (c->osv_mixed)
        for (int x = 0; x < 2; ++x)
            for (GemmBatch *g : {&c->refine.gb_w[x], &c->refine.gb_gh[x], &c->refine.gb_rot[x], &c->refine.gb_fin[x]})
                if ((e = gemm_batch_upload(*g)) != cudaSuccess) return c->cuda_fail(e, "upload refine batch");
    if ((e = bf16x4_batch_prepare(c->gb_gram, c->oz_gram)) != cudaSuccess ||
        (e = bf16x4_batch_prepare(c->gb_w, c->oz_w)) != cudaSuccess || (e = bf16x4_batch_prepare(c->gb_k, c->oz_k)) != cudaSuccess)
        return c->cuda_fail(e, "tensor-core tiling");
    if (c->prm.precision == OSV_MIXED_BF16X4 &&
        (e = c->oz_reserve((size_t)std::max({c->oz_gram.scratch_bytes, c->oz_w.scratch_bytes, c->oz_k.scratch_bytes}))) !=
            cudaSuccess)
        return c->cuda_fail(e, "slice scratch");
    return OSV_OK;
}

// Plan-time autotuner (mixed precision): launch shapes are timed on the device with CUDA events and the fastest
// is kept.  Timed runs read the plan's own buffers whatever they hold (the work of these kernels does not depend on
// the values) and write only outputs that the build overwrites afterwards.
//   - the FP32 Householder tridiagonalisation: a pair of CTAs per matrix, or one CTA per matrix and two per SM;
//   - the double-float GEMM tile shape (64x64, 80x80, 48x80, 80x48, 48x48) of every batch of the build whose
//     problems all have beta = 0 and no atomic accumulation (re-running such a batch is harmless).
// The report (osv_autotune_report) lists, per item, the rule's choice, the tuned choice and the timings.
osv_status autotune_plan(osv_ctx *c) {
    c->tune_report.clear();
    if (c->osv_mixed && c->tri_force >= 0) c->refine.tri_variant = c->tri_force;
    if (!c->autotune || !c->osv_mixed) return OSV_OK;
    cudaStream_t s = c->stream;
    cudaEvent_t a = c->take_event(), b = c->take_event();
    cudaError_t e = cudaSuccess;
    auto timed = [&](const std::function<cudaError_t()> &run, int reps) -> double {
        if (e != cudaSuccess) return 0.0;
        if ((e = cudaEventRecord(a, s)) != cudaSuccess) return 0.0;
        for (int q = 0; q < reps && e == cudaSuccess; ++q) e = run();
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        return ms / reps;
    };
    const char *shape_name[5] = {"64x64", "80x80", "48x80", "80x48", "48x48"};
    std::string js = "{";
    double gain = 0.0, spent = 0.0;
    // 1. tridiagonalisation launch shape (unless fixed by osv_set_tridiag_variant), timed on the first
    // min(n_occ, 2 x 152) matrices (a full wave of the widest variant); a variant this GPU cannot launch (no room
    // for its cluster) is skipped
    if (c->tri_force >= 0) {
        js += "\"tridiag\": {\"choice\": \"fixed\"}";
    } else {
        const char *tri_name[kTriVariants] = {"cta_pair", "single_cta_2_per_sm", "cluster_4", "cluster_8", "cluster_16",
                                              "delayed_2", "delayed_2_2_per_sm", "delayed_4", "staged_2_2_per_sm",
                                              "staged_2", "staged_2_depth_2", "staged_2_depth_3", "staged_2_8_rows"};
        const int m = std::min(c->n_occ, 2 * 152), nv = c->n_vir;
        double t[kTriVariants];
        int best = 0;
        for (int v = 0; v < kTriVariants; ++v) {
            t[v] = -1.0;
            if (e != cudaSuccess) break;
            t[v] = timed([&] { return osv_tridiag<float>(c->refine.tri_d, m, nv, s, v); }, 1);
            if (e == cudaErrorNotSupported) {
                e = cudaSuccess;
                t[v] = -1.0;
                continue;
            }
            if (e == cudaSuccess && t[v] < t[best]) best = v;
        }
        // a larger batch: the two fastest on the subset again on the whole batch (waves of different sizes)
        double tf[2] = {-1.0, -1.0};
        int fin[2] = {best, -1};
        if (e == cudaSuccess && m < c->n_occ) {
            for (int v = 0; v < kTriVariants; ++v)
                if (v != best && t[v] >= 0.0 && (fin[1] < 0 || t[v] < t[fin[1]])) fin[1] = v;
            for (int f = 0; f < 2 && e == cudaSuccess; ++f)
                if (fin[f] >= 0) {
                    tf[f] = timed([&] { return osv_tridiag<float>(c->refine.tri_d, c->n_occ, nv, s, fin[f]); }, 1);
                    spent += tf[f];
                }
            if (e == cudaSuccess && fin[1] >= 0 && tf[1] < tf[0]) best = fin[1];
        }
        if (e == cudaSuccess) {
            c->refine.tri_variant = best;
            gain += (t[0] - t[best]) * c->n_occ / m;
            std::string ms = "{";
            for (int v = 0; v < kTriVariants; ++v) {
                char b2[64];
                if (t[v] >= 0.0) {
                    spent += t[v];
                    snprintf(b2, sizeof b2, "%s\"%s\": %.3f", ms.size() > 1 ? ", " : "", tri_name[v], t[v]);
                } else {
                    snprintf(b2, sizeof b2, "%s\"%s\": null", ms.size() > 1 ? ", " : "", tri_name[v]);
                }
                ms += b2;
            }
            char buf[160];
            snprintf(buf, sizeof buf, "\"tridiag\": {\"rule\": \"cta_pair\", \"choice\": \"%s\", \"matrices_timed\": %d, \"ms\": ",
                     tri_name[best], m);
            js += buf + ms + "}";
            if (fin[1] >= 0 && tf[1] >= 0.0) {
                char b3[160];
                snprintf(b3, sizeof b3, ", \"ms_whole_batch\": {\"%s\": %.3f, \"%s\": %.3f}", tri_name[fin[0]], tf[0],
                         tri_name[fin[1]], tf[1]);
                js += b3;
            }
            js += "}";
        }
    }
    // 2. double-float GEMM tile shapes
    std::vector<std::pair<std::string, GemmBatch *>> batches = {
        {"sf_blocks", &c->gb_sf}, {"pair_fx1", &c->gb_fx1}, {"pair_fx2", &c->gb_fx2}, {"pair_v", &c->gb_v},
        {"pair_kt1", &c->gb_kt1}, {"pair_kt2", &c->gb_kt2}, {"coupling_c1", &c->gb_c1}, {"coupling_c2", &c->gb_c2}};
    for (int x = 0; x < 2; ++x) {
        const std::string k = std::to_string(x);
        batches.push_back({"refine_w" + k, &c->refine.gb_w[x]});
        batches.push_back({"refine_gh" + k, &c->refine.gb_gh[x]});
        batches.push_back({"refine_rot" + k, &c->refine.gb_rot[x]});
        batches.push_back({"refine_fin" + k, &c->refine.gb_fin[x]});
    }
    js += ", \"gemm_df\": {";
    bool first = true;
    for (auto &nb : batches) {
        GemmBatch &g = *nb.second;
        if (g.h.empty() || g.tiles == 0) continue;
        bool ok = true;
        for (const GemmDesc &d : g.h) ok = ok && d.beta == 0.0 && !d.atomic;
        if (!ok) continue;
        double t[5];
        for (int sh = 0; sh < 5; ++sh) {
            if ((e = gemm_batch_set_df_shape(g, sh)) != cudaSuccess) break;
            gemm_batch_run_df(g, s);   // warm-up
            t[sh] = timed([&] { return gemm_batch_run_df(g, s); }, 3);
            spent += 4 * t[sh];
        }
        if (e != cudaSuccess) break;
        int best = 0;
        for (int sh = 1; sh < 5; ++sh)
            if (t[sh] < t[best]) best = sh;
        if ((e = gemm_batch_set_df_shape(g, best)) != cudaSuccess) break;
        gain += t[g.df_rule] - t[best];
        char buf[512];
        snprintf(buf, sizeof buf, "%s\"%s\": {\"rule\": \"%s\", \"choice\": \"%s\", \"ms\": [%.4f, %.4f, %.4f, %.4f, %.4f]}",
                 first ? "" : ", ", nb.first.c_str(), shape_name[g.df_rule], shape_name[best], t[0], t[1], t[2], t[3], t[4]);
        js += buf;
        first = false;
    }
    c->pool.push_back(a);
    c->pool.push_back(b);
    if (e != cudaSuccess) return c->cuda_fail(e, "autotune");
    char buf[160];
    snprintf(buf, sizeof buf, "}, \"gain_ms_per_build\": %.3f, \"tuning_ms\": %.1f}", gain, spent);
    js += buf;
    c->tune_report = js;
    return OSV_OK;
}

osv_status run_osv_build(osv_ctx *c) {
    cudaError_t e;
    cudaStream_t s = c->stream;
    const int n = c->n_occ, nv = c->n_vir, nm = c->nmax;
#define CK(x, what) \
    do { \
        if ((e = (x)) != cudaSuccess) return c->cuda_fail(e, what); \
    } while (0)
    CK(cudaMemsetAsync(c->derr, 0, sizeof(int), s), "memset");
    if (c->B_dtype == 1) {
        StageTimer t(*c, "b_to_fp64");
        CK(launch_f32_to_f64((const float *)c->B_in, c->B64own, c->aux_ptr[n] * (long long)nv, s), "f32->f64");
    }
    {
        StageTimer t(*c, "tkk_gram");
        CK(c->run_dense(c->gb_gram, c->oz_gram), "gram");
        if (c->osv_mixed) {
            CK(launch_tkk_scale<float>(c->Tkk, c->refine.A32, c->eps, c->focc, n, nv, c->derr, s), "tkk");
        } else {
            CK(launch_tkk_scale<double>(c->Tkk, c->Awork, c->eps, c->focc, n, nv, c->derr, s), "tkk");
        }
    }
    {
        StageTimer t(*c, "osv_eigh");
        if (c->osv_mixed) {
            CK(osv_mixed_eigh(c->refine, n, nv, nm, c->Q, c->omega, c->nosv, c->prm.l_osv, c->prm.n_osv_fixed,
                              c->derr, s), "osv refine");
        } else {
            CK(osv_tridiag<double>(c->tri_osv.d, n, nv, s), "osv tridiag");
            CK(osv_tri_eigvals<double>(c->tri_osv.d, n, nv, nm, s), "osv eigenvalues");
            CK(launch_osv_count(c->omega, nv, c->nosv, n, nm, c->prm.l_osv, c->prm.n_osv_fixed, s), "osv count");
            CK(cudaMemsetAsync(c->Ytri, 0, (size_t)n * nm * nv * sizeof(double), s), "memset Y");
            CK(osv_tri_kept_vectors<double>(c->tri_osv.d, n, nv, nm, c->nosv, c->Ytri, c->tri_work, s), "osv vectors");
            CK(cudaMemcpyAsync(c->Q, c->Ytri, (size_t)n * nm * nv * sizeof(double), cudaMemcpyDeviceToDevice, s),
               "copy Q");
            CK(osv_reflect<double>(c->tri_osv.d, n, nv, nm, c->nosv, c->Q, 0, s), "osv back-transform");
        }
        CK(launch_scale_cols(c->Q, c->eps, c->Qe, (long long)n * nm, nv, s), "Qe");
    }
    {
        StageTimer t(*c, "sf_blocks");
        CK(c->run_small(c->gb_sf), "s/f blocks");
    }
    {
        StageTimer t(*c, "half_transform");
        CK(c->run_dense(c->gb_w, c->oz_w), "half transform");
    }
    {
        StageTimer t(*c, "k_blocks");
        CK(c->run_dense(c->gb_k, c->oz_k), "K blocks");
    }
    {
        StageTimer t(*c, "pair_basis");
        // pair eigenproblems: FP32 Jacobi + FP64 polish in the mixed modes, FP64 Jacobi otherwise (large
        // orders: Householder + QL)
        const bool pmix = c->prm.precision != OSV_FP64 && 2 * nm <= kJacobiMixedMax;
        auto pair_eigh = [&](const HostDev<EighDesc> &d) -> cudaError_t {
            const int np_ = (int)c->pairs.size();
            if (pmix) return eigh_small_jacobi_mixed(d.d, np_, 2 * nm, c->derr, s);
            if (2 * nm <= kJacobiMax) return eigh_small_jacobi(d.d, np_, 2 * nm, c->derr, s);
            return eigh_batched(d.d, np_, 2 * nm, 1, c->derr, s);
        };
        CK(launch_block_copy(c->bc_pair.d, (int)c->bc_pair.h.size(), s), "pair assemble");
        CK(pair_eigh(c->eig_s), "pair overlap eigh");
        CK(launch_pair_x(c->pinfo.d, (int)c->pairs.size(), c->Sp, c->sw, c->X, c->rdim, c->prm.tau_red, s), "pair x");
        CK(c->run_small(c->gb_fx1), "fx1");
        CK(c->run_small(c->gb_fx2), "fx2");
        CK(pair_eigh(c->eig_f), "pair fock eigh");
        CK(launch_clean_w(c->pinfo.d, (int)c->pairs.size(), c->rdim, c->Fx, c->pe, s), "clean");
        CK(c->run_small(c->gb_v), "V");
    }
    {
        StageTimer t(*c, "pair_transform");
        CK(c->run_small(c->gb_kt1), "kt1");
        CK(c->run_small(c->gb_kt2), "kt2");
        CK(launch_block_copy(c->bc_coup.d, (int)c->bc_coup.h.size(), s), "coupling assemble");
        CK(c->run_small(c->gb_c1), "c1");
        CK(c->run_small(c->gb_c2), "c2");
        if (c->prm.precision != OSV_FP64) {   // FP32 copies for the mixed residual iterations
            CK(launch_to_f32(c->pe, c->e32, c->pair_vec, s), "e32");
            CK(launch_to_f32(c->Kt, c->Kt32, c->pair_mat, s), "Kt32");
            CK(launch_to_f32(c->Stil, c->S32, c->coup_mat, s), "S32");
        }
    }
#undef CK
    return OSV_OK;
}

osv_status error_word_status(osv_ctx *c, int h) {
    if (h == kDevEighNoConv) return c->fail(OSV_ERR_TIMEOUT, "eigensolver hit its iteration cap");
    if (h == kDevNonFinite) return c->fail(OSV_ERR_NUMERIC, "non-finite value in T_kk (check B, eps, f_occ)");
    if (h == kDevTimeout) return c->fail(OSV_ERR_TIMEOUT, "a bounded tensor-core wait expired");
    return OSV_OK;
}

osv_status device_error(osv_ctx *c) {
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, c->derr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return c->cuda_fail(e, "read error word");
    return error_word_status(c, h);
}

}  // namespace

extern "C" {

osv_status osv_build(osv_ctx *c, const osv_problem *pb, const osv_params *prm, int *n_osv_out) {
    if (!c) return OSV_ERR_INVALID;
    if (!c->have_clusters) return c->fail(OSV_ERR_INVALID, "clusters_build must precede osv_build");
    osv_status st;
    if ((st = check_params(c, prm)) != OSV_OK) return st;
    if ((st = check_problem(c, pb)) != OSV_OK) return st;
    if (pb->n_occ != c->n_occ || pb->n_vir != c->n_vir || pb->n_aux != c->n_aux ||
        memcmp(pb->aux_ptr, c->aux_ptr.data(), (c->n_occ + 1) * sizeof(int64_t)) != 0 ||
        memcmp(pb->aux_idx, c->aux_idx.data(), c->aux_idx.size() * sizeof(int32_t)) != 0 ||
        prm->mbe_order != c->prm.mbe_order || prm->r2b != c->prm.r2b || prm->r3b != c->prm.r3b)
        return c->fail(OSV_ERR_INVALID, "problem or cluster parameters differ from clusters_build");
    if (!pb->f_occ || !pb->eps_vir || !pb->B) return c->fail(OSV_ERR_INVALID, "device arrays are NULL");
    cudaSetDevice(c->device);
    const int nmax = prm->n_osv_fixed > 0 ? std::min(prm->n_osv_fixed, pb->n_vir) : std::min(prm->n_osv_max, pb->n_vir);
    const bool mixed = prm->precision != OSV_FP64 && nmax <= kRefineMaxN;
    const bool replan = !c->built || nmax != c->nmax || pb->B_dtype != c->B_dtype || pb->B != c->B_in ||
                        mixed != c->osv_mixed;
    c->prm = *prm;
    c->focc = pb->f_occ;
    c->eps = pb->eps_vir;
    if (replan) {
        if (c->stream) cudaStreamSynchronize(c->stream);
        c->release();
        c->nmax = nmax;
        c->osv_mixed = mixed;
        c->B_in = pb->B;
        c->B_dtype = pb->B_dtype;
        plan_clusters(c);
        if ((st = build_plan(c)) != OSV_OK || (st = autotune_plan(c)) != OSV_OK) {
            c->release();
            return st;
        }
        c->built = true;
    }
    c->solved = false;
    if ((st = run_osv_build(c)) != OSV_OK) return st;
    if (n_osv_out) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return c->cuda_fail(e, "osv_build");
        if ((st = device_error(c)) != OSV_OK) return st;
        e = cudaMemcpy(n_osv_out, c->nosv, c->n_occ * sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return c->cuda_fail(e, "copy n_osv");
    }
    return OSV_OK;
}

osv_status osv_overlap_metric(osv_ctx *c, const osv_problem *pb, const osv_params *prm, double *s2b_out) {
    if (!c) return OSV_ERR_INVALID;
    if (!s2b_out) return c->fail(OSV_ERR_INVALID, "s2b_out is NULL");
    if (!prm) return c->fail(OSV_ERR_INVALID, "params is NULL");
    // the OSVs of every LMO: a plan of the 1b clusters alone (the cluster list is chosen afterwards)
    osv_params p1 = *prm;
    p1.mbe_order = 1;
    osv_status st;
    if ((st = clusters_setup(c, pb, &p1, nullptr, nullptr, 0.0, 0.0)) != OSV_OK) return st;
    if ((st = osv_build(c, pb, &p1, nullptr)) != OSV_OK) return st;
    const int n = c->n_occ, nm = c->nmax, nv = c->n_vir;
    const long long nr = (long long)n * nm;
    double *G = nullptr, *s = nullptr;
    cudaError_t e;
    if ((e = c->dalloc(G, (size_t)(nr * nr))) != cudaSuccess || (e = c->dalloc(s, (size_t)n * n)) != cudaSuccess)
        return c->cuda_fail(e, "cudaMalloc metric");
    // G = Q Q^T over all OSV rows, one problem per LMO's rows (the dense back end of the precision mode)
    GemmBatch gb;
    for (int i = 0; i < n; ++i)
        gb.add(gemm(nm, (int)nr, nv, c->Q + (long long)i * nm * nv, nv, 0, c->Q, nv, 1, G + (long long)i * nm * nr, nr));
    osv::TcTiles oz;
    e = gemm_batch_upload(gb);
    if (e == cudaSuccess && c->prm.precision == OSV_MIXED_BF16X4) {
        e = bf16x4_batch_prepare(gb, oz);
        if (e == cudaSuccess) e = c->oz_reserve((size_t)oz.scratch_bytes);
    }
    if (e == cudaSuccess) {
        StageTimer t(*c, "osv_metric");
        e = c->run_dense(gb, oz);
        if (e == cudaSuccess) e = launch_s2b(G, c->nosv, n, nm, s, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    gemm_batch_free(gb);
    osv::tc_tiles_free(oz);
    if (e != cudaSuccess) return c->cuda_fail(e, "overlap metric");
    if ((st = device_error(c)) != OSV_OK) return st;
    if ((e = cudaMemcpy(s2b_out, s, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return c->cuda_fail(e, "copy s2b");
    return OSV_OK;
}

osv_status cluster_residual_solve(osv_ctx *c, int *n_iter_out, int32_t *cluster_status) {
    if (!c) return OSV_ERR_INVALID;
    if (!c->built) return c->fail(OSV_ERR_INVALID, "osv_build must precede cluster_residual_solve");
    cudaSetDevice(c->device);
    cudaError_t e;
    SolveArgs a{};
    a.clusters = c->cinfo.d;
    a.order = c->order.d;
    a.slots = c->slots.d;
    a.terms = c->terms.d;
    a.pairs = c->pinfo.d;
    a.rdim = c->rdim;
    a.e = c->pe;
    a.Kt = c->Kt;
    a.sblk = c->Stil;
    a.focc = c->focc;
    a.n_occ = c->n_occ;
    a.T = c->Tslot;
    a.R = c->Rslot;
    a.G1 = c->G1;
    a.gstride = c->gstride;
    a.E_cluster = c->Ecl;
    a.iters = c->iters;
    a.tol = c->prm.tol;
    a.max_iter = c->prm.max_iter;
    a.e32 = c->e32;
    a.Kt32 = c->Kt32;
    a.sblk32 = c->S32;
    a.T32 = c->T32;
    a.R32 = c->R32;
    a.H32 = c->H32;
    a.G1_32 = c->G1_32;
    a.evals64 = c->evals64;
    a.evals32 = c->evals32;
    a.np_max = 2 * c->nmax;
    a.next = c->work_next;
    a.ncl = (int)c->cl.size();
    if ((e = cudaMemsetAsync(c->Tslot, 0, c->slot_mat * sizeof(double), c->stream)) != cudaSuccess)
        return c->cuda_fail(e, "memset T");
    if ((e = cudaMemsetAsync(c->Rslot, 0, c->slot_mat * sizeof(double), c->stream)) != cudaSuccess)
        return c->cuda_fail(e, "memset R");
    {
        StageTimer t(*c, "residual");
        if ((e = launch_residual(a, (int)c->cl.size(), c->prm.precision != OSV_FP64, c->stream)) != cudaSuccess)
            return c->cuda_fail(e, "residual");
    }
    if (cluster_status) {
        if ((e = cudaMemcpyAsync(cluster_status, c->iters, c->cl.size() * sizeof(int), cudaMemcpyDeviceToDevice,
                                 c->stream)) != cudaSuccess)
            return c->cuda_fail(e, "status copy");
    }
    c->solved = true;
    c->combined = false;
    if (n_iter_out) {
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return c->cuda_fail(e, "residual");
        osv_status st = device_error(c);
        if (st != OSV_OK) return st;
        std::vector<int> it(c->cl.size());
        if ((e = cudaMemcpy(it.data(), c->iters, it.size() * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return c->cuda_fail(e, "iters");
        int mx = 0;
        bool nc = false;
        for (int v : it) {
            if (v < 0) nc = true;
            mx = std::max(mx, v);
        }
        *n_iter_out = nc ? c->prm.max_iter : mx;
        if (nc) return c->fail(OSV_ERR_NOCONV, "some clusters did not converge");
    }
    return OSV_OK;
}

osv_status mbe3_combine(osv_ctx *c) {
    if (!c) return OSV_ERR_INVALID;
    if (!c->solved) return c->fail(OSV_ERR_INVALID, "cluster_residual_solve must precede mbe3_combine");
    cudaSetDevice(c->device);
    StageTimer t(*c, "combine");
    cudaError_t e = launch_combine(c->pinfo.d, (int)c->pairs.size(), c->comb_ptr.d, c->comb_src.d, c->comb_w.d,
                                   c->Tslot, c->Tc, c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "combine");
    c->combined = true;
    return OSV_OK;
}

namespace {

// Posterior plan: for every stored pair p = (i, j), the LMOs k of the clusters that hold both i and j, and the terms
// of Eq. 4 over them (the same coupling blocks as the cluster solves, which hold every such k with i and j).
osv_status build_posterior_plan(osv_ctx *c) {
    const int np_ = (int)c->pairs.size();
    std::vector<std::vector<int>> ks(np_);
    for (const auto &m : c->cl)
        for (size_t a = 0; a < m.size(); ++a)
            for (size_t b = a; b < m.size(); ++b) {
                auto &v = ks[c->pid(m[a], m[b])];
                v.insert(v.end(), m.begin(), m.end());
            }
    c->post_slots.h.clear();
    c->post_cl.h.clear();
    c->post_terms.h.clear();
    for (int p = 0; p < np_; ++p) {
        auto &v = ks[p];
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        const PairInfo &P = c->pinfo.h[p];
        Slot S{};
        S.pair = p;
        S.cluster = p;
        S.t_off = P.off;
        S.mult = P.i == P.j ? 1 : 2;
        c->post_slots.h.push_back(S);
        ClusterInfo C{};
        C.slot0 = p;
        C.slot1 = p + 1;
        C.term0 = (int)c->post_terms.h.size();
        C.weight = 1;
        C.size = (int)v.size();
        auto add = [&](int x, int y, int fx, int fy) -> bool {
            const int q = c->pid(x, y);
            if (q < 0) return false;
            const long long key = (long long)std::min(p, q) * (long long)np_ + std::max(p, q);
            auto it = c->coupling_id.find(key);
            if (it == c->coupling_id.end()) return false;
            Term T{};
            T.dst = p;
            T.src = q;
            T.fx = fx;
            T.fy = fy;
            T.t_trans = x > y ? 1 : 0;
            T.s_trans = p > q ? 1 : 0;
            T.coupling = it->second;
            T.sblk = c->coup_off[it->second];
            c->post_terms.h.push_back(T);
            return true;
        };
        for (int k : v) {
            if (k != P.j && !add(P.i, k, k, P.j)) return c->fail(OSV_ERR_INVALID, "posterior: missing coupling block");
            if (k != P.i && !add(k, P.j, P.i, k)) return c->fail(OSV_ERR_INVALID, "posterior: missing coupling block");
        }
        C.term1 = (int)c->post_terms.h.size();
        c->post_cl.h.push_back(C);
    }
    cudaError_t e;
    if ((e = c->upload(c->post_slots)) != cudaSuccess || (e = c->upload(c->post_cl)) != cudaSuccess ||
        (e = c->upload(c->post_terms)) != cudaSuccess || (e = c->dalloc(c->post_R1, c->pair_mat)) != cudaSuccess ||
        (e = c->dalloc(c->post_T2, c->pair_mat)) != cudaSuccess || (e = c->dalloc(c->post_R2, c->pair_mat)) != cudaSuccess ||
        (e = c->dalloc(c->post_rn, 2LL * np_)) != cudaSuccess || (e = c->dalloc(c->post_E, 2LL * np_)) != cudaSuccess ||
        (e = c->dalloc(c->post_G1, (long long)np_ * c->gstride)) != cudaSuccess)
        return c->cuda_fail(e, "posterior plan");
    c->post_built = true;
    return OSV_OK;
}

}  // namespace

osv_status posterior_correction(osv_ctx *c, double *E_global, double *E_corrected, double *dR_max) {
    if (!c || !E_global || !E_corrected) return c ? c->fail(OSV_ERR_INVALID, "NULL output") : OSV_ERR_INVALID;
    if (!c->combined) return c->fail(OSV_ERR_INVALID, "mbe3_combine must precede posterior_correction");
    cudaSetDevice(c->device);
    osv_status st;
    if (!c->post_built && (st = build_posterior_plan(c)) != OSV_OK) return st;
    const int np_ = (int)c->pairs.size();
    SolveArgs a{};
    a.clusters = c->post_cl.d;
    a.slots = c->post_slots.d;
    a.terms = c->post_terms.d;
    a.pairs = c->pinfo.d;
    a.rdim = c->rdim;
    a.e = c->pe;
    a.Kt = c->Kt;
    a.sblk = c->Stil;
    a.focc = c->focc;
    a.n_occ = c->n_occ;
    a.G1 = c->post_G1;
    a.gstride = c->gstride;
    a.np_max = 2 * c->nmax;
    cudaError_t e;
    {
        StageTimer t(*c, "posterior");
        e = launch_posterior(a, np_, c->Tc, c->post_R1, c->post_T2, c->post_R2, c->post_rn, c->post_E,
                             c->post_E + np_, c->prm.precision != OSV_FP64, c->stream);
    }
    if (e != cudaSuccess) return c->cuda_fail(e, "posterior");
    std::vector<double> rn(np_), E(2LL * np_);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess ||
        (e = cudaMemcpy(rn.data(), c->post_rn, np_ * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(E.data(), c->post_E, 2LL * np_ * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return c->cuda_fail(e, "posterior copy");
    double e1 = 0.0, e2 = 0.0, r = 0.0;
    for (int p = 0; p < np_; ++p) {
        e1 += E[p];
        e2 += E[np_ + p];
        r = std::max(r, rn[p]);
    }
    *E_global = e1;
    *E_corrected = e2;
    if (dR_max) *dR_max = r;
    if (!std::isfinite(e1) || !std::isfinite(e2)) return c->fail(OSV_ERR_NUMERIC, "posterior energy is not finite");
    return OSV_OK;
}

osv_status weak_pairs_energy(osv_ctx *c, const double *s2b, double l2b, double l_discard, double *E_weak,
                             int *n_weak) {
    if (!c || !E_weak) return c ? c->fail(OSV_ERR_INVALID, "E_weak is NULL") : OSV_ERR_INVALID;
    if (!s2b || !std::isfinite(l2b) || !std::isfinite(l_discard))
        return c->fail(OSV_ERR_INVALID, "s2b must be non-NULL and l2b, l_discard finite");
    if (!c->solved) return c->fail(OSV_ERR_INVALID, "cluster_residual_solve must precede weak_pairs_energy");
    const int n = c->n_occ, nm = c->nmax, nv = c->n_vir;
    *E_weak = 0.0;
    if (n_weak) *n_weak = 0;
    if (c->prm.mbe_order < 2 || c->prm.mbe_order > 3) return OSV_OK;   // no weak 2b clusters below MBE(2)
    // weak pairs: l_discard <= s2b_ij <= l2b (i < j), not a pair of a selected cluster
    std::vector<std::pair<int, int>> wl;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const double x = s2b[(size_t)i * n + j];
            if (!std::isfinite(x)) return c->fail(OSV_ERR_INVALID, "non-finite s2b entry");
            if (x >= l_discard && x <= l2b && c->pid(i, j) < 0) wl.push_back({i, j});
        }
    const int nw = (int)wl.size();
    if (n_weak) *n_weak = nw;
    if (nw == 0) return OSV_OK;
    cudaSetDevice(c->device);
    const bool full = full_domains(c);
    const long long nn = (long long)nm * nm;
    // device memory of this call: the cross half transforms Q_j B_i and Q_i B_j, the blocks and the workspaces
    std::vector<long long> yoff(nw + 1, 0);
    for (int w = 0; w < nw; ++w) yoff[w + 1] = yoff[w] + (long long)nm * (c->a_of(wl[w].first) + c->a_of(wl[w].second));
    std::vector<int> kmap;
    std::vector<std::pair<size_t, int>> kref(nw);
    if (!full) {
        std::vector<int> pi, pj;
        for (int w = 0; w < nw; ++w) {
            common_domain(c, wl[w].first, wl[w].second, pi, pj);
            kref[w] = {kmap.size(), (int)pi.size()};
            kmap.insert(kmap.end(), pi.begin(), pi.end());
            kmap.insert(kmap.end(), pj.begin(), pj.end());
        }
    }
    double *Y = nullptr, *blk = nullptr, *work = nullptr, *E = nullptr;
    int *dmap = nullptr;
    WeakPair *dwp = nullptr;
    GemmBatch gy, gk, gsf;
    osv::TcTiles oy, ok;
    auto cleanup = [&]() {
        for (void *p : {(void *)Y, (void *)blk, (void *)work, (void *)E, (void *)dmap, (void *)dwp})
            if (p) cudaFree(p);
        gemm_batch_free(gy);
        gemm_batch_free(gk);
        gemm_batch_free(gsf);
        osv::tc_tiles_free(oy);
        osv::tc_tiles_free(ok);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&Y, std::max<long long>(yoff[nw], 1) * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&blk, 4 * nw * nn * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&work, 7 * nw * nn * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&E, nw * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&dmap, std::max<size_t>(kmap.size(), 1) * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&dwp, nw * sizeof(WeakPair))) != cudaSuccess) {
        cleanup();
        return c->cuda_fail(e, "weak pairs");
    }
    if (!kmap.empty() && (e = cudaMemcpy(dmap, kmap.data(), kmap.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) {
        cleanup();
        return c->cuda_fail(e, "weak pairs");
    }
    std::vector<WeakPair> h(nw);
    for (int w = 0; w < nw; ++w) {
        const int i = wl[w].first, j = wl[w].second;
        const long long ai = c->a_of(i), aj = c->a_of(j);
        double *Yij = Y + yoff[w], *Yji = Yij + (long long)nm * ai;   // Q_j B_i (nm x a_i), Q_i B_j (nm x a_j)
        const double *Qi = c->Q + (long long)i * nm * nv, *Qj = c->Q + (long long)j * nm * nv;
        gy.add(gemm(nm, (int)ai, nv, Qj, nv, 0, c->B64 + c->b_off(i), ai, 0, Yij, ai));
        gy.add(gemm(nm, (int)aj, nv, Qi, nv, 0, c->B64 + c->b_off(j), aj, 0, Yji, aj));
        double *Kur = blk + 4 * w * nn, *Kll = Kur + nn, *S = Kll + nn, *F = S + nn;
        const double *Xi = c->W + c->w_off[i] + (long long)c->slot_of(i, i) * nm * ai;   // Q_i B_i
        const double *Xj = c->W + c->w_off[j] + (long long)c->slot_of(j, j) * nm * aj;   // Q_j B_j
        GemmDesc g1 = gemm(nm, nm, full ? c->n_aux : 0, Xi, ai, 0, Xj, aj, 1, Kur, nm);
        GemmDesc g2 = gemm(nm, nm, full ? c->n_aux : 0, Yij, ai, 0, Yji, aj, 1, Kll, nm);
        if (!full) {
            g1.K = g2.K = kref[w].second;
            g1.k_idx_a = g2.k_idx_a = dmap + kref[w].first;
            g1.k_idx_b = g2.k_idx_b = dmap + kref[w].first + kref[w].second;
        }
        gk.add(g1);
        gk.add(g2);
        gsf.add(gemm(nm, nm, nv, Qi, nv, 0, Qj, nv, 1, S, nm));
        gsf.add(gemm(nm, nm, nv, Qi, nv, 0, c->Qe + (long long)j * nm * nv, nv, 1, F, nm));
        const PairInfo &Pi = c->pinfo.h[c->pid(i, i)], &Pj = c->pinfo.h[c->pid(j, j)];
        WeakPair &W = h[w];
        W.i = i;
        W.j = j;
        W.Kur = Kur;
        W.Kll = Kll;
        W.S = S;
        W.F = F;
        W.Vi = c->V + Pi.off;
        W.Vj = c->V + Pj.off;
        W.ei = c->pe + Pi.e_off;
        W.ej = c->pe + Pj.e_off;
        W.ri = c->rdim + c->pid(i, i);
        W.rj = c->rdim + c->pid(j, j);
        W.Ti = c->Tslot + c->slots.h[c->cinfo.h[i].slot0].t_off;   // the 1b cluster {i} is cluster i
        W.Tj = c->Tslot + c->slots.h[c->cinfo.h[j].slot0].t_off;
        W.work = work + 7 * w * nn;
    }
    const bool mixed = c->prm.precision == OSV_MIXED_BF16X4;
    e = cudaMemcpy(dwp, h.data(), nw * sizeof(WeakPair), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = gemm_batch_upload(gy);
    if (e == cudaSuccess) e = gemm_batch_upload(gk);
    if (e == cudaSuccess) e = gemm_batch_upload(gsf);
    if (e == cudaSuccess && mixed) {
        if ((e = bf16x4_batch_prepare(gy, oy)) == cudaSuccess && (e = bf16x4_batch_prepare(gk, ok)) == cudaSuccess)
            e = c->oz_reserve((size_t)std::max(oy.scratch_bytes, ok.scratch_bytes));
    }
    if (e == cudaSuccess) {
        StageTimer t(*c, "weak_pairs");
        if ((e = c->run_dense(gy, oy)) == cudaSuccess && (e = c->run_dense(gk, ok)) == cudaSuccess &&
            (e = c->run_small(gsf)) == cudaSuccess)
            e = launch_weak_pairs(dwp, nw, nm, c->focc, c->n_occ, E, c->stream);
    }
    std::vector<double> Eh(nw);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemcpy(Eh.data(), E, nw * sizeof(double), cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) return c->cuda_fail(e, "weak pairs");
    osv_status st = device_error(c);
    if (st != OSV_OK) return st;
    double sum = 0.0;
    for (double x : Eh) sum += x;
    *E_weak = sum;
    if (!std::isfinite(sum)) return c->fail(OSV_ERR_NUMERIC, "weak-pair energy is not finite");
    return OSV_OK;
}

osv_status osv_pair_amplitudes(osv_ctx *c, int i, int j, double *t_out) {
    if (!c || !t_out) return OSV_ERR_INVALID;
    if (!c->combined) return c->fail(OSV_ERR_INVALID, "mbe3_combine must precede osv_pair_amplitudes");
    if (i < 0 || j < 0 || i >= c->n_occ || j >= c->n_occ) return c->fail(OSV_ERR_INVALID, "LMO index out of range");
    const int p = c->pid(i, j);
    if (p < 0) return c->fail(OSV_ERR_INVALID, "the pair belongs to no selected cluster");
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "sync");
    const PairInfo &P = c->pinfo.h[p];
    const int nv = c->n_vir, nm = c->nmax, np = P.np;
    const int dom[2] = {P.i, P.j};
    const int nd = P.i == P.j ? 1 : 2;
    // domain rows (OSVs of the pair's LMOs; rows beyond n_k are zero), basis V (columns) and collective T~
    std::vector<double> Pr((size_t)np * nv), V((size_t)np * np), T((size_t)np * np);
    for (int x = 0; x < nd; ++x)
        if ((e = cudaMemcpy(Pr.data() + (size_t)x * nm * nv, c->Q + (long long)dom[x] * nm * nv,
                            (size_t)nm * nv * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return c->cuda_fail(e, "copy Q");
    if ((e = cudaMemcpy(V.data(), c->V + P.off, V.size() * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(T.data(), c->Tc + P.off, T.size() * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return c->cuda_fail(e, "copy pair");
    // U = V^T P (np x nv): the orthonormal pair basis in the virtual space; t = U^T T~ U
    std::vector<double> U((size_t)np * nv, 0.0), TU((size_t)np * nv, 0.0);
    for (int a = 0; a < np; ++a)
        for (int r = 0; r < np; ++r) {
            const double v = V[(size_t)r * np + a];
            if (v == 0.0) continue;
            for (int x = 0; x < nv; ++x) U[(size_t)a * nv + x] += v * Pr[(size_t)r * nv + x];
        }
    for (int a = 0; a < np; ++a)
        for (int b = 0; b < np; ++b) {
            const double v = T[(size_t)a * np + b];
            if (v == 0.0) continue;
            for (int x = 0; x < nv; ++x) TU[(size_t)a * nv + x] += v * U[(size_t)b * nv + x];
        }
    const bool swap = i > j;   // stored pair (j, i): t_ij = t_ji^T
    for (int x = 0; x < nv; ++x)
        for (int y = 0; y < nv; ++y) {
            double acc = 0.0;
            for (int a = 0; a < np; ++a) acc += U[(size_t)a * nv + x] * TU[(size_t)a * nv + y];
            t_out[swap ? (size_t)y * nv + x : (size_t)x * nv + y] = acc;
        }
    return OSV_OK;
}

osv_status energy(osv_ctx *c, double *E_out, double *E_linear_out) {
    if (!c || !E_out) return c ? c->fail(OSV_ERR_INVALID, "E_out is NULL") : OSV_ERR_INVALID;
    if (!c->solved) return c->fail(OSV_ERR_INVALID, "cluster_residual_solve must precede energy");
    cudaSetDevice(c->device);
    cudaError_t e;
    {
        StageTimer t(*c, "energy");
        e = launch_energy(c->pinfo.d, c->rdim, c->Kt, c->Tc, (int)c->pairs.size(), c->lin, c->Ecl,
                                  c->cinfo.d, (int)c->cl.size(), c->Eout, c->stream);
    }
    if (e != cudaSuccess) return c->cuda_fail(e, "energy");
    double h[2];
    if ((e = cudaMemcpyAsync(h, c->Eout, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
        return c->cuda_fail(e, "energy copy");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return c->cuda_fail(e, "energy");
    osv_status st = device_error(c);
    if (st != OSV_OK) return st;
    *E_out = h[0];
    if (E_linear_out) *E_linear_out = h[1];
    if (!std::isfinite(h[0])) return c->fail(OSV_ERR_NUMERIC, "energy is not finite");
    // clusters that hit max_iter carry iters = -1 (whether or not cluster_residual_solve was asked to check)
    std::vector<int> it(c->cl.size());
    if ((e = cudaMemcpy(it.data(), c->iters, it.size() * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return c->cuda_fail(e, "iters");
    const long long bad = std::count_if(it.begin(), it.end(), [](int v) { return v < 0; });
    if (bad) return c->fail(OSV_ERR_NOCONV, std::to_string(bad) + " clusters did not converge within max_iter");
    return OSV_OK;
}

osv_status osv_cluster_count(osv_ctx *c, int *n_clusters) {
    if (!c || !n_clusters) return OSV_ERR_INVALID;
    *n_clusters = (int)c->cl.size();
    return OSV_OK;
}

osv_status osv_cluster_info(osv_ctx *c, int32_t *members, int32_t *weight, double *en, int32_t *iters) {
    if (!c) return OSV_ERR_INVALID;
    const size_t nc = c->cl.size();
    if (members)
        for (size_t q = 0; q < nc; ++q)
            for (int t = 0; t < 3; ++t) members[3 * q + t] = t < (int)c->cl[q].size() ? c->cl[q][t] : -1;
    if (weight)
        for (size_t q = 0; q < nc; ++q) weight[q] = c->cl_w[q];
    if ((en || iters) && !c->solved) return c->fail(OSV_ERR_INVALID, "no solved clusters");
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "sync");
    if (en && (e = cudaMemcpy(en, c->Ecl, nc * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return c->cuda_fail(e, "copy");
    if (iters && (e = cudaMemcpy(iters, c->iters, nc * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return c->cuda_fail(e, "copy");
    return OSV_OK;
}

osv_status osv_eigenvalues(osv_ctx *c, int k, double *w_out) {
    if (!c || !w_out) return OSV_ERR_INVALID;
    if (!c->built || k < 0 || k >= c->n_occ) return c->fail(OSV_ERR_INVALID, "bad LMO index or not built");
    cudaSetDevice(c->device);
    // the build computes only the n_max leading eigenvalues: the full spectrum is formed here, on demand
    const int nv = c->n_vir, nm = c->nmax;
    cudaError_t e;
    if (!c->osv_mixed) {
        if ((e = osv_tri_eigvals<double>(c->tri_osv.d, c->n_occ, nv, nv, c->stream)) != cudaSuccess)
            return c->cuda_fail(e, "eigenvalues");
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return c->cuda_fail(e, "sync");
        if ((e = cudaMemcpy(w_out, c->omega + (long long)k * nv, nv * sizeof(double), cudaMemcpyDeviceToHost)) !=
            cudaSuccess)
            return c->cuda_fail(e, "copy");
        return OSV_OK;
    }
    // mixed: the leading n_max refined in FP64, the rest from the FP32 tridiagonal
    if ((e = osv_tri_eigvals<float>(c->refine.tri_d, c->n_occ, nv, nv, c->stream)) != cudaSuccess)
        return c->cuda_fail(e, "eigenvalues");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return c->cuda_fail(e, "sync");
    std::vector<float> w32(nv);
    if ((e = cudaMemcpy(w32.data(), c->refine.w32 + (long long)k * nv, nv * sizeof(float), cudaMemcpyDeviceToHost)) !=
            cudaSuccess ||
        (e = cudaMemcpy(w_out, c->refine.lam + (long long)k * nm, nm * sizeof(double), cudaMemcpyDeviceToHost)) !=
            cudaSuccess)
        return c->cuda_fail(e, "copy");
    for (int i = nm; i < nv; ++i) w_out[i] = w32[i];
    return OSV_OK;
}

osv_status gradient_backward(osv_ctx *c, double dE_scale, void *dE_dB, double *dE_dFocc) {
    if (!c) return OSV_ERR_INVALID;
    if (!c->solved) return c->fail(OSV_ERR_INVALID, "cluster_residual_solve must precede gradient_backward");
    cudaSetDevice(c->device);
    std::string msg;
    cudaError_t e = c->adj.run(*c, dE_scale, dE_dB, dE_dFocc, msg);
    if (e != cudaSuccess) return c->cuda_fail(e, msg.c_str());
    // a bounded wait that gave up, or a non-finite value, leaves its mark in the device error word
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return c->cuda_fail(e, "gradient_backward");
    return device_error(c);
}

}  // extern "C"

namespace {

// Pinned host block the recorded step copies its results into: E and E_linear, the error word, per-cluster
// iteration counts.
constexpr size_t kPinE = 0, kPinErr = 16, kPinIters = 24;

// Enqueue one step on c->stream with the plan already in place (nothing allocates, uploads or synchronises):
// osv_build's device steps, the cluster solves, the MBE(3) combination, the energy and, when grad, the adjoint into
// zeroed dB/dF; then the results are copied into the pinned block.
osv_status record_step(osv_ctx *c, bool grad, double scale, void *dB, double *dF, size_t nb, size_t nf) {
    osv_status st;
    cudaError_t e;
    if ((st = run_osv_build(c)) != OSV_OK) return st;
    if ((st = cluster_residual_solve(c, nullptr, nullptr)) != OSV_OK) return st;
    if ((st = mbe3_combine(c)) != OSV_OK) return st;
    {
        StageTimer t(*c, "energy");
        e = launch_energy(c->pinfo.d, c->rdim, c->Kt, c->Tc, (int)c->pairs.size(), c->lin, c->Ecl, c->cinfo.d,
                          (int)c->cl.size(), c->Eout, c->stream);
    }
    if (e != cudaSuccess) return c->cuda_fail(e, "energy");
    if (grad) {
        if (dB && (e = cudaMemsetAsync(dB, 0, nb, c->stream)) != cudaSuccess) return c->cuda_fail(e, "memset dE_dB");
        if (dF && (e = cudaMemsetAsync(dF, 0, nf, c->stream)) != cudaSuccess) return c->cuda_fail(e, "memset dE_dF");
        std::string msg;
        if ((e = c->adj.run(*c, scale, dB, dF, msg)) != cudaSuccess) return c->cuda_fail(e, msg.c_str());
    }
    char *h = (char *)c->gpin;
    if ((e = cudaMemcpyAsync(h + kPinE, c->Eout, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(h + kPinErr, c->derr, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h + kPinIters, c->iters, c->cl.size() * sizeof(int), cudaMemcpyDeviceToHost,
                             c->stream)) != cudaSuccess)
        return c->cuda_fail(e, "result copies");
    return OSV_OK;
}

}  // namespace

extern "C" {

osv_status osv_graph_capture(osv_ctx *c, const osv_problem *pb, const osv_params *prm, double dE_scale,
                             void *dE_dB, double *dE_dFocc) {
    if (!c) return OSV_ERR_INVALID;
    cudaSetDevice(c->device);
    c->graph_release();
    const bool grad = dE_dB || dE_dFocc;
    osv_status st;
    cudaError_t e;
    // one eager step: plans (and tunes) a new shape, checks the inputs and leaves this step's results in place
    if ((st = osv_build(c, pb, prm, nullptr)) != OSV_OK || (st = cluster_residual_solve(c, nullptr, nullptr)) != OSV_OK ||
        (st = mbe3_combine(c)) != OSV_OK)
        return st;
    double E0, El0;
    if ((st = energy(c, &E0, &El0)) != OSV_OK) return st;
    const size_t nb = (size_t)c->aux_ptr[c->n_occ] * c->n_vir * (c->B_dtype == 0 ? sizeof(double) : sizeof(float));
    const size_t nf = (size_t)c->n_occ * c->n_occ * sizeof(double);
    if (grad) {
        if (dE_dB && (e = cudaMemsetAsync(dE_dB, 0, nb, c->stream)) != cudaSuccess) return c->cuda_fail(e, "memset");
        if (dE_dFocc && (e = cudaMemsetAsync(dE_dFocc, 0, nf, c->stream)) != cudaSuccess)
            return c->cuda_fail(e, "memset");
        if ((st = gradient_backward(c, dE_scale, dE_dB, dE_dFocc)) != OSV_OK) return st;
    }
    if ((e = cudaMallocHost(&c->gpin, kPinIters + std::max<size_t>(c->cl.size(), 1) * sizeof(int))) != cudaSuccess) {
        c->gpin = nullptr;
        return c->cuda_fail(e, "pinned result block");
    }
    if (!c->gstream && (e = cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking)) != cudaSuccess) {
        c->gstream = nullptr;
        return c->cuda_fail(e, "capture stream");
    }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return c->cuda_fail(e, "graph capture");
    // record the same step on the capture stream; the launches it counts are recorded, not run
    cudaStream_t user = c->stream;
    c->capturing = true;
    c->stream = c->gstream;
    const long long l0 = g_launches.load();
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
        st = c->cuda_fail(e, "begin capture");
    } else {
        st = record_step(c, grad, dE_scale, dE_dB, dE_dFocc, nb, nf);
        const cudaError_t e2 = cudaStreamEndCapture(c->gstream, &g);
        if (st == OSV_OK && e2 != cudaSuccess) st = c->cuda_fail(e2, "end capture");
    }
    g_launches.fetch_sub(g_launches.load() - l0);
    c->stream = user;
    c->capturing = false;
    if (st == OSV_OK) {
        size_t nn = 0;
        if ((e = cudaGraphGetNodes(g, nullptr, &nn)) == cudaSuccess) {
            std::vector<cudaGraphNode_t> nodes(nn);
            if ((e = cudaGraphGetNodes(g, nodes.data(), &nn)) == cudaSuccess)
                for (cudaGraphNode_t x : nodes) {
                    cudaGraphNodeType t;
                    if ((e = cudaGraphNodeGetType(x, &t)) != cudaSuccess) break;
                    if (t == cudaGraphNodeTypeKernel) ++c->graph_kernels;
                }
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, g, 0);
        if (e != cudaSuccess) {
            c->gexec = nullptr;
            st = c->cuda_fail(e, "graph instantiate");
        }
    }
    if (g) cudaGraphDestroy(g);
    if (st != OSV_OK) {
        c->graph_release();
        return st;
    }
    c->graph_grad = grad;
    return OSV_OK;
}

osv_status osv_graph_launch(osv_ctx *c, double *E_out, double *E_linear_out) {
    if (!c) return OSV_ERR_INVALID;
    if (!c->gexec) return c->fail(OSV_ERR_INVALID, "no recorded step: osv_graph_capture (again after a re-plan)");
    cudaSetDevice(c->device);
    cudaError_t e = cudaGraphLaunch(c->gexec, c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "graph launch");
    count_launch(c->graph_kernels);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return c->cuda_fail(e, "graph launch");
    c->solved = c->combined = true;
    if (c->prof)
        for (auto &ev : c->gev) {
            float t = 0.f;
            if ((e = cudaEventElapsedTime(&t, ev.a, ev.b)) != cudaSuccess) return c->cuda_fail(e, "stage event time");
            c->gtimes.push_back({ev.name, t});
        }
    const char *h = (const char *)c->gpin;
    osv_status st = error_word_status(c, *(const int *)(h + kPinErr));
    if (st != OSV_OK) return st;
    double E[2];
    memcpy(E, h + kPinE, sizeof(E));
    if (E_out) *E_out = E[0];
    if (E_linear_out) *E_linear_out = E[1];
    if (!std::isfinite(E[0])) return c->fail(OSV_ERR_NUMERIC, "energy is not finite");
    const int *it = (const int *)(h + kPinIters);
    const long long bad = std::count_if(it, it + c->cl.size(), [](int v) { return v < 0; });
    if (bad) return c->fail(OSV_ERR_NOCONV, std::to_string(bad) + " clusters did not converge within max_iter");
    return OSV_OK;
}

osv_status osv_graph_kernels(osv_ctx *c, long long *count) {
    if (!c || !count) return OSV_ERR_INVALID;
    *count = c->gexec ? c->graph_kernels : 0;
    return OSV_OK;
}

osv_status osv_autotune(osv_ctx *c, int on) {
    if (!c) return OSV_ERR_INVALID;
    c->autotune = on != 0;
    return OSV_OK;
}

osv_status osv_autotune_report(osv_ctx *c, char *buf, int len, int *needed) {
    if (!c) return OSV_ERR_INVALID;
    const int n = (int)c->tune_report.size() + 1;
    if (needed) *needed = n;
    if (buf && len > 0) {
        strncpy(buf, c->tune_report.c_str(), (size_t)len - 1);
        buf[len - 1] = 0;
    }
    return OSV_OK;
}

osv_status osv_set_tridiag_variant(osv_ctx *c, int variant) {
    if (!c) return OSV_ERR_INVALID;
    if (variant < -1 || variant >= kTriVariants) return c->fail(OSV_ERR_INVALID, "tridiagonalisation variant out of range");
    c->tri_force = variant;
    return OSV_OK;
}

osv_status osv_set_wait_budget(osv_ctx *c, long long cycles) {
    if (!c) return OSV_ERR_INVALID;
    c->wait_budget = cycles > 0 ? cycles : 0;
    return OSV_OK;
}

osv_status osv_kernel_launches(long long *count) {
    if (!count) return OSV_ERR_INVALID;
    *count = g_launches.load();
    return OSV_OK;
}

osv_status osv_profile_enable(osv_ctx *c, int on) {
    if (!c) return OSV_ERR_INVALID;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto &e : c->pev) {
        c->pool.push_back(e.a);
        c->pool.push_back(e.b);
    }
    c->pev.clear();
    c->gtimes.clear();
    c->prof = on != 0;
    return OSV_OK;
}

osv_status osv_profile_read(osv_ctx *c, int max_stages, char *names, double *ms, int *calls, int *n_stages) {
    if (!c || !n_stages || max_stages < 0) return OSV_ERR_INVALID;
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "profile sync");
    std::vector<std::string> order;
    std::map<std::string, std::pair<double, int>> acc;
    for (auto &ev : c->pev) {
        float t = 0.f;
        if ((e = cudaEventElapsedTime(&t, ev.a, ev.b)) != cudaSuccess) return c->cuda_fail(e, "event time");
        if (!acc.count(ev.name)) order.push_back(ev.name);
        acc[ev.name].first += t;
        acc[ev.name].second += 1;
    }
    for (auto &gt : c->gtimes) {
        if (!acc.count(gt.first)) order.push_back(gt.first);
        acc[gt.first].first += gt.second;
        acc[gt.first].second += 1;
    }
    *n_stages = (int)order.size();
    for (int q = 0; q < (int)order.size() && q < max_stages; ++q) {
        if (names) {
            strncpy(names + 32 * q, order[q].c_str(), 31);
            names[32 * q + 31] = 0;
        }
        if (ms) ms[q] = acc[order[q]].first;
        if (calls) calls[q] = acc[order[q]].second;
    }
    return OSV_OK;
}

osv_status osv_residual_flops(osv_ctx *c, double *flops) {
    if (!c || !flops) return OSV_ERR_INVALID;
    if (!c->solved) return c->fail(OSV_ERR_INVALID, "no solved clusters");
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "sync");
    std::vector<int> r(c->pairs.size()), it(c->cl.size());
    if ((e = cudaMemcpy(r.data(), c->rdim, r.size() * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(it.data(), c->iters, it.size() * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return c->cuda_fail(e, "copy");
    double total = 0.0;
    for (size_t q = 0; q < c->cl.size(); ++q) {
        const int evals = (it[q] < 0 ? c->prm.max_iter : it[q]) + 1;
        double per = 0.0;
        for (int t = c->cinfo.h[q].term0; t < c->cinfo.h[q].term1; ++t) {
            const double rp = r[c->slots.h[c->terms.h[t].dst].pair], rq = r[c->slots.h[c->terms.h[t].src].pair];
            per += 2.0 * (rp * rq * rq + rp * rp * rq);
        }
        total += per * evals;
    }
    *flops = total;
    return OSV_OK;
}

osv_status osv_adjoint_flops(osv_ctx *c, double *flops) {
    if (!c || !flops) return OSV_ERR_INVALID;
    if (!c->solved) return c->fail(OSV_ERR_INVALID, "no solved clusters");
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "sync");
    std::vector<int> r(c->pairs.size());
    if ((e = cudaMemcpy(r.data(), c->rdim, r.size() * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return c->cuda_fail(e, "copy");
    double total = 0.0;
    for (size_t q = 0; q < c->cl.size(); ++q) {
        const ClusterInfo &C = c->cinfo.h[q];
        if (C.weight == 0) continue;
        for (int s = C.slot0; s < C.slot1; ++s) {
            const double rp = r[c->slots.h[s].pair];
            total += 8.0 * rp * rp * rp;
        }
        for (int t = C.term0; t < C.term1; ++t) {
            const double rp = r[c->slots.h[c->terms.h[t].dst].pair], rq = r[c->slots.h[c->terms.h[t].src].pair];
            total += 4.0 * rp * rp * rq + 4.0 * rp * rq * rq;
        }
    }
    *flops = total;
    return OSV_OK;
}

osv_status osv_residual_work(osv_ctx *c, double *flops32, double *flops64) {
    if (!c || !flops32 || !flops64) return OSV_ERR_INVALID;
    if (!c->solved) return c->fail(OSV_ERR_INVALID, "no solved clusters");
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "sync");
    std::vector<int> r(c->pairs.size()), e32(c->cl.size()), e64(c->cl.size());
    if ((e = cudaMemcpy(r.data(), c->rdim, r.size() * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(e32.data(), c->evals32, e32.size() * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(e64.data(), c->evals64, e64.size() * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return c->cuda_fail(e, "copy");
    double f32 = 0.0, f64 = 0.0;
    for (size_t q = 0; q < c->cl.size(); ++q) {
        double per = 0.0;
        for (int t = c->cinfo.h[q].term0; t < c->cinfo.h[q].term1; ++t) {
            const double rp = r[c->slots.h[c->terms.h[t].dst].pair], rq = r[c->slots.h[c->terms.h[t].src].pair];
            per += 2.0 * (rp * rq * rq + rp * rp * rq);
        }
        f32 += per * (c->prm.precision != OSV_FP64 ? e32[q] : 0);
        f64 += per * e64[q];
    }
    *flops32 = f32;
    *flops64 = f64;
    return OSV_OK;
}

osv_status osv_solve_counts(osv_ctx *c, long long *updates32, long long *evals64, int *unconverged) {
    if (!c || !updates32 || !evals64 || !unconverged) return OSV_ERR_INVALID;
    if (!c->solved) return c->fail(OSV_ERR_INVALID, "no solved clusters");
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "sync");
    std::vector<int> it(c->cl.size()), ev(c->cl.size());
    if ((e = cudaMemcpy(it.data(), c->iters, it.size() * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(ev.data(), c->evals64, ev.size() * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return c->cuda_fail(e, "copy");
    long long u = 0, f = 0;
    int bad = 0;
    for (size_t q = 0; q < it.size(); ++q) {
        f += ev[q];
        if (it[q] < 0) ++bad;
        else if (c->prm.precision != OSV_FP64) u += it[q] - ev[q] + 1;   // iters = FP32 updates + FP64 evals - 1
    }
    *updates32 = u;
    *evals64 = f;
    *unconverged = bad;
    return OSV_OK;
}

osv_status osv_syev_batched(const double *A, int n, int batch, double *w, double *Zt, void *cuda_stream) {
    if (!A || !w || !Zt || n < 1 || n > 4096 || batch < 1) {
        g_noctx_err = "osv_syev_batched: bad argument";
        return OSV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const long long nn = (long long)n * n;
    double *work = nullptr, *zw = nullptr, *vec = nullptr;
    int *err = nullptr;
    auto cleanup = [&]() {
        if (work) cudaFree(work);
        if (zw) cudaFree(zw);
        if (vec) cudaFree(vec);
        if (err) cudaFree(err);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&work, batch * nn * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&zw, batch * nn * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&vec, 3LL * batch * n * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&err, sizeof(int))) != cudaSuccess) {
        cleanup();
        g_noctx_err = std::string("osv_syev_batched: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? OSV_ERR_OOM : OSV_ERR_CUDA;
    }
    std::vector<EighDesc> h(batch);
    for (int b = 0; b < batch; ++b) {
        EighDesc &D = h[b];
        D.A = work + b * nn;
        D.lda = n;
        D.n = n;
        D.w = w + (long long)b * n;
        D.Zt = Zt + b * nn;
        D.ldz = n;
        D.zwork = zw + b * nn;
        D.d = vec + 3LL * b * n;
        D.e = D.d + n;
        D.tau = D.e + n;
    }
    EighDesc *dd = nullptr;
    if ((e = cudaMalloc(&dd, batch * sizeof(EighDesc))) == cudaSuccess &&
        (e = cudaMemcpyAsync(dd, h.data(), batch * sizeof(EighDesc), cudaMemcpyHostToDevice, s)) == cudaSuccess &&
        (e = cudaMemcpyAsync(work, A, batch * nn * sizeof(double), cudaMemcpyDeviceToDevice, s)) == cudaSuccess &&
        (e = cudaMemsetAsync(err, 0, sizeof(int), s)) == cudaSuccess &&
        (e = eigh_batched(dd, batch, n, 0, err, s)) == cudaSuccess)
        e = cudaStreamSynchronize(s);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (dd) cudaFree(dd);
    cleanup();
    if (e != cudaSuccess) {
        g_noctx_err = std::string("osv_syev_batched: ") + cudaGetErrorString(e);
        return OSV_ERR_CUDA;
    }
    if (herr) {
        g_noctx_err = "osv_syev_batched: QL iteration cap reached";
        return OSV_ERR_TIMEOUT;
    }
    return OSV_OK;
}

}  // extern "C"
