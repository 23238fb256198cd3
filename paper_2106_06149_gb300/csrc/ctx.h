// Context of libosvmbe (shared by the C ABI in api.cu and the adjoint in adjoint.cu).
#pragma once
#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "../../include/osvmbe.h"
#include "adjoint.h"
#include "osv_eig.h"
#include "osv_refine.h"
#include "tc_gemm.h"

namespace osv {
struct ProfEvent {
    const char *name;
    cudaEvent_t a, b;
};
template <class T>
struct HostDev {
    std::vector<T> h;
    T *d = nullptr;
};
}  // namespace osv

struct osv_ctx {
    template <class T>
    using HostDev = osv::HostDev<T>;
    using GemmBatch = osv::GemmBatch;
    using PairInfo = osv::PairInfo;
    using Slot = osv::Slot;
    using Term = osv::Term;
    using ClusterInfo = osv::ClusterInfo;
    using BlockCopy = osv::BlockCopy;
    using EighDesc = osv::EighDesc;
    using GemmDesc = osv::GemmDesc;

    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;

    // problem and parameters
    osv_params prm{};
    int n_occ = 0, n_vir = 0, n_aux = 0, nmax = 0;
    std::vector<double> centres;
    std::vector<int64_t> aux_ptr;
    std::vector<int32_t> aux_idx;
    const double *focc = nullptr, *eps = nullptr;
    const void *B_in = nullptr;
    int B_dtype = 0;
    const double *B64 = nullptr;   // fp64 DF blocks (caller's buffer or the internal copy)

    // clusters (host)
    bool have_clusters = false, built = false, solved = false, combined = false;
    std::vector<std::vector<int>> cl;
    std::vector<int> cl_w;
    int ncl_order[3] = {0, 0, 0};

    // pairs / neighbours / couplings (host)
    std::vector<std::pair<int, int>> pairs;
    std::map<long long, int> pair_id;
    std::vector<std::vector<int>> nb;
    std::map<long long, int> coupling_id;
    std::vector<std::pair<int, int>> couplings;

    // device arrays
    std::vector<void *> allocs;
    double *Tkk = nullptr, *Awork = nullptr, *Zc = nullptr, *omega = nullptr, *dsc = nullptr, *esc = nullptr,
           *tausc = nullptr;
    int *nosv = nullptr, *derr = nullptr;
    double *B64own = nullptr;
    double *Q = nullptr, *Qe = nullptr, *sblk = nullptr, *fblk = nullptr, *W = nullptr;
    std::vector<long long> w_off;          // per LMO offset of W^{(i)} (doubles)
    double *Kp = nullptr, *Sp = nullptr, *Fp = nullptr, *X = nullptr, *Fx = nullptr, *V = nullptr, *Kt = nullptr,
           *ptmp = nullptr, *Tc = nullptr, *sw = nullptr, *pe = nullptr, *pz = nullptr, *pd = nullptr,
           *pee = nullptr, *ptau = nullptr;
    int *rdim = nullptr;
    long long pair_mat = 0, pair_vec = 0;  // totals
    double *Scp = nullptr, *Stil = nullptr, *ctmp = nullptr;
    long long coup_mat = 0;
    double *Tslot = nullptr, *Rslot = nullptr, *G1 = nullptr, *Ecl = nullptr, *lin = nullptr, *Eout = nullptr;
    // FP32 copies and work arrays of the mixed residual solve
    float *e32 = nullptr, *Kt32 = nullptr, *S32 = nullptr, *T32 = nullptr, *R32 = nullptr, *H32 = nullptr, *G1_32 = nullptr;
    int *evals64 = nullptr;
    int *evals32 = nullptr;
    int *iters = nullptr;
    int *work_next = nullptr;             // work counter of the persistent residual launch
    long long slot_mat = 0, gstride = 0;

    HostDev<PairInfo> pinfo;
    HostDev<Slot> slots;
    HostDev<Term> terms;
    HostDev<ClusterInfo> cinfo;
    HostDev<int> order;
    HostDev<int> comb_ptr, comb_w;
    HostDev<long long> comb_src;
    std::vector<long long> coup_off;       // per coupling offset (doubles) of its n_pa x n_pb blocks
    HostDev<BlockCopy> bc_pair, bc_coup;
    HostDev<EighDesc> eig_s, eig_f;
    HostDev<osv::TriDesc> tri_osv;         // OSV eigenproblems (FP64 tridiagonal route)
    double *Ytri = nullptr, *tri_work = nullptr;
    bool osv_mixed = false;                // mixed precisions: FP32 tridiagonal route + FP64 refinement
    osv::OsvRefine refine;
    HostDev<int> rows_w;                   // a_rows maps for the half transforms
    HostDev<int> kidx;                     // common-fitting-domain position lists
    GemmBatch gb_gram, gb_sf, gb_w, gb_k, gb_fx1, gb_fx2, gb_v, gb_kt1, gb_kt2, gb_c1, gb_c2;
    osv::TcTiles oz_gram, oz_w, oz_k;          // exact-slice BF16x4 tilings

    osv::AdjointPlan adj;
    // one-step posterior correction (built on first use after a solve): one pseudo-cluster per stored pair
    bool post_built = false;
    HostDev<Slot> post_slots;
    HostDev<ClusterInfo> post_cl;
    HostDev<Term> post_terms;
    double *post_R1 = nullptr, *post_T2 = nullptr, *post_R2 = nullptr, *post_rn = nullptr, *post_E = nullptr,
           *post_G1 = nullptr;
    long long wait_budget = 0;             // tensor-core main-loop wait budget in clock cycles (0 = default)
    // plan-time autotuner (mixed precision): launch shapes timed on the device, the fastest kept
    bool autotune = true;
    int tri_force = -1;                    // FP32 tridiagonalisation launch shape fixed by the caller (-1: tuned)
    std::string tune_report;               // JSON: per tuned item the rule's choice, the tuned choice, timings
    // one whole step recorded as a CUDA graph (osv_graph_capture / osv_graph_launch)
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;        // non-blocking stream the step is recorded on
    long long graph_kernels = 0;           // kernel nodes of the recorded step
    bool graph_grad = false;
    void *gpin = nullptr;                  // pinned host: E, E_linear, error word, per-cluster iterations
    bool capturing = false;                // recording: stage timers become event-record nodes of the graph
    std::vector<osv::ProfEvent> gev;       // the stage events recorded in the graph
    std::vector<std::pair<const char *, float>> gtimes;   // stage times of the replays run while profiling
    void graph_release() {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        for (auto &e : gev) {
            pool.push_back(e.a);
            pool.push_back(e.b);
        }
        gev.clear();
        if (gpin) cudaFreeHost(gpin);
        gpin = nullptr;
        graph_kernels = 0;
    }

    // per-stage CUDA-event profiling (osv_profile_enable / osv_profile_read)
    bool prof = false;
    std::vector<osv::ProfEvent> pev;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t take_event() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }

    osv_status fail(osv_status s, const std::string &m) {
        err = m;
        return s;
    }
    osv_status cuda_fail(cudaError_t e, const char *where) {
        err = std::string(where) + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? OSV_ERR_OOM : OSV_ERR_CUDA;
    }
    template <class T>
    cudaError_t dalloc(T *&p, size_t count) {
        p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e == cudaSuccess) allocs.push_back((void *)p);
        return e;
    }
    // dense DF contractions: FP64 CUDA cores or exact BF16 slices on the tcgen05 tensor cores
    cudaError_t run_dense(const GemmBatch &b, const osv::TcTiles &oz) {
        if (prm.precision == OSV_MIXED_BF16X4) return osv::bf16x4_batch_run(oz, oz_scratch, derr, wait_budget, stream);
        return osv::gemm_batch_run(b, stream);
    }
    // the small FP64-accurate GEMM batches (pair and refinement blocks): FP64 CUDA cores, or double-float on the
    // FP32 pipe in the mixed modes
    cudaError_t run_small(const GemmBatch &b) {
        if (prm.precision != OSV_FP64) return osv::gemm_batch_run_df(b, stream);
        return osv::gemm_batch_run(b, stream);
    }
    // slice images of the exact-slice GEMM batches (one buffer, grown to the largest batch)
    unsigned char *oz_scratch = nullptr;
    size_t oz_cap = 0;
    cudaError_t oz_reserve(size_t bytes) {
        if (bytes <= oz_cap) return cudaSuccess;
        if (oz_scratch) {
            if (stream) cudaStreamSynchronize(stream);
            cudaFree(oz_scratch);
            oz_scratch = nullptr;
            oz_cap = 0;
        }
        cudaError_t e = cudaMalloc(&oz_scratch, bytes);
        if (e == cudaSuccess) oz_cap = bytes;
        return e;
    }
    template <class T>
    cudaError_t upload(HostDev<T> &hd) {
        cudaError_t e = dalloc(hd.d, hd.h.size());
        if (e != cudaSuccess || hd.h.empty()) return e;
        return cudaMemcpy(hd.d, hd.h.data(), hd.h.size() * sizeof(T), cudaMemcpyHostToDevice);
    }
    void release() {
        for (void *p : allocs) cudaFree(p);
        allocs.clear();
        for (GemmBatch *g : {&gb_gram, &gb_sf, &gb_w, &gb_k, &gb_fx1, &gb_fx2, &gb_v, &gb_kt1, &gb_kt2, &gb_c1, &gb_c2}) {
            gemm_batch_free(*g);
            g->h.clear();
        }
        for (int x = 0; x < 2; ++x)
            for (GemmBatch *g : {&refine.gb_w[x], &refine.gb_gh[x], &refine.gb_rot[x], &refine.gb_fin[x]}) {
                gemm_batch_free(*g);
                g->h.clear();
            }
        refine = osv::OsvRefine{};
        if (oz_scratch) cudaFree(oz_scratch);
        oz_scratch = nullptr;
        oz_cap = 0;
        for (osv::TcTiles *t : {&oz_gram, &oz_w, &oz_k}) osv::tc_tiles_free(*t);
        adj.release();
        graph_release();
        built = solved = combined = post_built = false;
    }
    int pid(int i, int j) const {
        auto it = pair_id.find((long long)std::min(i, j) * n_occ + std::max(i, j));
        return it == pair_id.end() ? -1 : it->second;
    }
    int slot_of(int i, int m) const {   // position of m in nb(i)
        const auto &v = nb[i];
        return int(std::lower_bound(v.begin(), v.end(), m) - v.begin());
    }
    long long a_of(int i) const { return aux_ptr[i + 1] - aux_ptr[i]; }
    long long b_off(int i) const { return aux_ptr[i] * (long long)n_vir; }
};


// Records CUDA events around one stage of the pipeline on the context's stream when profiling is on.
struct StageTimer {
    osv_ctx &c;
    osv::ProfEvent e{};
    StageTimer(osv_ctx &ctx, const char *name) : c(ctx) {
        if (!c.prof && !c.capturing) return;
        e.name = name;
        e.a = c.take_event();
        e.b = c.take_event();
        record(e.a);
    }
    void record(cudaEvent_t ev) {
        if (c.capturing) cudaEventRecordWithFlags(ev, c.stream, cudaEventRecordExternal);
        else cudaEventRecord(ev, c.stream);
    }
    ~StageTimer() {
        if (!e.a) return;
        record(e.b);
        (c.capturing ? c.gev : c.pev).push_back(e);
    }
};
