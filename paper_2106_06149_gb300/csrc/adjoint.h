// Adjoint (gradient) of the MBE(3)-OSV-MP2 energy: dE/dB and dE/df_occ (amplitudes variational, Sec. 2.1).
#pragma once
#include <string>
#include <vector>

#include "kernels.cuh"
#include "tc_gemm.h"

struct osv_ctx;

namespace osv {

// What the per-cluster partial kernels read and accumulate (device pointers): cluster / slot / term lists, pair
// dimensions, occupied Fock, pair energies, slot amplitudes, coupling blocks; accumulators dE/dS~ and dE/dF~ per
// pair (GS, GF), dE/dS~ per coupling block (GSc), dE/df_occ (dF).  ld: shared-memory leading dimension of the
// double-float kernel.
struct AdjArgsS {
    const ClusterInfo *clusters;
    const int *order;
    const Slot *slots;
    const Term *terms;
    const PairInfo *pairs;
    const int *rdim;
    const double *focc, *e, *Tslot, *Stil;
    int n_occ, ncl, ld;
    double *GS, *GF, *GSc, *dF;
    double *TbS;   // tensor-core kernel: Tb = 2T - T^T per slot (slot amplitude layout), formed by its slot phase
    int *ebS;      // and the scale exponent of each slot's Tb
};

// The same partials on the tensor cores (exact BF16 slices of every operand, tcgen05 with the sums in tensor
// memory) for pair orders <= kAdjTcMaxOrder; err receives kDevTimeout if a bounded wait expires.
constexpr int kAdjTcMaxOrder = 80;
cudaError_t launch_cluster_adjoint_tc(const AdjArgsS &a, int ncl, int *err, long long budget, cudaStream_t s);

struct AdjointPlan {
    bool planned = false;
    std::vector<void *> allocs;
    // accumulators in the pseudo-canonical pair bases, their OSV-basis images, LMO-pair blocks
    double *GS = nullptr, *GF = nullptr, *GK = nullptr, *GSo = nullptr, *GFo = nullptr, *GKo = nullptr,
           *ptmp = nullptr, *GSc = nullptr, *GSco = nullptr, *ctmp = nullptr, *HS = nullptr, *HF = nullptr;
    // chain to W, Q, B and the OSV relaxation
    double *Z = nullptr, *dQ = nullptr, *dB64 = nullptr, *dF64 = nullptr, *A1 = nullptr;
    double *TbS = nullptr;   // Tb per cluster slot (tensor-core adjoint)
    int *ebS = nullptr;
    double *scratch = nullptr;
    int *zrows = nullptr;   // per off-diagonal pair: W row maps of its two stacked-K products into Z
    long long pstride = 0;
    int grid = 0;
    struct {
        std::vector<BlockCopy> h;
        BlockCopy *d = nullptr;
    } bc_hs;
    GemmBatch gb_kc1, gb_kc2, gb_f1, gb_f2, gb_k1, gb_k2, gb_c1, gb_c2, gb_z, gb_db, gb_dq, gb_gt, gb_rb;
    GemmBatch gb_at;                            // mixed relaxation: A1 T (FP64 residual of the resolvent solve)
    TcTiles oz_z, oz_db, oz_dq, oz_gt, oz_rb;   // tensor-core tilings, exact BF16x4

    void release();
    cudaError_t plan(osv_ctx &c);
    cudaError_t run(osv_ctx &c, double scale, void *dB, double *dF, std::string &msg);
};

}  // namespace osv
