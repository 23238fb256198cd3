// Grouped split-TF32 GEMM on tcgen05 tensor cores (same GemmDesc batches as the FP64 grouped GEMM).
#pragma once
#include "kernels.cuh"

namespace osv {

struct TcTiles {
    long long *d_tile0 = nullptr;
    long long tiles = 0;
    GemmDesc *d_desc = nullptr;   // exact-slice GEMM: descriptors with scale arrays attached
    int *d_exps = nullptr;
    int nprob = 0;
};

// per-problem 128 x 64 tile offsets of an uploaded batch
cudaError_t tc_batch_prepare(GemmBatch &b, TcTiles &tt);
// err: device int set to kDevTimeout if a bounded mbarrier wait expires
cudaError_t tc_batch_run(const GemmBatch &b, const TcTiles &tt, int *err, cudaStream_t s);
void tc_tiles_free(TcTiles &tt);

// Exact-slice BF16x4 GEMM (unbiased, ~24 significant bits): own 128 x 64 tiling, per-row scale arrays.
cudaError_t bf16x4_batch_prepare(GemmBatch &b, TcTiles &tt);
cudaError_t bf16x4_batch_run(const TcTiles &tt, int *err, cudaStream_t s);

}  // namespace osv
