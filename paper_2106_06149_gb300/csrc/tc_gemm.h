// Grouped exact-slice GEMM on tcgen05 tensor cores (tc_oz.cu): tilings of the same GemmDesc batches as the FP64
// grouped GEMM.
#pragma once
#include <vector>

#include "kernels.cuh"

namespace osv {

struct TcTiles {
    long long tiles = 0;          // output tiles of the GEMM launch
    GemmDesc *d_desc = nullptr;   // exact-slice GEMM: descriptors with scale arrays attached
    int *d_exps = nullptr;
    int nprob = 0;
    // exact-slice GEMM: row-scale job prefixes per operand, the slicing jobs (128 x 32 operand tiles), the output
    // tiles (with the slice images they read) and the row tables of packed tiles; the scratch size the batch needs
    long long *d_sjobs0 = nullptr;
    long long jobs = 0, scratch_bytes = 0, sjobs = 0;   // sjobs: row-scale jobs (blocks of 32 operand rows)
    void *d_ops = nullptr;                              // distinct operands (shared by problems that read them)
    void *d_jobs = nullptr, *d_otiles = nullptr, *d_rows = nullptr;
    int nops = 0;
    long long packed_tiles = 0;                         // output tiles whose rows come from several problems
    std::vector<TcTiles> parts;                         // non-empty: the batch runs as these consecutive parts
};

void tc_tiles_free(TcTiles &tt);

// Exact-slice BF16x4 GEMM (unbiased, ~31 significant bits, tc_oz.cu): 128 x 128 tiling, per-row scale arrays,
// operands pre-sliced into scratch (tt.scratch_bytes, 16-byte aligned, shared by batches run one after another).
// Problems of fewer than 128 rows that read the same B operand share output tiles (row packing).
cudaError_t bf16x4_batch_prepare(GemmBatch &b, TcTiles &tt);
// budget: clock cycles of each main-loop wait before the tile gives up and raises kDevTimeout (<= 0: the default)
cudaError_t bf16x4_batch_run(const TcTiles &tt, unsigned char *scratch, int *err, long long budget, cudaStream_t s);

}  // namespace osv
