// osv_syev_batched_noalloc: the batched FP64 symmetric eigensolver of osv_syev_batched without any device
// allocation.  Meant for callers that cannot call cudaMalloc: code that runs under an external memory manager
// owning the whole device memory (a caching or arena allocator, where a stray cudaMalloc fails or fragments the
// pool), and latency-sensitive callers that cannot afford the implicit device-wide synchronisation of
// cudaFree.  Its scratch lives in file-scope __device__ arrays that every GPU loading this library holds until
// the process exits.
#include <string>
#include <vector>

#include "../../include/osvmbe.h"
#include "common.cuh"

namespace osv {
void set_noctx_error(const std::string &msg);   // defined in api.cu (message for osv_last_error(NULL))
}

namespace {

// Scratch: eigenvector accumulation (batch * n * n) and the tridiagonal vectors (3 * batch * n), in doubles.
constexpr long long kScratchDoubles = 1LL << 20;   // 8 MiB per device
constexpr int kMaxBatch = 1024;

static __device__ __align__(256) double g_scratch[kScratchDoubles];
static __device__ __align__(256) osv::EighDesc g_desc[kMaxBatch];
static __device__ __align__(256) int g_err[64];

struct DeviceAddrs {
    double *scratch = nullptr;
    osv::EighDesc *desc = nullptr;
    int *err = nullptr;
};

// Device addresses of the static arrays for the current device, looked up on every call: a cached address would
// go stale if the caller tears the primary context down (cudaDeviceReset) and a later call runs in a new one.  In
// host code the names g_scratch / g_desc / g_err are host-side stand-ins, never device addresses.
cudaError_t device_addrs(DeviceAddrs &a) {
    cudaError_t e;
    if ((e = cudaGetSymbolAddress((void **)&a.scratch, g_scratch)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void **)&a.desc, g_desc)) != cudaSuccess) return e;
    return cudaGetSymbolAddress((void **)&a.err, g_err);
}

}  // namespace

extern "C" osv_status osv_syev_batched_noalloc(const double *A, int n, int batch, double *w, double *Zt,
                                               void *cuda_stream) {
    if (!A || !w || !Zt || n < 1 || n > 4096 || batch < 1) {
        osv::set_noctx_error("osv_syev_batched_noalloc: bad argument (need A, w, Zt non-NULL, 1 <= n <= 4096, batch >= 1)");
        return OSV_ERR_INVALID;
    }
    const long long need = (long long)batch * n * n + 3LL * batch * n;
    if (batch > kMaxBatch || need > kScratchDoubles) {
        osv::set_noctx_error("osv_syev_batched_noalloc: batch*n*n + 3*batch*n = " + std::to_string(need) +
                             " doubles (batch " + std::to_string(batch) + ") exceeds the static scratch of " +
                             std::to_string(kScratchDoubles) + " doubles / " + std::to_string(kMaxBatch) +
                             " matrices; use osv_syev_batched");
        return OSV_ERR_INVALID;
    }
    DeviceAddrs a;
    cudaError_t e = device_addrs(a);
    if (e != cudaSuccess) {
        osv::set_noctx_error(std::string("osv_syev_batched_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return OSV_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const long long nn = (long long)n * n;
    std::vector<osv::EighDesc> h(batch);
    for (int b = 0; b < batch; ++b) {
        osv::EighDesc &D = h[b];
        D.A = Zt + b * nn;      // the caller's Zt holds the working copy, then the eigenvectors
        D.lda = n;
        D.n = n;
        D.n_dev = nullptr;
        D.w = w + (long long)b * n;
        D.Zt = Zt + b * nn;
        D.ldz = n;
        D.zwork = a.scratch + b * nn;
        D.d = a.scratch + batch * nn + 3LL * b * n;
        D.e = D.d + n;
        D.tau = D.e + n;
    }
    if (A != Zt) e = cudaMemcpyAsync(Zt, A, batch * nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.desc, h.data(), batch * sizeof(osv::EighDesc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.err, 0, sizeof(int), s);   // the error word starts at zero
    if (e == cudaSuccess) e = osv::eigh_batched(a.desc, batch, n, 0, a.err, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, a.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        osv::set_noctx_error(std::string("osv_syev_batched_noalloc: ") + cudaGetErrorString(e));
        return OSV_ERR_CUDA;
    }
    if (herr) {
        osv::set_noctx_error("osv_syev_batched_noalloc: QL iteration cap reached");
        return OSV_ERR_TIMEOUT;
    }
    return OSV_OK;
}
