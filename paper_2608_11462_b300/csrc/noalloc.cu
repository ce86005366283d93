// noalloc.cu -- a dense PHS product that allocates no device memory.
//
// phs_dense_matvec stages the caller's n x 2 points in a scratch array that it
// allocates per call.  Some callers cannot allocate: real-time loops that must not
// trigger the implicit device synchronisation of cudaMalloc/cudaFree, and applications
// that reserve all device memory for their own pool up front.
// phs_dense_matvec_noalloc stages the points in a fixed file-scope device array
// instead (kNoAllocMaxPoints points, 1 MiB, held by every GPU that loads this library
// until the process exits) and otherwise runs the same exact all-pairs kernel.  The
// array's device address is looked up once per device, by the first call made with
// that device current, and kept for the life of the process: after a
// cudaDeviceReset the module is loaded again and that address is stale, so the
// library must not be used across a reset of a device it has run on.
#include <mutex>

#include "phs_internal.cuh"

namespace phs {
namespace {

constexpr int64_t kNoAllocMaxPoints = 65536;
constexpr int kMaxDevices = 64;

// In host code this name is only a host-side stand-in for the device array: its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double2 g_noalloc_pts[kNoAllocMaxPoints];

std::mutex g_noalloc_mu;
double2 *g_noalloc_addr[kMaxDevices] = {};

// device address of g_noalloc_pts on the current device (looked up once per device)
double2 *noalloc_scratch() {
    int dev = -1;
    PHS_CUDA(cudaGetDevice(&dev));
    PHS_REQUIRE(dev >= 0 && dev < kMaxDevices, PHS_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        PHS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_pts));
        g_noalloc_addr[dev] = static_cast<double2 *>(p);
    }
    return g_noalloc_addr[dev];
}

__global__ void pack_points(const double *pts, int64_t n, double2 *dst) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = make_double2(pts[2 * j], pts[2 * j + 1]);
}

}  // namespace
}  // namespace phs

extern "C" phs_status phs_dense_matvec_noalloc(const double *pts_dev, int64_t n, int k, const double *t_dev,
                                               double *out_dev, phs_stream_t stream) {
    PHS_TRY
    PHS_REQUIRE(pts_dev && t_dev && out_dev && n >= 0 && k >= 1 && k <= 5, PHS_ERR_INVALID_ARG, "bad arguments");
    PHS_REQUIRE(n <= phs::kNoAllocMaxPoints, PHS_ERR_INVALID_ARG,
                "phs_dense_matvec_noalloc: n exceeds the fixed scratch capacity of 65536 points");
    double2 *scratch = phs::noalloc_scratch();
    if (n > 0) {
        cudaStream_t s = (cudaStream_t)stream;
        phs::pack_points<<<phs::blocks_for(n, 256), 256, 0, s>>>(pts_dev, n, scratch);
        PHS_LAUNCH_CHECK();
        phs::dense_matvec64(scratch, n, k, t_dev, out_dev, s);
    }
    PHS_CATCH
}
