// noalloc.cu - transmission_bwd without a caller-supplied work buffer.
//
// Some callers cannot allocate device memory themselves: a host program
// whose device memory is handed out entirely by another framework's
// allocator, or a tight loop that cannot pay for cudaMalloc's implicit
// device synchronisation.  For them this file keeps the backward pass's
// scratch (one row of partial gradient sums per 1024-ray block) in a
// fixed-size array that lives in the library's own device image.  The
// caller still provides the rays, sigma, dL/dT and the gradient output.
//
// Costs and limits, stated for users:
//  - every GPU that loads the library holds NOALLOC_SCRATCH_BYTES for this
//    array until the process exits;
//  - n is limited so that the partial sums fit in the array (about 44
//    million rays with 8 materials; more with fewer materials);
//  - all calls share the array: two calls whose kernels overlap on the GPU
//    (different streams, no ordering between them) race on it.  Order them
//    on one stream, or use transmission_bwd with separate work buffers;
//  - the first call on a device looks up the array's device address (once
//    per device, with that device current); make that first call before
//    any stream capture.  The address is kept for the life of the process:
//    after cudaDeviceReset (or a release of the device's primary context)
//    the module is loaded again elsewhere, so do not call this entry point
//    on a device that has been reset.
// The partial sums are written in full before they are read, so nothing in
// the array needs clearing between calls.
#include <cstdint>
#include <mutex>

#include "trk.h"
#include "trk_internal.h"
#include "trk_launch.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(4) << 20;   // 4 MiB

static __device__ __align__(256) unsigned char g_bwd_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_lock;
void* g_addr[64] = {nullptr};

// Device address of g_bwd_scratch on the current device (looked up once).
trk_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return trk_status(trk::set_error(TRK_E_CUDA, "transmission_bwd_noalloc: %s", cudaGetErrorString(e)));
    if (dev < 0 || dev >= 64) return trk_status(trk::set_error(TRK_E_UNSUPPORTED, "transmission_bwd_noalloc: device %d", dev));
    std::lock_guard<std::mutex> lk(g_lock);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bwd_scratch);
        if (e != cudaSuccess || !p)
            return trk_status(trk::set_error(TRK_E_CUDA, "transmission_bwd_noalloc: cudaGetSymbolAddress: %s",
                                             cudaGetErrorString(e)));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return TRK_OK;
}

}  // namespace

extern "C" {

trk_status transmission_bwd_noalloc(trk_geom_t g, int tracker, int64_t n, const double* dev_rays,
                                    const double* dev_sigma, double pitch, const double* dev_gT, double* dev_grad,
                                    void* stream) {
    if (!g || g->magic != TRK_GEOM_MAGIC || n < 0)
        return trk_status(trk::set_error(TRK_E_INVALID, "transmission_bwd_noalloc: bad arguments"));
    size_t need = 0;
    trk_status st = transmission_bwd_work_bytes(g, n, &need);
    if (st != TRK_OK) return st;
    if (need > NOALLOC_SCRATCH_BYTES) {
        const long long per_block = (long long)(g->n_mat + TRK_NGEOM_PARAMS) * 8;
        const long long max_rays = (long long)(NOALLOC_SCRATCH_BYTES / size_t(per_block)) * trk::TRK_RAYS_PER_BLOCK;
        return trk_status(trk::set_error(TRK_E_NOMEM,
                                         "transmission_bwd_noalloc: %lld rays need %zu scratch bytes, the fixed array "
                                         "holds %zu (at most %lld rays for this geometry); use transmission_bwd",
                                         (long long)n, need, NOALLOC_SCRATCH_BYTES, max_rays));
    }
    void* scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != TRK_OK) return st;
    return transmission_bwd(g, tracker, n, dev_rays, dev_sigma, pitch, dev_gT, dev_grad, scratch,
                            NOALLOC_SCRATCH_BYTES, stream);
}

}  // extern "C"
