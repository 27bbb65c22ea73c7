// qmcrt_noalloc.cu -- qmcrt_trace_single_noalloc: single scattering straight into a
// caller's FP64 image, with the fixed-point accumulation scratch held in this file's
// own device array instead of a buffer the caller allocates.
//
// The scratch lives for as long as the library is loaded, on every GPU that loads it
// (QMCRT_NOALLOC_MAX_PIXELS x 3 int64 values = 6 MiB per GPU).  Calls share it: each
// call clears the part it uses before tracing, and two calls whose work overlaps on
// the GPU (different streams, or different host threads) corrupt each other's
// images.  Every call looks up the array's device address with the caller's device
// current (a cudaDeviceReset gives the array a new address, so nothing is cached);
// the first lookup on a device may load the library's kernels, so make the first call
// before any stream capture.
#include <cstring>

#include "qmcrt.h"
#include "qmcrt_internal.h"

namespace {

static __device__ __align__(256) long long g_noalloc_accum[3 * QMCRT_NOALLOC_MAX_PIXELS];

// Device address of g_noalloc_accum on the current device.  In host code the array's
// name stands for a host-side shadow, not a device address: only this address may be
// handed to a kernel.
int accum_address(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_accum);
    if (e != cudaSuccess || !p)
        return qmcrt::set_error(QMCRT_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    *out = p;
    return QMCRT_OK;
}

}  // namespace

extern "C" int qmcrt_trace_single_noalloc(const qmcrt_medium *medium, const qmcrt_source *source,
                                          const qmcrt_dust *dust, const qmcrt_observer *obs,
                                          const qmcrt_points_desc *pts, const qmcrt_trace_opts *opts,
                                          int32_t frac_bits, double scale, double *d_image, void *stream)
{
    if (!obs || obs->struct_size != sizeof(qmcrt_observer))
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "obs is NULL or has the wrong struct_size");
    if (!d_image) return qmcrt::set_error(QMCRT_ERR_INVALID_ARG, "d_image is NULL");
    if (obs->nx < 1 || obs->ny < 1 || (long long)obs->nx * obs->ny > QMCRT_NOALLOC_MAX_PIXELS)
        return qmcrt::set_error(QMCRT_ERR_INVALID_ARG,
                                "image of %d x %d pixels: the allocation-free entry point holds at most %d pixels",
                                obs->nx, obs->ny, QMCRT_NOALLOC_MAX_PIXELS);
    void *accum = nullptr;
    int rc = accum_address(&accum);
    if (rc) return rc;
    qmcrt_image im;
    memset(&im, 0, sizeof im);
    im.struct_size = sizeof im;
    im.accum = QMCRT_ACCUM_I64;
    im.d_accum = accum;
    im.n_images = 1;
    im.frac_bits = frac_bits;
    // every argument is checked before the first enqueue: a rejected call leaves
    // nothing on the stream (nor in a graph being captured)
    rc = qmcrt::check_trace_single(medium, source, dust, obs, pts, opts, &im);
    if (rc) return rc;
    const size_t bytes = (size_t)3 * obs->nx * obs->ny * sizeof(long long);
    const cudaError_t e = cudaMemsetAsync(accum, 0, bytes, (cudaStream_t)stream);
    if (e != cudaSuccess) return qmcrt::set_error(QMCRT_ERR_CUDA, "clearing the scratch: %s", cudaGetErrorString(e));
    rc = qmcrt_trace_single(medium, source, dust, obs, pts, opts, &im, nullptr, stream);
    if (rc) return rc;
    return qmcrt_image_reduce(&im, obs->nx, obs->ny, 1, scale, d_image, stream);
}
