// vs_bp_stereo_noalloc: the stereo step with library-owned scratch, for
// callers that cannot allocate device memory themselves.
//
// The scratch is one file-scope __device__ array of VS_BP_NOALLOC_SCRATCH_BYTES
// bytes.  Every GPU that loads the library carries one copy until the process
// exits.  In host code the array's name only stands for the symbol, so its
// device address is looked up with cudaGetSymbolAddress (with the device
// current) and that address is what the kernels receive.
#include "vs_common.cuh"

#include <mutex>

namespace vs {
namespace {

static __device__ __align__(256) uint8_t g_bp_scratch[VS_BP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_bp_scratch for the current device.  Outside stream
// capture it is looked up on every call: if the runtime loads the module
// again (after cudaDeviceReset, for example) the array may move, and a
// remembered address would then point at freed memory.  While `st` is being
// captured, the address of the last lookup on this device is used instead (a
// lookup may have to load the module, which must not happen inside a
// capture), so a device's first call must come before any capture.
int scratch_address(cudaStream_t st, void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return VS_ECUDA;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        (void)cudaGetLastError();
        return VS_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bp_scratch) != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return VS_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    } else if (g_scratch_ptr[dev] == nullptr) {
        return VS_ECUDA;   // first call on this device inside a capture
    }
    *out = g_scratch_ptr[dev];
    return VS_OK;
}

// Arguments and size of a pair for the built-in scratch.
int noalloc_check(int w, int h, const vs_bp_params *p)
{
    const size_t need = vs_bp_workspace_size(w, h, p);
    if (need == 0)
        return VS_EINVAL;
    if (need > (size_t)VS_BP_NOALLOC_SCRATCH_BYTES)
        return VS_EWORKSPACE;   // the built-in scratch is too small for this pair
    return VS_OK;
}

}  // namespace
}  // namespace vs

extern "C" int vs_bp_stereo_noalloc(const uint8_t *left, const uint8_t *right, int w, int h, int pitch,
                                    const vs_bp_params *p, uint8_t *labels, int labels_pitch, void *stream)
{
    using namespace vs;
    int rc = noalloc_check(w, h, p);
    if (rc != VS_OK)
        return rc;
    void *ws = nullptr;
    rc = scratch_address((cudaStream_t)stream, &ws);
    if (rc != VS_OK)
        return rc;
    // The kernels read no scratch byte before writing it in the same call, so
    // nothing has to be cleared between calls.
    return vs_bp_stereo(left, right, w, h, pitch, p, labels, labels_pitch, ws, (size_t)VS_BP_NOALLOC_SCRATCH_BYTES,
                        stream);
}

extern "C" int vs_bp_noalloc_status(int w, int h, const vs_bp_params *p, void *stream)
{
    using namespace vs;
    int rc = noalloc_check(w, h, p);
    if (rc != VS_OK)
        return rc;
    void *ws = nullptr;
    rc = scratch_address((cudaStream_t)stream, &ws);
    if (rc != VS_OK)
        return rc;
    return vs_bp_status(ws, (size_t)VS_BP_NOALLOC_SCRATCH_BYTES, w, h, p, stream);
}
