// vs_bp_stereo_noalloc: the stereo step with library-owned scratch, for
// callers that cannot allocate device memory themselves.
//
// The scratch is one file-scope __device__ array of VS_BP_NOALLOC_SCRATCH_BYTES
// bytes.  Every GPU that loads the library carries one copy until the process
// exits.  In host code the array's name only stands for the symbol, so its
// device address is looked up once per device with cudaGetSymbolAddress (with
// that device current) and that address is what the kernels receive.
#include "vs_common.cuh"

#include <mutex>

namespace vs {
namespace {

static __device__ __align__(256) uint8_t g_bp_scratch[VS_BP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_bp_scratch on the current device (looked up on first use).
int scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return VS_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bp_scratch) != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return VS_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return VS_OK;
}

}  // namespace
}  // namespace vs

extern "C" int vs_bp_stereo_noalloc(const uint8_t *left, const uint8_t *right, int w, int h, int pitch,
                                    const vs_bp_params *p, uint8_t *labels, int labels_pitch, void *stream)
{
    using namespace vs;
    const size_t need = vs_bp_workspace_size(w, h, p);
    if (need == 0)
        return VS_EINVAL;
    if (need > (size_t)VS_BP_NOALLOC_SCRATCH_BYTES)
        return VS_EWORKSPACE;   // the built-in scratch is too small for this pair
    void *ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc != VS_OK)
        return rc;
    // The kernels read no scratch byte before writing it in the same call, so
    // nothing has to be cleared between calls.
    return vs_bp_stereo(left, right, w, h, pitch, p, labels, labels_pitch, ws, (size_t)VS_BP_NOALLOC_SCRATCH_BYTES,
                        stream);
}
