// Shared helpers of the CUDA virtual-stereo library (device code, launch
// bookkeeping).  Nothing here is shared with the CPU checker.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <utility>

#include <nvtx3/nvToolsExt.h>

#include "../../include/vstereo.h"

namespace vs {

// A named NVTX range around one entry point's work on the host (the stages
// of a pair appear by name in a profiler's timeline; without a tool
// attached a push and a pop cost a few nanoseconds).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Counts every kernel the library enqueues (vs_kernel_launches()).
void note_launch(unsigned n = 1);

// Status after a launch: VS_ECUDA if the runtime reports an error.
int launch_status();

// Library streams for independent work of one call (batches of pairs): up to
// kLibStreams per device, created on first use and kept.  fork_join runs
// body(k, side stream k) for k < n, every side stream ordered after the work
// already enqueued on `st`, and makes `st` wait for all of them -- with
// events, so it also works while `st` is being captured into a CUDA graph.
// The streams are shared by the device's calls: do not run two forked calls
// from different host threads at once.  Returns the first non-OK status of
// a body, or VS_ECUDA.
constexpr int kLibStreams = 4;
int fork_join(cudaStream_t st, int n, const std::function<int(int, cudaStream_t)> &body);

// Optional CUDA-event timing of selected launches (vs_profile_enable).
// prof_begin returns a slot (or -1 when timing is off) and records its start
// event on `st`; prof_end records the matching stop event.
enum ProfTag {
    kProfSweepL0 = 0,
    kProfSweepCoarse = 1,
    kProfRemap = 2,
    kProfJbu = 3,
    kProfBpOther = 4,
    kProfSmoothFwd = 5,
    kProfSmoothAdj = 6
};
int prof_begin(int tag, cudaStream_t st);
void prof_end(int slot, cudaStream_t st);

// Both frames of a pair through the block remap kernel in one launch (the
// left frame's full-res, low-res RGB and grey outputs, the right frame's
// grey); VS_EINVAL where that kernel does not apply (vs_remap.cu).
int remap_pair(const uint8_t *left, const uint8_t *right, int W, int H, int pitch, const vs_camera *cam, int scale,
               uint8_t *dst, int dst_pitch, uint8_t *low_rgb, int low_rgb_pitch, uint8_t *gray_l, uint8_t *gray_r,
               int gray_pitch, cudaStream_t st);

// Programmatic dependent launch.  Every kernel of the library starts with
// pdl_begin(): it waits until the previous kernel on the stream has finished
// and its writes are visible (a no-op when launched without the attribute),
// then lets the next kernel be scheduled.  Launched through launch_pdl, the
// next kernel's launch and set-up overlap this kernel's last wave.
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_smem(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                   Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args &&...args)
{
    return launch_pdl_smem(kern, grid, block, 0, st, std::forward<Args>(args)...);
}

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Packed 2 x 16-bit unsigned minimum (PTX ISA 8.0+, sm_90 and later).
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// 0 <= n < 2^23 as a float: n added into the mantissa of 2^23, minus 2^23
// (exact; an integer add and a float add instead of a quarter-rate
// conversion)
__device__ __forceinline__ float exact_float(int n)
{
    return __int_as_float(0x4B000000 + n) - 8388608.0f;
}

// Byte permute: result byte i = byte sel[i] of {b:a} (a = bytes 0..3); a
// selector nibble with bit 3 set replicates the sign bit of that byte.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

}  // namespace vs
