// The general min-sum path (vs_bp_wide.cu): Eq. 1 for the parameters the
// byte-message kernels of vs_bp.cu cannot hold -- more than 128 labels,
// truncations above 127, or coarse data terms beyond 16 bits.  Internal to
// the library; vs_bp_stereo and its companions dispatch here.
#pragma once

#include "vs_common.cuh"

#include <utility>
#include <vector>

namespace vs {

// Parameters the general path accepts (labels 2..256, levels 1..8,
// smooth_trunc <= 65535, data_trunc * 4^(levels-1) <= 2^28).
bool bp_wide_params_ok(int w, int h, const vs_bp_params *p);
size_t bp_wide_workspace_size(int w, int h, const vs_bp_params *p);
// Offset of the status word inside the workspace.
size_t bp_wide_status_offset(int w, int h, const vs_bp_params *p);
// Eq. 1 on `st`; the workspace is checked by the caller.
// check_shrink: test aid of the checked build (bytes taken off the end of the
// workspace's registered range); kCheckKeepRanges: keep the ranges a batch
// registered for all its pairs.
constexpr size_t kCheckKeepRanges = ~(size_t)0;
void bp_wide_run(const uint8_t *left, const uint8_t *right, int w, int h, int pitch, const vs_bp_params *p,
                 uint8_t *labels, int labels_pitch, uint8_t *ws, cudaStream_t st, size_t check_shrink = 0);
// Final level-0 incoming messages as int32 [4][h][w][labels].
void bp_wide_export(const uint8_t *ws, int w, int h, const vs_bp_params *p, int32_t *out, cudaStream_t st);
#ifdef VS_CHECKED
// The first bounds violation the general path's kernels recorded (site + 1,
// 0 if none) and its address; clears it.
unsigned long long bp_wide_check_take(unsigned long long *addr);
void bp_wide_check_ranges(cudaStream_t st, const std::vector<std::pair<const void *, size_t>> &bufs);
#endif

}  // namespace vs
