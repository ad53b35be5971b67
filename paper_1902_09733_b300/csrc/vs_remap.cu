// Section 2.1 undistort/rectify remap fused with the Section 2.2 downsample.
//
// One CTA owns a tile of TLW x TLH low-resolution pixels, i.e. an aligned
// block of (TLW s) x (TLH s) full-resolution pixels.  Each thread maps its
// destination pixels through the radial lens model (FP32), samples the
// source bilinearly in fixed point (weights in 1/4096: a two-term dot
// product per row and channel, no byte-to-float conversions), rounds, writes
// the full-resolution RGB and keeps a copy in shared memory; the CTA then
// reduces every s x s block to the low-res RGB mean and its grey.  One
// launch per frame, no intermediate buffers.
#include "vs_common.cuh"

namespace vs {
namespace {

constexpr int kRemapThreads = 256;
constexpr int kTileFullW = 64;   // full-res tile width target
constexpr int kTileFullH = 16;   // full-res tile height target
constexpr int kTilePixMax = kTileFullW * kTileFullH;

struct RemapArgs {
    const uint8_t *src;
    uint8_t *dst;
    uint8_t *low_rgb;
    uint8_t *low_gray;
    int W, H, src_pitch, dst_pitch, low_rgb_pitch, low_gray_pitch;
    int s, w, h;                // scale and low-res size
    int tlw, tlh;               // tile size in low-res pixels
    float fx, fy, cx, cy, k1, k2;
    float inv_fx, inv_fy;   // 1/fx, 1/fy rounded once on the host
    int dst_vec;            // dst rows allow 4-byte stores of 4-pixel groups
    int src_words;          // src rows start on 4-byte boundaries (aligned word gathers)
    float R[9];
    int has_R;
};

__device__ __forceinline__ float tap(const uint8_t *src, int pitch, int W, int H, int x, int y, int ch)
{
    if (x < 0 || y < 0 || x >= W || y >= H)
        return 0.0f;
    return (float)__ldg(src + (size_t)y * pitch + (size_t)x * 3 + ch);
}

// Destination pixels are processed four consecutive ones per thread, so the
// 48 tap loads of a thread are all in flight together and its 12 output
// bytes leave as three 32-bit stores when the row allows it.
__global__ void __launch_bounds__(kRemapThreads) k_remap_down(RemapArgs a)
{
    pdl_begin();
    __shared__ uint8_t tile[kTilePixMax * 3];
    const int tfw = a.tlw * a.s, tfh = a.tlh * a.s;   // full-res tile size
    const int u0 = blockIdx.x * tfw, v0 = blockIdx.y * tfh;
    const bool want_low = (a.low_rgb != nullptr) || (a.low_gray != nullptr);
    const int quads = (tfw + 3) / 4;                  // 4-pixel groups per tile row

    for (int g = threadIdx.x; g < quads * tfh; g += blockDim.x) {
        const int lv = g / quads, lu0 = 4 * (g % quads);
        const int v = v0 + lv;
        uint8_t out[12];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int lu = lu0 + q, u = u0 + lu;
            int ival[3] = {0, 0, 0};   // rounded sample; 0 for rays that miss the frame
            if (lu < tfw && u < a.W && v < a.H) {
                float xn = ((float)u - a.cx) * a.inv_fx;
                float yn = ((float)v - a.cy) * a.inv_fy;
                bool valid = true;
                if (a.has_R) {
                    const float X = a.R[0] * xn + a.R[3] * yn + a.R[6];
                    const float Y = a.R[1] * xn + a.R[4] * yn + a.R[7];
                    const float Z = a.R[2] * xn + a.R[5] * yn + a.R[8];
                    if (Z <= 0.0f) {
                        valid = false;
                    } else {
                        xn = X / Z;
                        yn = Y / Z;
                    }
                }
                if (valid) {
                    const float r2 = xn * xn + yn * yn;
                    const float radial = 1.0f + a.k1 * r2 + a.k2 * r2 * r2;
                    const float sx = a.fx * (xn * radial) + a.cx;
                    const float sy = a.fy * (yn * radial) + a.cy;
                    if (sx > -1.0f && sx < (float)a.W && sy > -1.0f && sy < (float)a.H) {
                        const float fx0 = floorf(sx), fy0 = floorf(sy);
                        const int x0 = (int)fx0, y0 = (int)fy0;
                        const float ax = sx - fx0, ay = sy - fy0;
                        // the two taps of each row per channel, packed as (R0 R1 G0 G1) and
                        // (B0 B1 . .), top row t_*, bottom row b_*; taps outside the frame are 0
                        uint32_t t_rg, t_b, b_rg, b_b;
                        if (x0 >= 0 && y0 >= 0 && x0 + 2 < a.W && y0 + 1 < a.H && a.src_words) {
                            // all four taps in the frame, and the aligned words that
                            // cover each row's 6 bytes end inside that row: 4 to 6 loads
                            const uint8_t *p0 = a.src + (size_t)y0 * a.src_pitch + 3 * x0;
                            const uint32_t o = (uint32_t)(reinterpret_cast<uintptr_t>(p0) & 3u);
                            const uint32_t *q0 = reinterpret_cast<const uint32_t *>(p0 - o);
                            const uint32_t *q1 = reinterpret_cast<const uint32_t *>(p0 - o + a.src_pitch);
                            const uint32_t a0 = __ldg(q0), a1 = __ldg(q0 + 1), b0 = __ldg(q1), b1 = __ldg(q1 + 1);
                            // byte o + 5 lies in a third word only for o = 3 (it is then
                            // byte 3x0 + 5 of the row, inside it since x0 + 3 <= W)
                            const uint32_t a2 = o == 3 ? __ldg(q0 + 2) : 0u, b2 = o == 3 ? __ldg(q1 + 2) : 0u;
                            // bytes o .. o+5 of each row: (R0 G0 B0 R1) from {a1:a0}, (G1 B1) from {a2:a1}
                            const uint32_t s_lo = o | ((o + 1) << 4) | ((o + 2) << 8) | ((o + 3) << 12);
                            const uint32_t s_hi = o | ((o + 1) << 4);
                            const uint32_t r0a = prmt(a0, a1, s_lo), r0b = prmt(a1, a2, s_hi);
                            const uint32_t r1a = prmt(b0, b1, s_lo), r1b = prmt(b1, b2, s_hi);
                            t_rg = prmt(r0a, r0b, 0x4130u), t_b = prmt(r0a, r0b, 0x0052u);
                            b_rg = prmt(r1a, r1b, 0x4130u), b_b = prmt(r1a, r1b, 0x0052u);
                        } else {
                            // byte loads, with frame checks where a tap may be outside
                            uint32_t tq[2][2][3];   // [row][column][channel]
#pragma unroll
                            for (int jy = 0; jy < 2; ++jy)
#pragma unroll
                                for (int jx = 0; jx < 2; ++jx)
#pragma unroll
                                    for (int ch = 0; ch < 3; ++ch)
                                        tq[jy][jx][ch] = (uint32_t)tap(a.src, a.src_pitch, a.W, a.H, x0 + jx, y0 + jy, ch);
                            t_rg = tq[0][0][0] | (tq[0][1][0] << 8) | (tq[0][0][1] << 16) | (tq[0][1][1] << 24);
                            t_b = tq[0][0][2] | (tq[0][1][2] << 8);
                            b_rg = tq[1][0][0] | (tq[1][1][0] << 8) | (tq[1][0][1] << 16) | (tq[1][1][1] << 24);
                            b_b = tq[1][0][2] | (tq[1][1][2] << 8);
                        }
                        // fixed-point bilinear blend: weights in 1/4096, each row's two taps
                        // per channel in one 16 x 8-bit two-term dot product, the rows in
                        // 32-bit integers; within 0.06 of the exact value before rounding
                        const uint32_t axq = (uint32_t)__float2int_rn(ax * 4096.0f);
                        const uint32_t ayq = (uint32_t)__float2int_rn(ay * 4096.0f);
                        const uint32_t wx = (axq << 16) | (4096u - axq);   // (left, right) tap weights
                        const uint32_t top[3] = {__dp2a_lo(wx, t_rg, 0u), __dp2a_hi(wx, t_rg, 0u),
                                                 __dp2a_lo(wx, t_b, 0u)};
                        const uint32_t bot[3] = {__dp2a_lo(wx, b_rg, 0u), __dp2a_hi(wx, b_rg, 0u),
                                                 __dp2a_lo(wx, b_b, 0u)};
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) {
                            const uint32_t vv = top[ch] * (4096u - ayq) + bot[ch] * ayq;   // < 2^32
                            ival[ch] = (int)((vv + (1u << 23)) >> 24);   // round half up
                        }
                    }
                }
            }
#pragma unroll
            for (int ch = 0; ch < 3; ++ch)
                out[3 * q + ch] = (uint8_t)min(max(ival[ch], 0), 255);
        }
        if (v >= a.H)
            continue;
        const int u = u0 + lu0;
        const int nq = min(4, min(tfw - lu0, a.W - u));   // pixels of this group inside tile and frame
        if (a.dst && nq > 0) {
            uint8_t *d = a.dst + (size_t)v * a.dst_pitch + (size_t)u * 3;
            if (nq == 4 && a.dst_vec && (u & 3) == 0) {
                uint32_t w[3];
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    w[k] = (uint32_t)out[4 * k] | ((uint32_t)out[4 * k + 1] << 8) | ((uint32_t)out[4 * k + 2] << 16) |
                           ((uint32_t)out[4 * k + 3] << 24);
                uint32_t *d32 = reinterpret_cast<uint32_t *>(d);
                d32[0] = w[0];
                d32[1] = w[1];
                d32[2] = w[2];
            } else {
#pragma unroll
                for (int k = 0; k < 12; ++k)
                    if (k < 3 * nq)
                        d[k] = out[k];
            }
        }
        if (want_low) {
#pragma unroll
            for (int k = 0; k < 12; ++k)
                if (k < 3 * nq)
                    tile[(lv * tfw + lu0) * 3 + k] = out[k];
        }
    }
    if (!want_low)
        return;
    __syncthreads();
    for (int j = threadIdx.x; j < a.tlw * a.tlh; j += blockDim.x) {
        const int lx = j % a.tlw, ly = j / a.tlw;
        const int xl = blockIdx.x * a.tlw + lx, yl = blockIdx.y * a.tlh + ly;
        if (xl >= a.w || yl >= a.h)
            continue;
        int sum[3] = {0, 0, 0};
        int n = 0;
        for (int jj = 0; jj < a.s; ++jj) {
            const int v = yl * a.s + jj;
            if (v >= a.H)
                break;
            for (int ii = 0; ii < a.s; ++ii) {
                const int u = xl * a.s + ii;
                if (u >= a.W)
                    break;
                const int t = ((ly * a.s + jj) * tfw + lx * a.s + ii) * 3;
                sum[0] += tile[t];
                sum[1] += tile[t + 1];
                sum[2] += tile[t + 2];
                ++n;
            }
        }
        int mean[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
            mean[ch] = (sum[ch] + n / 2) / n;
        if (a.low_rgb) {
            uint8_t *d = a.low_rgb + (size_t)yl * a.low_rgb_pitch + (size_t)xl * 3;
            d[0] = (uint8_t)mean[0];
            d[1] = (uint8_t)mean[1];
            d[2] = (uint8_t)mean[2];
        }
        if (a.low_gray)
            a.low_gray[(size_t)yl * a.low_gray_pitch + xl] =
                (uint8_t)((77 * mean[0] + 150 * mean[1] + 29 * mean[2] + 128) >> 8);
    }
}

}  // namespace
}  // namespace vs

extern "C" int vs_rectify_remap(const uint8_t *src, int W, int H, int src_pitch,
                                const vs_camera *cam, const float *R9,
                                uint8_t *dst, int dst_pitch, int scale,
                                uint8_t *low_rgb, int low_rgb_pitch,
                                uint8_t *low_gray, int low_gray_pitch, void *stream)
{
    using namespace vs;
    if (!src || !cam || W <= 0 || H <= 0 || src_pitch < 3 * W)
        return VS_EINVAL;
    if (!dst && !low_rgb && !low_gray)
        return VS_EINVAL;
    if (dst && dst_pitch < 3 * W)
        return VS_EINVAL;
    const float cv[6] = {cam->fx, cam->fy, cam->cx, cam->cy, cam->k1, cam->k2};
    for (float f : cv)
        if (!isfinite(f))
            return VS_EINVAL;
    if (cam->fx == 0.0f || cam->fy == 0.0f)
        return VS_EINVAL;
    const bool want_low = low_rgb || low_gray;
    if (want_low && (scale < 1 || scale > 16))
        return VS_EINVAL;
    const int s = want_low ? scale : 1;
    const int w = (W + s - 1) / s, h = (H + s - 1) / s;
    if (low_rgb && low_rgb_pitch < 3 * w)
        return VS_EINVAL;
    if (low_gray && low_gray_pitch < w)
        return VS_EINVAL;

    RemapArgs a;
    a.src = src;
    a.dst = dst;
    a.low_rgb = low_rgb;
    a.low_gray = low_gray;
    a.W = W;
    a.H = H;
    a.src_pitch = src_pitch;
    a.dst_pitch = dst_pitch;
    a.low_rgb_pitch = low_rgb_pitch;
    a.low_gray_pitch = low_gray_pitch;
    a.s = s;
    a.w = w;
    a.h = h;
    a.tlw = kTileFullW / s > 0 ? kTileFullW / s : 1;
    a.tlh = kTileFullH / s > 0 ? kTileFullH / s : 1;
    a.fx = cam->fx;
    a.fy = cam->fy;
    a.cx = cam->cx;
    a.cy = cam->cy;
    a.k1 = cam->k1;
    a.k2 = cam->k2;
    a.inv_fx = (float)(1.0 / (double)cam->fx);
    a.inv_fy = (float)(1.0 / (double)cam->fy);
    // 4-pixel groups start at multiples of 4 pixels (12 bytes) of the row
    a.dst_vec = dst != nullptr && aligned(dst, 4) && dst_pitch % 4 == 0;
    a.src_words = aligned(src, 4) && src_pitch % 4 == 0;
    a.has_R = R9 != nullptr;
    for (int i = 0; i < 9; ++i)
        a.R[i] = R9 ? R9[i] : (i % 4 == 0 ? 1.0f : 0.0f);
    const int tfw = a.tlw * s, tfh = a.tlh * s;
    dim3 grid((W + tfw - 1) / tfw, (H + tfh - 1) / tfh);
    const int slot = prof_begin(kProfRemap, (cudaStream_t)stream);
    launch_pdl(k_remap_down, dim3(grid), dim3(kRemapThreads), (cudaStream_t)stream, a);
    prof_end(slot, (cudaStream_t)stream);
    note_launch();
    return launch_status();
}
