// Section 2.1 undistort/rectify remap fused with the Section 2.2 downsample.
//
// Each destination pixel is mapped through the radial lens model (FP32) and
// the source sampled bilinearly in fixed point (weights in 1/4096: a two-term
// dot product per row and channel, no byte-to-float conversions), rounded
// half up; the kernel writes the full-resolution RGB and reduces every s x s
// block to the low-res RGB mean and its grey.  One launch per frame, no
// intermediate buffers.  k_remap_sq serves scales 2, 4 and 8 without
// rotation (the pair pipeline); k_remap_down everything else, staging its
// tile in shared memory for the block means.
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
    // k_remap_sq<S, true>: a second frame of the same camera and size sampled
    // at the same coordinates, only its low-res grey written
    const uint8_t *src2;
    uint8_t *low_gray2;
    int src2_pitch, low_gray2_pitch;
};

__device__ __forceinline__ uint32_t tap(const uint8_t *src, int pitch, int W, int H, int x, int y, int ch)
{
    if (x < 0 || y < 0 || x >= W || y >= H)
        return 0u;
    return (uint32_t)__ldg(src + (size_t)y * pitch + (size_t)x * 3 + ch);
}

// The normalised ray of destination pixel (u, v), rotated by R^T when a
// rotation is given; false for a ray with non-positive depth.
__device__ __forceinline__ bool ray(const RemapArgs &a, int u, int v, float &xn, float &yn)
{
    xn = __fmul_rn(__fsub_rn((float)u, a.cx), a.inv_fx);
    yn = __fmul_rn(__fsub_rn((float)v, a.cy), a.inv_fy);
    if (!a.has_R)
        return true;
    const float X = a.R[0] * xn + a.R[3] * yn + a.R[6];
    const float Y = a.R[1] * xn + a.R[4] * yn + a.R[7];
    const float Z = a.R[2] * xn + a.R[5] * yn + a.R[8];
    if (!(Z > 0.0f))
        return false;
    xn = X / Z;
    yn = Y / Z;
    return true;
}

// Radial distortion 1 + k1 r^2 + k2 r^4 and the pinhole back to source
// pixels; explicit fused multiply-adds, so every kernel rounds alike.
__device__ __forceinline__ void distort(const RemapArgs &a, float xn, float yn, float &sx, float &sy)
{
    const float r2 = fmaf(xn, xn, __fmul_rn(yn, yn));
    const float radial = fmaf(fmaf(a.k2, r2, a.k1), r2, 1.0f);
    sx = fmaf(a.fx, __fmul_rn(xn, radial), a.cx);
    sy = fmaf(a.fy, __fmul_rn(yn, radial), a.cy);
}

// Fixed-point bilinear blend: weights in 1/4096, each row's two taps per
// channel in one 16 x 8-bit two-term dot product, the rows in 32-bit
// integers.  t_rg / b_rg = (R0 R1 G0 G1) of the top / bottom row, t_b / b_b
// = (B0 B1 . .).  Returns value * 2^24 + 2^23 per channel: the rounded-half-up
// byte is bits 24..31 (the value is within 0.06 of the exact bilinear one).
__device__ __forceinline__ void blend(uint32_t t_rg, uint32_t t_b, uint32_t b_rg, uint32_t b_b, uint32_t axq,
                                      uint32_t ayq, uint32_t (&vv)[3])
{
    const uint32_t wx = axq * 0xFFFFu + 4096u;   // (4096 - axq, axq) as 2 x u16
    const uint32_t top[3] = {__dp2a_lo(wx, t_rg, 0u), __dp2a_hi(wx, t_rg, 0u), __dp2a_lo(wx, t_b, 0u)};
    const uint32_t bot[3] = {__dp2a_lo(wx, b_rg, 0u), __dp2a_hi(wx, b_rg, 0u), __dp2a_lo(wx, b_b, 0u)};
    const uint32_t ayc = 4096u - ayq;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch)
        vv[ch] = bot[ch] * ayq + (top[ch] * ayc + (1u << 23));   // < 2^32
}

// Taps of the 2 x 2 footprint at (x0, y0) from aligned words: needs x0 >= 0,
// y0 >= 0, x0 + 2 < W, y0 + 1 < H and word-aligned rows; q0 = the word that
// holds byte 3 x0 of row y0, o = that byte's position in it.  The words that
// cover a row's 6 bytes end inside that row: 4 to 6 loads.
__device__ __forceinline__ void taps_words(const uint32_t *q0, int pitch32, uint32_t o, uint32_t &t_rg,
                                           uint32_t &t_b, uint32_t &b_rg, uint32_t &b_b)
{
    const uint32_t *q1 = q0 + pitch32;
    const uint32_t a0 = __ldg(q0), a1 = __ldg(q0 + 1), b0 = __ldg(q1), b1 = __ldg(q1 + 1);
    // byte o + 5 lies in a third word only for o = 3 (it is then byte
    // 3 x0 + 5 of the row, inside it since x0 + 3 <= W)
    const uint32_t a2 = o == 3 ? __ldg(q0 + 2) : 0u, b2 = o == 3 ? __ldg(q1 + 2) : 0u;
    // bytes o .. o+5 of each row: (R0 G0 B0 R1) from {a1:a0}, (G1 B1) from {a2:a1}
    const uint32_t s_lo = o * 0x1111u + 0x3210u;
    const uint32_t s_hi = o * 0x11u + 0x10u;
    const uint32_t r0a = prmt(a0, a1, s_lo), r0b = prmt(a1, a2, s_hi);
    const uint32_t r1a = prmt(b0, b1, s_lo), r1b = prmt(b1, b2, s_hi);
    t_rg = prmt(r0a, r0b, 0x4130u), t_b = prmt(r0a, r0b, 0x0052u);
    b_rg = prmt(r1a, r1b, 0x4130u), b_b = prmt(r1a, r1b, 0x0052u);
}

// One destination pixel anywhere in the frame: blend accumulators as
// blend() returns them, 2^23 (byte 0) for rays that miss the frame.
__device__ __forceinline__ void sample_px(const RemapArgs &a, const uint8_t *src, int src_pitch, int u, int v,
                                          uint32_t (&vv)[3])
{
    vv[0] = vv[1] = vv[2] = 1u << 23;
    float xn, yn;
    if (!ray(a, u, v, xn, yn))
        return;
    float sx, sy;
    distort(a, xn, yn, sx, sy);
    if (!(sx > -1.0f && sx < (float)a.W && sy > -1.0f && sy < (float)a.H))
        return;
    const float fx0 = floorf(sx), fy0 = floorf(sy);
    const int x0 = (int)fx0, y0 = (int)fy0;
    const uint32_t axq = (uint32_t)__float2int_rn((sx - fx0) * 4096.0f);
    const uint32_t ayq = (uint32_t)__float2int_rn((sy - fy0) * 4096.0f);
    uint32_t t_rg, t_b, b_rg, b_b;
    if (x0 >= 0 && y0 >= 0 && x0 + 2 < a.W && y0 + 1 < a.H && a.src_words) {
        const uint8_t *p0 = src + (size_t)y0 * src_pitch + 3 * x0;
        const uint32_t o = (uint32_t)(reinterpret_cast<uintptr_t>(p0) & 3u);
        taps_words(reinterpret_cast<const uint32_t *>(p0 - o), src_pitch >> 2, o, t_rg, t_b, b_rg, b_b);
    } else {
        // byte loads, with frame checks where a tap may be outside
        uint32_t tq[2][2][3];   // [row][column][channel]
#pragma unroll
        for (int jy = 0; jy < 2; ++jy)
#pragma unroll
            for (int jx = 0; jx < 2; ++jx)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch)
                    tq[jy][jx][ch] = tap(src, src_pitch, a.W, a.H, x0 + jx, y0 + jy, ch);
        t_rg = tq[0][0][0] | (tq[0][1][0] << 8) | (tq[0][0][1] << 16) | (tq[0][1][1] << 24);
        t_b = tq[0][0][2] | (tq[0][1][2] << 8);
        b_rg = tq[1][0][0] | (tq[1][1][0] << 8) | (tq[1][0][1] << 16) | (tq[1][1][1] << 24);
        b_b = tq[1][0][2] | (tq[1][1][2] << 8);
    }
    blend(t_rg, t_b, b_rg, b_b, axq, ayq, vv);
}

// General kernel: any scale, rotation, alignment and frame size.  Destination
// pixels are processed four consecutive ones per thread, so the tap loads of
// a thread are in flight together and its 12 output bytes leave as three
// 32-bit stores when the row allows it.
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
            uint32_t vv[3] = {1u << 23, 1u << 23, 1u << 23};
            if (lu < tfw && u < a.W && v < a.H)
                sample_px(a, a.src, a.src_pitch, u, v, vv);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch)
                out[3 * q + ch] = (uint8_t)(vv[ch] >> 24);
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

constexpr float kFloorMagic = 12582912.0f;        // 1.5 x 2^23
constexpr uint32_t kFloorMagicBits = 0x4B400000u;

// The quad of four destination pixels u0 .. u0 + 3 of row v (inside the
// frame): coordinates from exact float arithmetic (integer-valued floats via
// the 2^23 mantissa, floors by a round-down add of 1.5 x 2^23) instead of
// conversions; when all four footprints are inside the frame, word gathers
// with no further checks, otherwise the general per-pixel sampler.  Writes
// the 12 bytes to dst (if wanted) and returns them packed in w.
// The quad's four pixels of `src` at the coordinates remap_quad found,
// packed as R0 G0 B0 R1 | G1 B1 R2 G2 | B2 R3 G3 B3.
__device__ __forceinline__ void sample_quad(const RemapArgs &a, const uint8_t *src, bool fast, const uint32_t (&off)[4],
                                            const uint32_t (&axq)[4], const uint32_t (&ayq)[4], int u0, int v,
                                            uint32_t (&w)[3])
{
    uint32_t vv[4][3];
    if (fast) {
        const uint32_t *src32 = reinterpret_cast<const uint32_t *>(src);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t t_rg, t_b, b_rg, b_b;
            taps_words(src32 + (off[q] >> 2), a.src_pitch >> 2, off[q] & 3u, t_rg, t_b, b_rg, b_b);
            blend(t_rg, t_b, b_rg, b_b, axq[q], ayq[q], vv[q]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            sample_px(a, src, a.src_pitch, u0 + q, v, vv[q]);
    }
    // the rounded bytes (bits 24..31)
    w[0] = prmt(prmt(vv[0][0], vv[0][1], 0x0073u), prmt(vv[0][2], vv[1][0], 0x0073u), 0x5410u);
    w[1] = prmt(prmt(vv[1][1], vv[1][2], 0x0073u), prmt(vv[2][0], vv[2][1], 0x0073u), 0x5410u);
    w[2] = prmt(prmt(vv[2][2], vv[3][0], 0x0073u), prmt(vv[3][1], vv[3][2], 0x0073u), 0x5410u);
}

// The lens model of a quad of four destination pixels once, then the
// samples of a.src (stored to a.dst when given) and, with PAIR, of a.src2.
template <bool PAIR>
__device__ __forceinline__ void remap_quad(const RemapArgs &a, int u0, int v, uint32_t (&w)[3], uint32_t (&w2)[3])
{
    float yn = __fmul_rn(__fsub_rn(exact_float(v), a.cy), a.inv_fy);
    uint32_t off[4], axq[4], ayq[4];
    bool fast = true;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float xn = __fmul_rn(__fsub_rn(exact_float(u0 + q), a.cx), a.inv_fx);
        float sx, sy;
        distort(a, xn, yn, sx, sy);
        // floors as integer-valued floats in [2^23, 2^24), exact for |s| < 2^22;
        // any other s (NaN and infinities too) gives an x0 / y0 that fails the
        // interior test below, since W and H are below 2^22
        const float bx = __fadd_rd(sx, kFloorMagic), by = __fadd_rd(sy, kFloorMagic);
        const int x0 = (int)(__float_as_uint(bx) - kFloorMagicBits);
        const int y0 = (int)(__float_as_uint(by) - kFloorMagicBits);
        fast = fast && (unsigned)x0 < (unsigned)(a.W - 2) && (unsigned)y0 < (unsigned)(a.H - 1);
        // round(frac * 4096) as the low bits of an integer-valued float
        axq[q] = __float_as_uint(fmaf(sx - (bx - kFloorMagic), 4096.0f, kFloorMagic)) - kFloorMagicBits;
        ayq[q] = __float_as_uint(fmaf(sy - (by - kFloorMagic), 4096.0f, kFloorMagic)) - kFloorMagicBits;
        off[q] = (uint32_t)y0 * (uint32_t)a.src_pitch + 3u * (uint32_t)x0;   // used only when fast
    }
    // only now wait for the previous kernel (which may still read the
    // buffers this one writes): the lens model above overlaps its last wave
    pdl_begin();
    sample_quad(a, a.src, fast, off, axq, ayq, u0, v, w);
    if (a.dst) {
        uint32_t *d32 = reinterpret_cast<uint32_t *>(a.dst + (size_t)v * a.dst_pitch + (size_t)u0 * 3);
        d32[0] = w[0];
        d32[1] = w[1];
        d32[2] = w[2];
    }
    if (PAIR)   // the second frame at the same coordinates (same size and row pitch)
        sample_quad(a, a.src2, fast, off, axq, ayq, u0, v, w2);
}

// Scale-2/4/8 kernel for the common case: no rotation, W a multiple of 4 and
// of s, H a multiple of s, both below 2^22, word-aligned source and
// destination rows, frame offsets below 2^31.  A CTA covers 64 x 16
// destination pixels and every lane one quad of 4 pixels of a row
// (remap_quad); the s x s block means are summed across the lanes of a
// block with shuffles:
//   s = 4: warp w takes block row w >> 1 and half w & 1 of the tile, lane
//          (r, i) = (lane >> 3, lane & 7) row r of block i: one quad per
//          block row, two shuffles;
//   s = 8: warp w takes block row w >> 2 and blocks 2 (w & 3), 2 (w & 3) + 1,
//          lane (b, r, h) = (lane >> 4, (lane >> 1) & 7, lane & 1) quad h of
//          row r of block b: four shuffles;
//   s = 2: warp w takes block row w, lane (r, q) = (lane >> 4, lane & 15) row
//          r of quad q, which spans two blocks: one shuffle.
template <int S, bool PAIR>
__global__ void __launch_bounds__(256) k_remap_sq(RemapArgs a)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int r, yl, xl, u0;
    if constexpr (S == 4) {
        r = lane >> 3;
        yl = blockIdx.y * 4 + (warp >> 1);
        xl = blockIdx.x * 16 + 8 * (warp & 1) + (lane & 7);
        u0 = 4 * xl;
    } else if constexpr (S == 8) {
        r = (lane >> 1) & 7;
        yl = blockIdx.y * 2 + (warp >> 2);
        xl = blockIdx.x * 8 + 2 * (warp & 3) + (lane >> 4);
        u0 = 8 * xl + 4 * (lane & 1);
    } else {
        r = lane >> 4;
        yl = blockIdx.y * 8 + warp;
        u0 = blockIdx.x * 64 + 4 * (lane & 15);
        xl = u0 / 2;
    }
    if (S * yl >= a.H)   // the whole warp (H is a multiple of S)
        return;
    const int v = S * yl + r;
    const bool inside = u0 < a.W;   // whole quad (W is a multiple of 4)
    uint32_t w[3] = {0u, 0u, 0u}, w2[3] = {0u, 0u, 0u};
    if (inside)
        remap_quad<PAIR>(a, u0, v, w, w2);
    if (!a.low_rgb && !a.low_gray && !PAIR)
        return;
    auto put = [&](int x, uint32_t R, uint32_t G, uint32_t B) {
        if (a.low_rgb) {
            uint8_t *d = a.low_rgb + (size_t)yl * a.low_rgb_pitch + (size_t)x * 3;
            d[0] = (uint8_t)R;
            d[1] = (uint8_t)G;
            d[2] = (uint8_t)B;
        }
        if (a.low_gray)
            a.low_gray[(size_t)yl * a.low_gray_pitch + x] = (uint8_t)((77u * R + 150u * G + 29u * B + 128u) >> 8);
    };
    const unsigned full = 0xFFFFFFFFu;
    // block means of one frame's words, handed to `out` by the block's lead lanes
    auto means = [&](const uint32_t (&w)[3], auto &&out) {
        if constexpr (S == 2) {
            // the quad's bytes R0 G0 B0 R1 | G1 B1 R2 G2 | B2 R3 G3 B3: pixels 0-1
            // belong to block xl, pixels 2-3 to block xl + 1
            const uint32_t rA = __dp4a(w[0], 0x01000001u, 0u);
            const uint32_t gA = __dp4a(w[0], 0x00000100u, __dp4a(w[1], 0x00000001u, 0u));
            const uint32_t bA = __dp4a(w[0], 0x00010000u, __dp4a(w[1], 0x00000100u, 0u));
            const uint32_t rB = __dp4a(w[1], 0x00010000u, __dp4a(w[2], 0x00000100u, 0u));
            const uint32_t gB = __dp4a(w[1], 0x01000000u, __dp4a(w[2], 0x00010000u, 0u));
            const uint32_t bB = __dp4a(w[2], 0x01000001u, 0u);
            uint32_t pA = rA | (gA << 16), pB = rB | (gB << 16), qAB = bA | (bB << 16);   // sums <= 4 x 255
            pA += __shfl_xor_sync(full, pA, 16);
            pB += __shfl_xor_sync(full, pB, 16);
            qAB += __shfl_xor_sync(full, qAB, 16);
            if (r != 0 || !inside)
                return;
            out(xl, ((pA & 0xFFFFu) + 2u) >> 2, ((pA >> 16) + 2u) >> 2, ((qAB & 0xFFFFu) + 2u) >> 2);
            out(xl + 1, ((pB & 0xFFFFu) + 2u) >> 2, ((pB >> 16) + 2u) >> 2, ((qAB >> 16) + 2u) >> 2);
        } else {
            // row sums of the quad per channel, then the block's other quads
            const uint32_t sr = __dp4a(w[0], 0x01000001u, __dp4a(w[1], 0x00010000u, __dp4a(w[2], 0x00000100u, 0u)));
            const uint32_t sg = __dp4a(w[0], 0x00000100u, __dp4a(w[1], 0x01000001u, __dp4a(w[2], 0x00010000u, 0u)));
            const uint32_t sb = __dp4a(w[0], 0x00010000u, __dp4a(w[1], 0x00000100u, __dp4a(w[2], 0x01000001u, 0u)));
            uint32_t rg = sr | (sg << 16), b = sb;   // each block sum <= 64 x 255 < 2^16
            if constexpr (S == 4) {
#pragma unroll
                for (int o = 8; o <= 16; o <<= 1) {
                    rg += __shfl_xor_sync(full, rg, o);
                    b += __shfl_xor_sync(full, b, o);
                }
            } else {
#pragma unroll
                for (int o = 1; o <= 8; o <<= 1) {
                    rg += __shfl_xor_sync(full, rg, o);
                    b += __shfl_xor_sync(full, b, o);
                }
            }
            constexpr uint32_t kHalf = S * S / 2, kShift = S == 4 ? 4 : 6;
            const bool lead = S == 4 ? r == 0 : (lane & 15) == 0;
            if (!lead || !inside)
                return;
            out(xl, ((rg & 0xFFFFu) + kHalf) >> kShift, ((rg >> 16) + kHalf) >> kShift, (b + kHalf) >> kShift);
        }
    };
    means(w, put);
    if (PAIR)   // the second frame: its grey only
        means(w2, [&](int x, uint32_t R, uint32_t G, uint32_t B) {
            a.low_gray2[(size_t)yl * a.low_gray2_pitch + x] = (uint8_t)((77u * R + 150u * G + 29u * B + 128u) >> 8);
        });
}

}  // namespace
}  // namespace vs

namespace vs {
namespace {

// The arguments of one frame's remap after the checks of vs_rectify_remap;
// *sq tells whether the block kernel k_remap_sq serves them.
int remap_args(const uint8_t *src, int W, int H, int src_pitch, const vs_camera *cam, const float *R9, uint8_t *dst,
               int dst_pitch, int scale, uint8_t *low_rgb, int low_rgb_pitch, uint8_t *low_gray, int low_gray_pitch,
               RemapArgs &a, bool &sq)
{
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

    a = RemapArgs{};
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
    // the block kernel: scale 2, 4 or 8, whole s x s blocks and 4-pixel
    // quads, word-aligned rows both ways, no rotation, 32-bit source offsets,
    // and the low-res output wanted
    sq = want_low && (s == 2 || s == 4 || s == 8) && !a.has_R && W % 4 == 0 && W % s == 0 && H % s == 0 &&
         W < (1 << 22) && H < (1 << 22) && a.src_words && (dst == nullptr || a.dst_vec) &&
         (long long)H * src_pitch < (1LL << 31);
    return VS_OK;
}

template <bool PAIR>
void launch_remap_sq(const RemapArgs &a, cudaStream_t st)
{
    dim3 grid((a.W + 63) / 64, (a.H + 15) / 16);
    if (a.s == 2)
        launch_pdl(k_remap_sq<2, PAIR>, dim3(grid), dim3(256), st, a);
    else if (a.s == 4)
        launch_pdl(k_remap_sq<4, PAIR>, dim3(grid), dim3(256), st, a);
    else
        launch_pdl(k_remap_sq<8, PAIR>, dim3(grid), dim3(256), st, a);
}

}  // namespace

// Both frames of a pair in one launch of the block kernel: the lens model of
// each destination quad once, the left frame sampled with the outputs of
// vs_rectify_remap, the right frame's low-res grey beside it.  Returns
// VS_EINVAL where the block kernel does not apply (the caller then remaps
// the frames one at a time).
int remap_pair(const uint8_t *left, const uint8_t *right, int W, int H, int pitch, const vs_camera *cam, int scale,
               uint8_t *dst, int dst_pitch, uint8_t *low_rgb, int low_rgb_pitch, uint8_t *gray_l, uint8_t *gray_r,
               int gray_pitch, cudaStream_t st)
{
    RemapArgs a;
    bool sq = false;
    int rc = remap_args(left, W, H, pitch, cam, nullptr, dst, dst_pitch, scale, low_rgb, low_rgb_pitch, gray_l,
                        gray_pitch, a, sq);
    if (rc != VS_OK || !sq || !right || !gray_r || !aligned(right, 4))
        return VS_EINVAL;
    a.src2 = right;
    a.src2_pitch = pitch;
    a.low_gray2 = gray_r;
    a.low_gray2_pitch = gray_pitch;
    const int slot = prof_begin(kProfRemap, st);
    launch_remap_sq<true>(a, st);
    prof_end(slot, st);
    note_launch();
    return launch_status();
}

}  // namespace vs

extern "C" int vs_rectify_remap(const uint8_t *src, int W, int H, int src_pitch,
                                const vs_camera *cam, const float *R9,
                                uint8_t *dst, int dst_pitch, int scale,
                                uint8_t *low_rgb, int low_rgb_pitch,
                                uint8_t *low_gray, int low_gray_pitch, void *stream)
{
    vs::NvtxRange nvtx_range("vs_rectify_remap");
    using namespace vs;
    RemapArgs a;
    bool sq = false;
    const int rc = remap_args(src, W, H, src_pitch, cam, R9, dst, dst_pitch, scale, low_rgb, low_rgb_pitch, low_gray,
                              low_gray_pitch, a, sq);
    if (rc != VS_OK)
        return rc;
    const int slot = prof_begin(kProfRemap, (cudaStream_t)stream);
    if (sq) {
        launch_remap_sq<false>(a, (cudaStream_t)stream);
    } else {
        const int tfw = a.tlw * a.s, tfh = a.tlh * a.s;
        dim3 grid((W + tfw - 1) / tfw, (H + tfh - 1) / tfh);
        launch_pdl(k_remap_down, dim3(grid), dim3(kRemapThreads), (cudaStream_t)stream, a);
    }
    prof_end(slot, (cudaStream_t)stream);
    note_launch();
    return launch_status();
}
