// Eq. 2 joint bilateral upsampling, optionally fused with the Eq. 3
// reprojection, and the stand-alone Eq. 3 kernel.
//
// A CTA covers a 64 x 8 tile of full-resolution pixels.  It stages the
// low-resolution labels and guide colours that the tile's windows can touch
// in shared memory (one uchar4 R,G,B,label per low-res pixel), then every
// thread evaluates the (2r+1)^2 window of its pixels from shared memory.
// Weights are taken relative to the tap with the smallest exponent: the
// exponent differences are formed from exact squared distances before they
// are scaled, so the weights that matter carry only a few ulp of error, and
// the normaliser is >= 1.
#include "vs_common.cuh"

#include <math.h>

namespace vs {
namespace {

constexpr int kTileW = 64, kTileH = 8;   // full-res pixels per CTA
constexpr int kThreadsY = 4;             // block = 64 x 4, two rows per thread
constexpr int kMaxR = 3;
constexpr int kStageW = kTileW + 2 * kMaxR + 1;
constexpr int kStageH = kTileH + 2 * kMaxR + 1;

struct JbuArgs {
    const uint8_t *labels, *guide_low, *guide_full;
    int labels_pitch, guide_low_pitch, guide_full_pitch;
    int w, h, W, H, s, r;
    float a_s;       // log2(e) / (2 sigma_s^2)
    float a_r;       // log2(e) / (2 sigma_r^2)
    float *disp, *xyz;
    float fx, cx, cy, fx_over_fy, baseline;
    // scales 2, 4, 8: the spatial exponent of tap t (window radius <= 3, up
    // to 49 taps) for the pixel at (px, py) of its s x s block,
    // (|p-q|^2 - |p-c|^2) a_s, at [(s py + px) 49 + t]; in the kernel
    // parameters, so each tap's multiply-add reads it from the constant bank
    float sp_as[64 * 49];
};

__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <bool kXYZ>
__global__ void __launch_bounds__(kTileW *kThreadsY) k_jbu(JbuArgs a)
{
    pdl_begin();
    __shared__ uchar4 stage[kStageH][kStageW];
    const int X0 = blockIdx.x * kTileW, Y0 = blockIdx.y * kTileH;
    // window centres of this tile: floor((x + 0.5) / s) = (2x + 1) / (2s)
    const int cx_lo = (2 * X0 + 1) / (2 * a.s), cy_lo = (2 * Y0 + 1) / (2 * a.s);
    const int qx0 = cx_lo - a.r, qy0 = cy_lo - a.r;
    const int sw = min(kStageW, (2 * min(X0 + kTileW - 1, a.W - 1) + 1) / (2 * a.s) + a.r - qx0 + 1);
    const int sh = min(kStageH, (2 * min(Y0 + kTileH - 1, a.H - 1) + 1) / (2 * a.s) + a.r - qy0 + 1);
    const int tid = threadIdx.y * kTileW + threadIdx.x;
    for (int i = tid; i < sw * sh; i += kTileW * kThreadsY) {
        const int sx = i % sw, sy = i / sw;
        const int qx = qx0 + sx, qy = qy0 + sy;
        uchar4 v = make_uchar4(0, 0, 0, 0);
        if (qx >= 0 && qy >= 0 && qx < a.w && qy < a.h) {
            const uint8_t *g = a.guide_low + (size_t)qy * a.guide_low_pitch + (size_t)qx * 3;
            v = make_uchar4(g[0], g[1], g[2], a.labels[(size_t)qy * a.labels_pitch + qx]);
        }
        stage[sy][sx] = v;
    }
    __syncthreads();

    const int x = X0 + threadIdx.x;
    if (x >= a.W)
        return;
    const float inv_s = 1.0f / (float)a.s;
    const float pxd = ((float)x + 0.5f) * inv_s - 0.5f;
    const int cxq = (2 * x + 1) / (2 * a.s);
    const int qxa = max(cxq - a.r, 0), qxb = min(cxq + a.r, a.w - 1);
#pragma unroll
    for (int rr = 0; rr < kTileH / kThreadsY; ++rr) {
        const int y = Y0 + threadIdx.y + rr * kThreadsY;
        if (y >= a.H)
            break;
        const float pyd = ((float)y + 0.5f) * inv_s - 0.5f;
        const int cyq = (2 * y + 1) / (2 * a.s);
        const int qya = max(cyq - a.r, 0), qyb = min(cyq + a.r, a.h - 1);
        const uint8_t *gp = a.guide_full + (size_t)y * a.guide_full_pitch + (size_t)x * 3;
        const int R = gp[0], Gc = gp[1], B = gp[2];
        // pass 1: the tap with the smallest exponent
        float kmin = INFINITY, ds_m = 0.0f;
        int dr_m = 0;
        for (int qy = qya; qy <= qyb; ++qy) {
            const float dy = pyd - (float)qy;
            for (int qx = qxa; qx <= qxb; ++qx) {
                const uchar4 q = stage[qy - qy0][qx - qx0];
                const float dx = pxd - (float)qx;
                const float ds = fmaf(dx, dx, dy * dy);
                const int dR = R - q.x, dG = Gc - q.y, dB = B - q.z;
                const int dr = dR * dR + dG * dG + dB * dB;
                const float k = fmaf(exact_float(dr), a.a_r, ds * a.a_s);
                if (k < kmin) {
                    kmin = k;
                    ds_m = ds;
                    dr_m = dr;
                }
            }
        }
        // pass 2: weights 2^-(k - k_min) from exact differences
        float num = 0.0f, den = 0.0f;
        for (int qy = qya; qy <= qyb; ++qy) {
            const float dy = pyd - (float)qy;
            for (int qx = qxa; qx <= qxb; ++qx) {
                const uchar4 q = stage[qy - qy0][qx - qx0];
                const float dx = pxd - (float)qx;
                const float ds = fmaf(dx, dx, dy * dy);
                const int dR = R - q.x, dG = Gc - q.y, dB = B - q.z;
                const int dr = dR * dR + dG * dG + dB * dB;
                // explicit fmaf: every instantiation rounds the same way
                const float e = fmaf(exact_float(dr) - exact_float(dr_m), a.a_r, (ds - ds_m) * a.a_s);
                const float wgt = ex2(-e);
                num = fmaf(wgt, (float)q.w, num);
                den += wgt;
            }
        }
        const float D = (float)a.s * num / den;
        const size_t p = (size_t)y * a.W + x;
        if (a.disp)
            a.disp[p] = D;
        if (kXYZ) {
            float X = __int_as_float(0x7fc00000), Y = X, Z = X;
            if (D > 0.0f) {
                const float bd = a.baseline / D;
                X = ((float)x - a.cx) * bd;
                Y = ((float)y - a.cy) * a.fx_over_fy * bd;
                Z = a.fx * bd;
            }
            a.xyz[3 * p + 0] = X;
            a.xyz[3 * p + 1] = Y;
            a.xyz[3 * p + 2] = Z;
        }
    }
}

// ---------------------------------------------------------------------------
// scales 2, 4 and 8: one thread per low-res window centre
//
// With s = S the S x S full-res pixels x = S k .. S k + S - 1, y = S l ..
// S l + S - 1 all have the window centre (k, l), so one thread loads the
// (2R+1)^2 taps once into registers and evaluates all S^2 pixels, a row of S
// at a time.  For a tap q and pixel p:
//   |I_p - I_q|^2 = |I_p|^2 + (|I_q|^2 - 2 I_p.I_q)
// where I_p.I_q is one dp4a; the |I_p|^2 term is the same for every tap of
// p and cancels against the reference tap, so only v_q = |I_q|^2 - 2 I_p.I_q
// is formed.  The reference tap is the one with the smallest v_q; the
// spatial offsets relative to the window centre (the nearest tap) are
// constants of the pixel's position in its S x S block (kernel parameters),
// so
//   exponent = (v_q - v_min) * a_r + (|p-q|^2 - |p-c|^2) * a_s >= 0
// and the window always holds a tap of weight >= 2^-(spatial spread); the
// host takes this kernel only while that spread is <= 100, so the
// normaliser stays a normal float.
// v_q is formed directly as the bit pattern of the float 2^23 + kVBias + v_q
// (|v_q| <= 2 * 195075 = kVBias keeps it in [2^23, 2^24), where floats are
// the integers), so v_q - v_min is one exact float subtraction instead of an
// integer-to-float conversion (a quarter-rate operation).  Taps outside the
// low-res frame are staged with the pattern of 2^127 (and colour 0), whose
// exponent is >= 2^127 a_r >= 2^27 with a_r >= 2^-100: weight exactly 0,
// skipped as in the definition.

constexpr int kS4CentresX = 32, kS4CentresY = 4;   // window centres per CTA
constexpr uint32_t kVBias = 2u * 195075u;            // 2 * 3 * 255^2
constexpr uint32_t kVMagic = 0x4B000000u + kVBias;   // float bits of 2^23 + kVBias
constexpr uint32_t kOffFrameBits = 0x7F000000u;      // float bits of 2^127
constexpr float kMinAr = 0x1p-100f;                  // floor of a_r on this path

// The S pixels of row y from full-res column S k on, as 24-bit RGB words.
// Rows start on 4-byte boundaries (checked on the host): for S = 4 and 8 the
// 3 S bytes are whole words; for S = 2 they are three 16-bit halves.
template <int S>
__device__ __forceinline__ void guide_pixels(const JbuArgs &a, int y, int k, uint32_t (&ip)[S])
{
    const uint8_t *row = a.guide_full + (size_t)y * a.guide_full_pitch;
    if constexpr (S == 2) {
        const uint16_t *h = reinterpret_cast<const uint16_t *>(row + (size_t)k * 6);
        const uint32_t h0 = h[0], h1 = h[1], h2 = h[2];
        ip[0] = h0 | ((h1 & 0xFFu) << 16);
        ip[1] = (h1 >> 8) | (h2 << 8);
    } else {
        constexpr int NW = 3 * S / 4;
        const uint32_t *g = reinterpret_cast<const uint32_t *>(row + (size_t)k * 3 * S);
        uint32_t w[NW + 1];
#pragma unroll
        for (int i = 0; i < NW; ++i)
            w[i] = g[i];
        w[NW] = 0u;
#pragma unroll
        for (int q = 0; q < S; ++q)   // pixel q: bytes 3q .. 3q + 2
            ip[q] = __funnelshift_r(w[(3 * q) / 4], w[(3 * q) / 4 + 1], 8 * ((3 * q) % 4)) & 0xFFFFFFu;
    }
}

template <int S, int R, bool kXYZ>
__global__ void __launch_bounds__(kS4CentresX *kS4CentresY, 4) k_jbu_sq(JbuArgs a)
{
    pdl_begin();
    constexpr int D = 2 * R + 1;
    constexpr int SW = kS4CentresX + 2 * R, SH = kS4CentresY + 2 * R;
    // (R | G<<8 | B<<16 | label<<24, bits of 2^23 + kVBias + R^2+G^2+B^2)
    __shared__ uint2 stage[SH][SW];
    const int k0 = blockIdx.x * kS4CentresX, l0 = blockIdx.y * kS4CentresY;
    for (int i = threadIdx.x; i < SW * SH; i += kS4CentresX * kS4CentresY) {
        const int sx = i % SW, sy = i / SW;
        const int qx = k0 - R + sx, qy = l0 - R + sy;
        uint2 v = make_uint2(0u, kOffFrameBits);
        if (qx >= 0 && qy >= 0 && qx < a.w && qy < a.h) {
            const uint8_t *g = a.guide_low + (size_t)qy * a.guide_low_pitch + (size_t)qx * 3;
            const uint32_t r = g[0], gg = g[1], b = g[2];
            const uint32_t lab = a.labels[(size_t)qy * a.labels_pitch + qx];
            v = make_uint2(r | (gg << 8) | (b << 16) | (lab << 24), kVMagic + r * r + gg * gg + b * b);
        }
        stage[sy][sx] = v;
    }
    __syncthreads();

    const int kx = threadIdx.x % kS4CentresX, ly = threadIdx.x / kS4CentresX;
    const int k = k0 + kx, l = l0 + ly;
    if (k >= a.w || l >= a.h)
        return;
    uint32_t tq[D * D];
    int tn[D * D];
    float tl[D * D];
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const uint2 v = stage[ly + j][kx + i];
            tq[j * D + i] = v.x;     // byte 3 (label) meets a zero byte of I_p in dp4a
            tn[j * D + i] = (int)v.y;
            tl[j * D + i] = (float)(v.x >> 24);
        }

    // the rows unrolled at S = 2 (each tap's spatial term then is a
    // constant-bank operand of its multiply-add); from S = 4 on a loop (one
    // constant load per tap), whose smaller code measured faster: 39.6
    // against 44.0 us per 2.7K launch at S = 4, where the unrolled 16 pixels
    // x 25 taps stalled on instruction fetch
#pragma unroll(S <= 2 ? S : 1)
    for (int py = 0; py < S; ++py) {
        const int y = S * l + py;
        if (y >= a.H)   // the last block row of a frame whose height is not a multiple of S
            break;
        uint32_t ip[S];
        guide_pixels<S>(a, y, k, ip);
        float dres[S];
#pragma unroll
        for (int px = 0; px < S; ++px) {
            int v[D * D];   // float bits of 2^23 + kVBias + v_q (2^127 off the frame)
            int vmin = 0x7FFFFFFF;
#pragma unroll
            for (int t = 0; t < D * D; ++t) {
                v[t] = tn[t] - 2 * (int)__dp4a(ip[px], tq[t], 0u);
                vmin = min(vmin, v[t]);
            }
            const float fmin = __int_as_float(vmin);
            float num = 0.0f, den = 0.0f;
            // spatial terms: p_down - q = ((px + 0.5)/S - 0.5 - i, (py + 0.5)/S - 0.5 - j)
#pragma unroll
            for (int t = 0; t < D * D; ++t) {
                const float e = fmaf(__int_as_float(v[t]) - fmin, a.a_r, a.sp_as[(S * py + px) * 49 + t]);
                const float wgt = ex2(-e);
                num = fmaf(wgt, tl[t], num);
                den += wgt;
            }
            // den >= 2^-100 (the reference tap) and <= 49: the fast reciprocal
            // division is within 2 ulp here
            dres[px] = __fdividef((float)S * num, den);
        }
        const size_t p = (size_t)y * a.W + (size_t)S * k;
        if (a.disp) {
            if constexpr (S == 2) {
                *reinterpret_cast<float2 *>(a.disp + p) = make_float2(dres[0], dres[1]);
            } else {
#pragma unroll
                for (int q = 0; q < S; q += 4)
                    *reinterpret_cast<float4 *>(a.disp + p + q) = make_float4(dres[q], dres[q + 1], dres[q + 2], dres[q + 3]);
            }
        }
        if (kXYZ) {
            float o[3 * S];
#pragma unroll
            for (int px = 0; px < S; ++px) {
                float X = __int_as_float(0x7fc00000), Y = X, Z = X;
                if (dres[px] > 0.0f) {
                    const float bd = __fdividef(a.baseline, dres[px]);   // dres <= S * 255
                    X = ((float)(S * k + px) - a.cx) * bd;
                    Y = ((float)y - a.cy) * a.fx_over_fy * bd;
                    Z = a.fx * bd;
                }
                o[3 * px] = X;
                o[3 * px + 1] = Y;
                o[3 * px + 2] = Z;
            }
            if constexpr (S == 2) {
                float2 *dst = reinterpret_cast<float2 *>(a.xyz + 3 * p);
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    dst[q] = make_float2(o[2 * q], o[2 * q + 1]);
            } else {
                float4 *dst = reinterpret_cast<float4 *>(a.xyz + 3 * p);
#pragma unroll
                for (int q = 0; q < 3 * S / 4; ++q)
                    dst[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
            }
        }
    }
}

template <int S, bool kXYZ>
void launch_jbu_sq(const JbuArgs &a, cudaStream_t st)
{
    dim3 grid((a.w + kS4CentresX - 1) / kS4CentresX, (a.h + kS4CentresY - 1) / kS4CentresY);
    const int block = kS4CentresX * kS4CentresY;
    switch (a.r) {
    case 0: launch_pdl(k_jbu_sq<S, 0, kXYZ>, dim3(grid), dim3(block), st, a); break;
    case 1: launch_pdl(k_jbu_sq<S, 1, kXYZ>, dim3(grid), dim3(block), st, a); break;
    case 2: launch_pdl(k_jbu_sq<S, 2, kXYZ>, dim3(grid), dim3(block), st, a); break;
    default: launch_pdl(k_jbu_sq<S, 3, kXYZ>, dim3(grid), dim3(block), st, a); break;
    }
}

template <bool kXYZ>
void launch_jbu_scaled(const JbuArgs &a, cudaStream_t st)
{
    if (a.s == 2)
        launch_jbu_sq<2, kXYZ>(a, st);
    else if (a.s == 4)
        launch_jbu_sq<4, kXYZ>(a, st);
    else
        launch_jbu_sq<8, kXYZ>(a, st);
}

struct ReprojArgs {
    const float *disp;
    float *xyz;
    int W, H;
    float fx, cx, cy, fx_over_fy, baseline;
};

__global__ void k_reproject(ReprojArgs a)
{
    pdl_begin();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)a.W * a.H)
        return;
    const int u = (int)(p % a.W), v = (int)(p / a.W);
    const float D = a.disp[p];
    float X = __int_as_float(0x7fc00000), Y = X, Z = X;
    if (D > 0.0f) {
        const float bd = a.baseline / D;
        X = ((float)u - a.cx) * bd;
        Y = ((float)v - a.cy) * a.fx_over_fy * bd;
        Z = a.fx * bd;
    }
    a.xyz[3 * p + 0] = X;
    a.xyz[3 * p + 1] = Y;
    a.xyz[3 * p + 2] = Z;
}

bool cam_ok(const vs_camera *cam)
{
    if (!cam)
        return false;
    const float v[4] = {cam->fx, cam->fy, cam->cx, cam->cy};
    for (float f : v)
        if (!isfinite(f))
            return false;
    return cam->fx != 0.0f && cam->fy != 0.0f;
}

int jbu_common(const uint8_t *labels, int w, int h, int labels_pitch, const uint8_t *guide_low,
               int guide_low_pitch, const uint8_t *guide_full, int W, int H, int guide_full_pitch,
               const vs_jbu_params *jp, const vs_camera *cam, float baseline, float *disp, float *xyz,
               cudaStream_t st)
{
    if (!labels || !guide_low || !guide_full || !jp || w <= 0 || h <= 0 || W <= 0 || H <= 0)
        return VS_EINVAL;
    if (jp->scale < 1 || jp->scale > 16 || jp->radius < 0 || jp->radius > kMaxR)
        return VS_EINVAL;
    if (!(jp->sigma_s > 0.0f) || !(jp->sigma_r > 0.0f) || !isfinite(jp->sigma_s) || !isfinite(jp->sigma_r))
        return VS_EINVAL;
    const int s = jp->scale;
    if (w != (W + s - 1) / s || h != (H + s - 1) / s)
        return VS_EINVAL;
    if (labels_pitch < w || guide_low_pitch < 3 * w || guide_full_pitch < 3 * W)
        return VS_EINVAL;
    if (!disp && !xyz)
        return VS_EINVAL;
    if (xyz && (!cam_ok(cam) || !(baseline > 0.0f) || !isfinite(baseline)))
        return VS_EINVAL;
    JbuArgs a;
    a.labels = labels;
    a.guide_low = guide_low;
    a.guide_full = guide_full;
    a.labels_pitch = labels_pitch;
    a.guide_low_pitch = guide_low_pitch;
    a.guide_full_pitch = guide_full_pitch;
    a.w = w;
    a.h = h;
    a.W = W;
    a.H = H;
    a.s = s;
    a.r = jp->radius;
    const double log2e = 1.4426950408889634;
    a.a_s = (float)(log2e / (2.0 * (double)jp->sigma_s * (double)jp->sigma_s));
    a.a_r = (float)(log2e / (2.0 * (double)jp->sigma_r * (double)jp->sigma_r));
    a.disp = disp;
    a.xyz = xyz;
    a.fx = cam ? cam->fx : 0.0f;
    a.cx = cam ? cam->cx : 0.0f;
    a.cy = cam ? cam->cy : 0.0f;
    a.fx_over_fy = cam ? cam->fx / cam->fy : 0.0f;
    a.baseline = baseline;
    // spatial exponents of the scale-2/4/8 windows: p_down - q = (ox - (i - r), oy - (j - r)),
    // (ox, oy) = ((px + 0.5) / s - 0.5, (py + 0.5) / s - 0.5); the squared distances are
    // exact in FP32 (s is a power of two) and the product with a_s rounds as it would on
    // the device
    for (int k = 0; k < 64 * 49; ++k)
        a.sp_as[k] = 0.0f;
    const bool sq_scale = s == 2 || s == 4 || s == 8;
    float sp_spread = 0.0f;   // largest spatial exponent of a window
    if (sq_scale && a.r <= 3) {
        const int D = 2 * a.r + 1;
        const float inv_s = 1.0f / (float)s;
        for (int py = 0; py < s; ++py)
            for (int px = 0; px < s; ++px)
                for (int j = 0; j < D; ++j)
                    for (int i = 0; i < D; ++i) {
                        const float ox = (px + 0.5f) * inv_s - 0.5f, oy = (py + 0.5f) * inv_s - 0.5f;
                        const float dx = ox - (float)(i - a.r), dy = oy - (float)(j - a.r);
                        const float sp = (dx * dx + dy * dy) - (ox * ox + oy * oy);
                        a.sp_as[(s * py + px) * 49 + j * D + i] = sp * a.a_s;
                        sp_spread = fmaxf(sp_spread, sp * a.a_s);
                    }
    }
    dim3 grid((W + kTileW - 1) / kTileW, (H + kTileH - 1) / kTileH);
    dim3 block(kTileW, kThreadsY);
    // the block kernels need whole s-pixel groups on every row, 4-byte aligned
    // guide rows for their word loads, 16-byte aligned outputs for their
    // vector stores, and a spatial spread that keeps the reference tap's
    // weight >= 2^-100
    const bool sq = sq_scale && W % s == 0 && guide_full_pitch % 4 == 0 && aligned(guide_full, 4) &&
                    (!disp || aligned(disp, 16)) && (!xyz || aligned(xyz, 16)) && sp_spread <= 100.0f;
    const int slot = prof_begin(kProfJbu, st);
    if (sq) {
        // a_r below 2^-100 makes every in-frame range term < 2^-80, which
        // changes no weight; the floor keeps off-frame taps at weight 0
        a.a_r = fmaxf(a.a_r, kMinAr);
        if (xyz)
            launch_jbu_scaled<true>(a, st);
        else
            launch_jbu_scaled<false>(a, st);
    } else if (xyz) {
        launch_pdl(k_jbu<true>, dim3(grid), dim3(block), st, a);
    } else {
        launch_pdl(k_jbu<false>, dim3(grid), dim3(block), st, a);
    }
    prof_end(slot, st);
    note_launch();
    return launch_status();
}

}  // namespace
}  // namespace vs

extern "C" int vs_guided_upsample(const uint8_t *labels, int w, int h, int labels_pitch,
                                  const uint8_t *guide_low, int guide_low_pitch,
                                  const uint8_t *guide_full, int W, int H, int guide_full_pitch,
                                  const vs_jbu_params *jp, float *disp, void *stream)
{
    vs::NvtxRange nvtx_range("vs_guided_upsample");
    if (!disp)
        return VS_EINVAL;
    return vs::jbu_common(labels, w, h, labels_pitch, guide_low, guide_low_pitch, guide_full, W, H,
                          guide_full_pitch, jp, nullptr, 0.0f, disp, nullptr, (cudaStream_t)stream);
}

extern "C" int vs_guided_upsample_reproject(const uint8_t *labels, int w, int h, int labels_pitch,
                                            const uint8_t *guide_low, int guide_low_pitch,
                                            const uint8_t *guide_full, int W, int H, int guide_full_pitch,
                                            const vs_jbu_params *jp, const vs_camera *cam, float baseline,
                                            float *disp, float *xyz, void *stream)
{
    vs::NvtxRange nvtx_range("vs_guided_upsample_reproject");
    if (!xyz)
        return VS_EINVAL;
    return vs::jbu_common(labels, w, h, labels_pitch, guide_low, guide_low_pitch, guide_full, W, H,
                          guide_full_pitch, jp, cam, baseline, disp, xyz, (cudaStream_t)stream);
}

extern "C" int vs_reproject(const float *disp, int W, int H, const vs_camera *cam, float baseline,
                            float *xyz, void *stream)
{
    vs::NvtxRange nvtx_range("vs_reproject");
    using namespace vs;
    if (!disp || !xyz || W <= 0 || H <= 0 || !cam_ok(cam) || !(baseline > 0.0f) || !isfinite(baseline))
        return VS_EINVAL;
    ReprojArgs a{disp, xyz, W, H, cam->fx, cam->cx, cam->cy, cam->fx / cam->fy, baseline};
    const long long n = (long long)W * H;
    launch_pdl(k_reproject, dim3((unsigned)((n + 255) / 256)), dim3(256), (cudaStream_t)stream, a);
    note_launch();
    return launch_status();
}
