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
                const float ds = dx * dx + dy * dy;
                const int dR = R - q.x, dG = Gc - q.y, dB = B - q.z;
                const int dr = dR * dR + dG * dG + dB * dB;
                const float k = ds * a.a_s + (float)dr * a.a_r;
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
                const float ds = dx * dx + dy * dy;
                const int dR = R - q.x, dG = Gc - q.y, dB = B - q.z;
                const int dr = dR * dR + dG * dG + dB * dB;
                const float e = (ds - ds_m) * a.a_s + (float)(dr - dr_m) * a.a_r;
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

struct ReprojArgs {
    const float *disp;
    float *xyz;
    int W, H;
    float fx, cx, cy, fx_over_fy, baseline;
};

__global__ void k_reproject(ReprojArgs a)
{
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
    dim3 grid((W + kTileW - 1) / kTileW, (H + kTileH - 1) / kTileH);
    dim3 block(kTileW, kThreadsY);
    const int slot = prof_begin(kProfJbu, st);
    if (xyz)
        k_jbu<true><<<grid, block, 0, st>>>(a);
    else
        k_jbu<false><<<grid, block, 0, st>>>(a);
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
    if (!xyz)
        return VS_EINVAL;
    return vs::jbu_common(labels, w, h, labels_pitch, guide_low, guide_low_pitch, guide_full, W, H,
                          guide_full_pitch, jp, cam, baseline, disp, xyz, (cudaStream_t)stream);
}

extern "C" int vs_reproject(const float *disp, int W, int H, const vs_camera *cam, float baseline,
                            float *xyz, void *stream)
{
    using namespace vs;
    if (!disp || !xyz || W <= 0 || H <= 0 || !cam_ok(cam) || !(baseline > 0.0f) || !isfinite(baseline))
        return VS_EINVAL;
    ReprojArgs a{disp, xyz, W, H, cam->fx, cam->cx, cam->cy, cam->fx / cam->fy, baseline};
    const long long n = (long long)W * H;
    k_reproject<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(a);
    note_launch();
    return launch_status();
}
