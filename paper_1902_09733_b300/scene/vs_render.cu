// CUDA ray-caster of the synthetic flight scenes: input generation for tests
// and benchmarks only (the stereo library never calls it).  It draws what the
// host renderer of paper_1902_09733_b300/synth.py draws -- a nadir pinhole
// camera with radial distortion over a tabulated heightfield with box
// buildings and a colour value-noise albedo -- with the same operations in
// the same order and precision: the lens inverted in FP64 by fixed-point
// iteration, ray positions and the march parameter in FP32, interpolation
// weights, heights, albedo and shading in FP64 (where the host's mixed
// float32 / integer arithmetic promotes to double).  The file is compiled
// without fused multiply-adds, so every operation rounds as on the host.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kMaxOctaves = 4;

struct Octave {
    float lam, hi;        // wavelength (m), largest lattice coordinate (m - 2.001)
    double amp;           // amplitude
    int m;                // lattice side
    const float *lat;     // m x m x 3
};

struct RenderArgs {
    const float *height;  // n x n heights (m)
    int n;
    float half, res, hhi; // half extent, cell size, largest grid coordinate (n - 1.001)
    Octave oct[kMaxOctaves];
    int noct;
    float nhalf;          // half extent of the noise lattices
    double top;           // highest surface: the march starts just above it
    double altitude;
    float t0, step, alt32;
    double fx, fy, cx, cy, k1, k2;
    float px, py, cosy, siny;
    int rotate;
    int march_steps, refine_steps;
    uint8_t *out;
    float *depth;         // nullable: the z-depth of each pixel along its undistorted ray
    int W, H;
};

// Bilinear height at ground point (X, Y): the grid coordinates in FP32, the
// weights and the blend in FP64.
__device__ double height_at(const RenderArgs &a, float X, float Y)
{
    float gx = (X + a.half) / a.res;
    float gy = (Y + a.half) / a.res;
    gx = fminf(fmaxf(gx, 0.0f), a.hhi);
    gy = fminf(fmaxf(gy, 0.0f), a.hhi);
    const int ix = (int)gx, iy = (int)gy;
    const double fx = (double)gx - (double)ix, fy = (double)gy - (double)iy;
    const int base = iy * a.n + ix;
    const float v00 = a.height[base], v10 = a.height[base + 1];
    const float v01 = a.height[base + a.n], v11 = a.height[base + a.n + 1];
    const double d0 = (double)(v10 - v00), d1 = (double)(v11 - v01);
    return ((double)v00 + fx * d0) * (1.0 - fy) + ((double)v01 + fx * d1) * fy;
}

// Colour value noise at (X, Y): smoothstep-interpolated lattice octaves.
__device__ void albedo_at(const RenderArgs &a, float X, float Y, double (&col)[3])
{
    for (int o = 0; o < a.noct; ++o) {
        const Octave &q = a.oct[o];
        float gx = (X + a.nhalf) / q.lam;
        float gy = (Y + a.nhalf) / q.lam;
        gx = fminf(fmaxf(gx, 0.0f), q.hi);
        gy = fminf(fmaxf(gy, 0.0f), q.hi);
        const int ix = (int)gx, iy = (int)gy;
        const double fx = (double)gx - (double)ix, fy = (double)gy - (double)iy;
        const double sx = fx * fx * (3.0 - 2.0 * fx);
        const double sy = fy * fy * (3.0 - 2.0 * fy);
        const float *l00 = q.lat + ((size_t)iy * q.m + ix) * 3;
        const float *l10 = l00 + 3, *l01 = l00 + (size_t)q.m * 3, *l11 = l01 + 3;
        for (int c = 0; c < 3; ++c) {
            const double v = ((double)l00[c] * (1.0 - sx) + (double)l10[c] * sx) * (1.0 - sy) +
                             ((double)l01[c] * (1.0 - sx) + (double)l11[c] * sx) * sy;
            const double av = q.amp * v;
            col[c] = o == 0 ? av : col[c] + av;
        }
    }
}

__global__ void __launch_bounds__(256) k_render(RenderArgs a)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    if (u >= a.W || v >= a.H)
        return;
    // the ideal ray of this distorted pixel
    const double xd = ((double)u - a.cx) / a.fx, yd = ((double)v - a.cy) / a.fy;
    double x = xd, y = yd;
    for (int i = 0; i < 8; ++i) {
        const double r2 = x * x + y * y;
        const double f = 1.0 + a.k1 * r2 + a.k2 * r2 * r2;
        x = xd / f;
        y = yd / f;
    }
    float xn = (float)x, yn = (float)y;
    if (a.rotate) {
        const float rx = a.cosy * xn - a.siny * yn;
        const float ry = a.siny * xn + a.cosy * yn;
        xn = rx;
        yn = ry;
    }
    auto gap = [&](float t) {   // >= 0 once the ray at depth t is at or below the surface
        const float X = a.px + t * xn, Y = a.py + t * yn;
        return (double)t - (a.altitude - height_at(a, X, Y));
    };
    float t_lo = a.t0, t_hi = a.alt32;
    for (int i = 1; i <= a.march_steps; ++i) {
        const float t = a.t0 + (float)i * a.step;
        if (gap(t) >= 0.0) {
            t_hi = t;
            t_lo = t - a.step;
            break;
        }
    }
    for (int i = 0; i < a.refine_steps; ++i) {
        const float tm = 0.5f * (t_lo + t_hi);
        if (gap(tm) >= 0.0)
            t_hi = tm;
        else
            t_lo = tm;
    }
    const float t = 0.5f * (t_lo + t_hi);
    if (a.depth)
        a.depth[(size_t)v * a.W + u] = t;
    const float X = a.px + t * xn, Y = a.py + t * yn;
    double col[3];
    albedo_at(a, X, Y, col);
    double hs = height_at(a, X, Y) / a.top;
    hs = fmin(fmax(hs, 0.0), 1.0);
    const double shade = 0.75 + 0.25 * hs;
    uint8_t *o = a.out + ((size_t)v * a.W + u) * 3;
    for (int c = 0; c < 3; ++c) {
        double rgb = 128.0 + 110.0 * col[c] * shade;
        rgb = fmin(fmax(rgb, 0.0), 255.0);
        o[c] = (uint8_t)rint(rgb);
    }
}

}  // namespace

extern "C" {

// One W x H RGB frame into `out` (device, W H 3 bytes) from camera pose
// (px, py) at `altitude` with heading given by its FP32 cosine and sine
// (rotate = 0: heading 0, the camera axes on the ground axes).  height: n x n
// device floats on a square of half extent `half` and cell `res`; octaves:
// `noct` (<= 4) device lattices of m x m x 3 floats with their wavelength and
// amplitude; cam6 = fx, fy, cx, cy, k1, k2; depth (nullable, device, W H
// floats) receives each pixel's z-depth.  Returns 0, -1 for bad arguments,
// or -4 for a CUDA error.
int vsr_render(const float *height, int n, float half, float res, int noct, const float *const *lat,
               const int *m, const float *lam, const double *amp, float nhalf, double top, double altitude,
               const double *cam6, float px, float py, int rotate, float cosy, float siny, uint8_t *out, int W,
               int H, float *depth, void *stream)
{
    if (!height || !out || !cam6 || n < 2 || noct < 1 || noct > kMaxOctaves || W <= 0 || H <= 0 || !(top > 0.0))
        return -1;
    RenderArgs a;
    a.height = height;
    a.n = n;
    a.half = half;
    a.res = res;
    a.hhi = (float)((double)n - 1.001);
    for (int o = 0; o < noct; ++o) {
        if (!lat[o] || m[o] < 2)
            return -1;
        a.oct[o].lam = lam[o];
        a.oct[o].amp = amp[o];
        a.oct[o].m = m[o];
        a.oct[o].hi = (float)((double)m[o] - 2.001);
        a.oct[o].lat = lat[o];
    }
    a.noct = noct;
    a.nhalf = nhalf;
    a.top = top;
    a.altitude = altitude;
    a.t0 = (float)(altitude - top - 1e-3);
    a.step = (float)((top + 1e-3) / 20.0);
    a.alt32 = (float)altitude;
    a.fx = cam6[0];
    a.fy = cam6[1];
    a.cx = cam6[2];
    a.cy = cam6[3];
    a.k1 = cam6[4];
    a.k2 = cam6[5];
    a.px = px;
    a.py = py;
    a.rotate = rotate;
    a.cosy = cosy;
    a.siny = siny;
    a.march_steps = 20;
    a.refine_steps = 12;
    a.out = out;
    a.depth = depth;
    a.W = W;
    a.H = H;
    k_render<<<dim3((W + 255) / 256, H), 256, 0, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

}  // extern "C"
