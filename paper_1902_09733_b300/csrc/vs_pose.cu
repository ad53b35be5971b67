// Pose path of Section 2.3 (Eq. 4-7): Harris corners, ZSSD matching, EPnP.
//
// k_harris_r25   Eq. 4 + Eq. 5 at every pixel: the integer luma of the RGB
//                frame, central differences A, B (frame edge repeated), the
//                products windowed by the 5 x 5 binomial [1 4 6 4 1]^T [1 4 6
//                4 1] (taps outside the frame skipped), 25 R = 25 det M -
//                tr(M)^2 (k = 0.04) -- exact int64, tiles staged in shared
//                memory, the window applied as two 1-D passes.
// k_harris_cells one CTA per cell of the grid (Section 3.2): the candidates
//                (inside the margin, 25 R above the threshold, beating each
//                of their 8 neighbours in (R, then the smaller raster index))
//                reduced to the cell's largest (R, smaller index).
// k_zssd         one CTA per corner: the patch and frame 2's search region
//                as packed luma in shared memory, one displacement per
//                thread at a time, n Z = n sum D^2 - (sum D)^2 exact in
//                integers from dp4a sums, the first smallest in raster order
//                of (dy, dx), then the parabola through the two neighbouring
//                costs on each axis (FP64).
// k_epnp         one CTA per problem (the left and right poses of a stereo
//                pair side by side), FP64: the points as weighted sums of four control
//                points (centroid and principal axes), the 12 x 12 normal
//                matrix of Eq. 6 (in normalised image coordinates: each
//                equation divided by fx or fy) and its four smallest
//                eigenvectors (cyclic Jacobi on three warps), the control
//                points' camera coordinates from N = 1, 2, 3 of them
//                (distance constraints, then Gauss-Newton on all four; one
//                warp each), [R, T] by orthogonal Procrustes (Eq. 7), the
//                best reprojection error; then up to twice more on the
//                points whose error is below max(2 px, 3 x the median).
// k_pose_average the poses of a later pair's left and right images (the
//                right one moved through the virtual rig) averaged: the
//                rotation nearest to their sum, the mean translation.
#include "vs_common.cuh"

#include <math.h>

#include <cmath>

namespace vs {
namespace {

constexpr int kHarrisTx = 32, kHarrisTy = 8;   // output tile
constexpr int kHalo = 3;                       // window 2 + derivative 1
constexpr int kMaxGrid = 64;
constexpr int kMaxRadius = 8, kMaxSearch = 32;
constexpr int kMaxPts = 4096;
constexpr int kEpnpThreads = 256;

__device__ __forceinline__ int luma(const uint8_t *p)
{
    return (77 * (int)p[0] + 150 * (int)p[1] + 29 * (int)p[2] + 128) >> 8;
}

// ---------------------------------------------------------------------------
// Harris

struct HarrisArgs {
    const uint8_t *rgb;
    int W, H, pitch;
    int64_t *r25;
};

__global__ void __launch_bounds__(kHarrisTx * kHarrisTy) k_harris_r25(HarrisArgs a)
{
    pdl_begin();
    constexpr int GW = kHarrisTx + 2 * kHalo, GH = kHarrisTy + 2 * kHalo;   // grey tile
    constexpr int PW = kHarrisTx + 4, PH = kHarrisTy + 4;                   // products (window halo 2)
    __shared__ int g[GH][GW];
    __shared__ int pxx[PH][PW], pyy[PH][PW], pxy[PH][PW];
    __shared__ int hxx[PH][kHarrisTx], hyy[PH][kHarrisTx], hxy[PH][kHarrisTx];
    const int x0 = blockIdx.x * kHarrisTx, y0 = blockIdx.y * kHarrisTy;
    const int tid = threadIdx.y * kHarrisTx + threadIdx.x, nt = kHarrisTx * kHarrisTy;
    // grey with the frame edge repeated (what the central differences read)
    for (int i = tid; i < GW * GH; i += nt) {
        const int ty = i / GW, tx = i - ty * GW;
        const int x = min(max(x0 - kHalo + tx, 0), a.W - 1), y = min(max(y0 - kHalo + ty, 0), a.H - 1);
        g[ty][tx] = luma(a.rgb + (size_t)y * a.pitch + 3 * (size_t)x);
    }
    __syncthreads();
    // products of the derivatives; 0 outside the frame (skipped window taps)
    for (int i = tid; i < PW * PH; i += nt) {
        const int ty = i / PW, tx = i - ty * PW;
        const int x = x0 - 2 + tx, y = y0 - 2 + ty;
        int A = 0, B = 0;
        if (x >= 0 && x < a.W && y >= 0 && y < a.H) {
            A = g[ty + 1][tx + 2] - g[ty + 1][tx];
            B = g[ty + 2][tx + 1] - g[ty][tx + 1];
        }
        pxx[ty][tx] = A * A;
        pyy[ty][tx] = B * B;
        pxy[ty][tx] = A * B;
    }
    __syncthreads();
    // window, horizontal pass
    const int b[5] = {1, 4, 6, 4, 1};
    for (int i = tid; i < PH * kHarrisTx; i += nt) {
        const int ty = i / kHarrisTx, tx = i - ty * kHarrisTx;
        int sxx = 0, syy = 0, sxy = 0;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            sxx += b[j] * pxx[ty][tx + j];
            syy += b[j] * pyy[ty][tx + j];
            sxy += b[j] * pxy[ty][tx + j];
        }
        hxx[ty][tx] = sxx;
        hyy[ty][tx] = syy;
        hxy[ty][tx] = sxy;
    }
    __syncthreads();
    // vertical pass and the response
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= a.W || y >= a.H)
        return;
    long long sxx = 0, syy = 0, sxy = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        sxx += b[i] * hxx[ty + i][tx];
        syy += b[i] * hyy[ty + i][tx];
        sxy += b[i] * hxy[ty + i][tx];
    }
    const long long tr = sxx + syy;
    a.r25[(size_t)y * a.W + x] = 25 * (sxx * syy - sxy * sxy) - tr * tr;
}

struct CellArgs {
    const int64_t *r25;
    int W, H, grid, margin;
    long long thr;
    int32_t *corners;   // grid^2 x 2
};

// (R, index) pairs: larger R wins, then the smaller index
__device__ __forceinline__ bool beats(long long ra, long long ia, long long rb, long long ib)
{
    return ra > rb || (ra == rb && ia < ib);
}

__global__ void __launch_bounds__(256) k_harris_cells(CellArgs a)
{
    pdl_begin();
    const int gx = blockIdx.x % a.grid, gy = blockIdx.x / a.grid;
    const int x0 = (int)((long long)gx * a.W / a.grid), x1 = (int)((long long)(gx + 1) * a.W / a.grid);
    const int y0 = (int)((long long)gy * a.H / a.grid), y1 = (int)((long long)(gy + 1) * a.H / a.grid);
    const int cw = x1 - x0, n = cw * (y1 - y0);
    long long best_r = LLONG_MIN, best_i = -1;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int y = y0 + k / cw, x = x0 + k % cw;
        if (x < a.margin || x >= a.W - a.margin || y < a.margin || y >= a.H - a.margin)
            continue;
        const long long r = a.r25[(size_t)y * a.W + x];
        if (r <= a.thr)
            continue;
        const long long idx = (long long)y * a.W + x;
        bool is_max = true;
        for (int dy = -1; dy <= 1 && is_max; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if ((dx == 0 && dy == 0) || x + dx < 0 || x + dx >= a.W || y + dy < 0 || y + dy >= a.H)
                    continue;
                const long long q = (long long)(y + dy) * a.W + x + dx;
                if (beats(a.r25[q], q, r, idx)) {
                    is_max = false;
                    break;
                }
            }
        if (is_max && (best_i < 0 || beats(r, idx, best_r, best_i))) {
            best_r = r;
            best_i = idx;
        }
    }
    __shared__ long long sr[256], si[256];
    sr[threadIdx.x] = best_r;
    si[threadIdx.x] = best_i;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const long long ri = sr[threadIdx.x + o], ii = si[threadIdx.x + o];
            if (ii >= 0 && (si[threadIdx.x] < 0 || beats(ri, ii, sr[threadIdx.x], si[threadIdx.x]))) {
                sr[threadIdx.x] = ri;
                si[threadIdx.x] = ii;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long i = si[0];
        a.corners[2 * blockIdx.x] = i < 0 ? -1 : (int32_t)(i % a.W);
        a.corners[2 * blockIdx.x + 1] = i < 0 ? -1 : (int32_t)(i / a.W);
    }
}

// ---------------------------------------------------------------------------
// ZSSD

struct ZssdArgs {
    const uint8_t *rgb1, *rgb2;
    int W, H, pitch, r, S;
    const int32_t *corners;
    double *pos;      // n x 2
    int64_t *cost;    // n
};

// One CTA per corner.  With D = I1 - I2 over the patch, exactly in integers,
//   sum D = sum I1 - sum I2,   sum D^2 = sum I1^2 - 2 sum I1 I2 + sum I2^2,
// and the three sums over the displaced patch of frame 2 come from dp4a on
// packed luma bytes: the cross-correlation with the patch of frame 1, the
// byte sum (dp4a with ones) and the sum of squares (dp4a of a word with
// itself), four pixels per instruction.  Frame 2's search region is staged
// as bytes in four copies shifted by 0..3 bytes, so the patch row at any
// column starts on a word.  The sums of frame 1's patch are taken once.
constexpr int kZssdWords = (2 * kMaxRadius + 1 + 3) / 4;            // words per patch row
constexpr int kZssdRegion = 2 * (kMaxSearch + kMaxRadius) + 1;      // region rows and columns
constexpr int kZssdRegionWords = (2 * kMaxSearch) / 4 + kZssdWords;  // words per shifted region row

__global__ void __launch_bounds__(256) k_zssd(ZssdArgs a)
{
    pdl_begin();
    __shared__ uint32_t p1w[2 * kMaxRadius + 1][kZssdWords];
    __shared__ __align__(16) uint8_t reg8[kZssdRegion][4 * (kZssdRegionWords + 1)];   // frame 2 around the corner, 0 outside
    __shared__ uint32_t r4[4][kZssdRegion][kZssdRegionWords];           // reg8 rows from byte 4w + s
    __shared__ long long p1sums[2];                                     // sum I1, sum I1^2
    __shared__ long long sz[256];
    __shared__ int sk[256];
    const int ci = blockIdx.x;
    const int x = a.corners[2 * ci], y = a.corners[2 * ci + 1];
    const int r = a.r, S = a.S, P = 2 * r + 1, RG = 2 * (S + r) + 1, ND = (2 * S + 1) * (2 * S + 1);
    const int WP = (P + 3) / 4, RW = (2 * S) / 4 + WP;
    const uint32_t lastmask = (P & 3) ? (1u << (8 * (P & 3))) - 1u : 0xFFFFFFFFu;
    const bool ok = x >= r && x < a.W - r && y >= r && y < a.H - r;
    if (!ok) {   // no corner, or its patch leaves frame 1
        if (threadIdx.x == 0) {
            a.pos[2 * ci] = a.pos[2 * ci + 1] = __longlong_as_double(0x7FF8000000000000LL);
            a.cost[ci] = -1;
        }
        return;
    }
    for (int i = threadIdx.x; i < P * kZssdWords; i += blockDim.x) {
        const int py = i / kZssdWords, w = i - py * kZssdWords;
        uint32_t v = 0u;
        for (int b = 0; b < 4; ++b) {
            const int px = 4 * w + b;
            if (px < P)
                v |= (uint32_t)luma(a.rgb1 + (size_t)(y - r + py) * a.pitch + 3 * (size_t)(x - r + px)) << (8 * b);
        }
        p1w[py][w] = v;
    }
    constexpr int RB = 4 * (kZssdRegionWords + 1);
    for (int i = threadIdx.x; i < RG * RB; i += blockDim.x) {
        const int ry = i / RB, rx = i - ry * RB;
        const int xx = x - S - r + rx, yy = y - S - r + ry;
        reg8[ry][rx] = (rx < RG && xx >= 0 && xx < a.W && yy >= 0 && yy < a.H)
                           ? (uint8_t)luma(a.rgb2 + (size_t)yy * a.pitch + 3 * (size_t)xx)
                           : (uint8_t)0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * RG * RW; i += blockDim.x) {
        const int s = i / (RG * RW), rem = i - s * RG * RW, ry = rem / RW, w = rem - ry * RW;
        const uint32_t *row = reinterpret_cast<const uint32_t *>(reg8[ry]);
        r4[s][ry][w] = __funnelshift_r(row[w], row[w + 1], 8 * s);
    }
    if (threadIdx.x == 0) {
        int s1 = 0, q1 = 0;
        for (int py = 0; py < P; ++py)
            for (int w = 0; w < WP; ++w) {
                s1 = (int)__dp4a(p1w[py][w], 0x01010101u, (unsigned)s1);
                q1 = (int)__dp4a(p1w[py][w], p1w[py][w], (unsigned)q1);
            }
        p1sums[0] = s1;
        p1sums[1] = q1;
    }
    __syncthreads();
    const long long npx = (long long)P * P, S1 = p1sums[0], Q1 = p1sums[1];
    auto zcost = [&](int dx, int dy) -> long long {   // -1 where the patch leaves frame 2
        const int xx = x + dx, yy = y + dy;
        if (xx < r || xx >= a.W - r || yy < r || yy >= a.H - r)
            return -1;
        const int cx = dx + S, cy = dy + S, sh = cx & 3, w0 = cx >> 2;
        unsigned cross = 0u, s2 = 0u, q2 = 0u;
        for (int py = 0; py < P; ++py) {
            const uint32_t *row = r4[sh][cy + py] + w0;
            const uint32_t *p = p1w[py];
#pragma unroll
            for (int w = 0; w < kZssdWords; ++w) {
                if (w >= WP)
                    break;
                const uint32_t rw = w == WP - 1 ? row[w] & lastmask : row[w];
                cross = __dp4a(p[w], rw, cross);
                s2 = __dp4a(rw, 0x01010101u, s2);
                q2 = __dp4a(rw, rw, q2);
            }
        }
        const long long sumD = S1 - (long long)s2;
        const long long sumD2 = Q1 - 2 * (long long)cross + (long long)q2;
        return npx * sumD2 - sumD * sumD;
    };
    long long best = -1;
    int bk = ND;
    for (int k = threadIdx.x; k < ND; k += blockDim.x) {
        const int dy = k / (2 * S + 1) - S, dx = k % (2 * S + 1) - S;
        const long long z = zcost(dx, dy);
        if (z >= 0 && (best < 0 || z < best)) {   // k rises within a thread: the first smallest
            best = z;
            bk = k;
        }
    }
    sz[threadIdx.x] = best;
    sk[threadIdx.x] = bk;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const long long zo = sz[threadIdx.x + o];
            const int ko = sk[threadIdx.x + o];
            const long long zm = sz[threadIdx.x];
            if (zo >= 0 && (zm < 0 || zo < zm || (zo == zm && ko < sk[threadIdx.x]))) {
                sz[threadIdx.x] = zo;
                sk[threadIdx.x] = ko;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x != 0)
        return;
    if (sz[0] < 0) {
        a.pos[2 * ci] = a.pos[2 * ci + 1] = __longlong_as_double(0x7FF8000000000000LL);
        a.cost[ci] = -1;
        return;
    }
    const int k = sk[0];
    const int by = k / (2 * S + 1) - S, bx = k % (2 * S + 1) - S;
    const long long c0 = sz[0];
    double off[2] = {0.0, 0.0};
    for (int axis = 0; axis < 2; ++axis) {
        const int ex = axis == 0 ? 1 : 0, ey = axis == 0 ? 0 : 1;
        const int mx = bx - ex, my = by - ey, qx = bx + ex, qy = by + ey;
        if (mx < -S || my < -S || qx > S || qy > S)
            continue;
        const long long cm = zcost(mx, my), cp = zcost(qx, qy);
        if (cm < 0 || cp < 0)
            continue;
        const long long den = cm - 2 * c0 + cp;
        if (den > 0)
            off[axis] = (double)(cm - cp) / (2.0 * (double)den);
    }
    a.pos[2 * ci] = (double)(x + bx) + off[0];
    a.pos[2 * ci + 1] = (double)(y + by) + off[1];
    a.cost[ci] = c0;
}

// ---------------------------------------------------------------------------
// EPnP, FP64, one CTA

// The rotation (c, s) of a Jacobi step on the pair (p, q).  The angle only
// has to be close to the one that zeroes A[p][q]: the step is an exact
// orthogonal transform whatever t is, because c = 1 / sqrt(1 + t^2) and
// s = t c are taken in FP64 from t, and a slightly inexact angle leaves a
// residue of A[p][q] about 1e-7 of its size, which later sweeps remove (the
// convergence test is unchanged).  So tan(angle) is formed in FP32 -- FP64
// divisions and square roots are long chains of FP64 instructions, which on
// this GPU run at a small fraction of the FP32 rate -- from
// theta = (A[q][q] - A[p][p]) / (2 A[p][q]) as t = sign(theta) /
// (|theta| + sqrt(theta^2 + 1)); a theta beyond the FP32 range gives t = 0
// (then |A[p][q]| < 1e-38 |A[q][q] - A[p][p]|, negligible).
__device__ __forceinline__ void jacobi_angle(double app, double aqq, double apq, double &c, double &s)
{
    const float theta = (float)(aqq - app) / (2.0f * (float)apq);
    const float at = fabsf(theta);
    float tf = 1.0f / (at + sqrtf(fmaf(at, at, 1.0f)));
    if (!(at < 1e30f))
        tf = 0.0f;
    const double t = theta >= 0.0f ? (double)tf : -(double)tf;
    c = rsqrt(fma(t, t, 1.0));
    s = t * c;
}

// Cyclic Jacobi for a 3 x 3 symmetric matrix on one warp: A (row-major) is
// diagonalised in place and V receives the eigenvectors as columns, both
// then sorted by eigenvalue, ascending; the sweeps stop once the squares of
// the off-diagonal entries sum to at most 1e-30 of the diagonal's.  Every
// lane calls it (A, V, ev in shared memory) and takes the same angles; lanes
// 0-2 update one element of each column, row and eigenvector pass.
__device__ void jacobi3_warp(double *A, double *V, double *ev)
{
    const int lane = threadIdx.x & 31;
    if (lane < 9)
        V[lane] = lane % 4 == 0 ? 1.0 : 0.0;
    __syncwarp();
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < 3; ++p) {
            diag += A[p * 3 + p] * A[p * 3 + p];
            for (int q = p + 1; q < 3; ++q)
                off += A[p * 3 + q] * A[p * 3 + q];
        }
        if (off <= 1e-30 * diag || off == 0.0)
            break;
        for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 3; ++q) {
                const double apq = A[p * 3 + q];
                if (apq == 0.0)
                    continue;
                double c, sn;
                jacobi_angle(A[p * 3 + p], A[q * 3 + q], apq, c, sn);
                __syncwarp();
                if (lane < 3) {   // columns p, q
                    const double akp = A[lane * 3 + p], akq = A[lane * 3 + q];
                    A[lane * 3 + p] = c * akp - sn * akq;
                    A[lane * 3 + q] = sn * akp + c * akq;
                }
                __syncwarp();
                if (lane < 3) {   // rows p, q and the eigenvector columns
                    const double apk = A[p * 3 + lane], aqk = A[q * 3 + lane];
                    A[p * 3 + lane] = c * apk - sn * aqk;
                    A[q * 3 + lane] = sn * apk + c * aqk;
                    const double vkp = V[lane * 3 + p], vkq = V[lane * 3 + q];
                    V[lane * 3 + p] = c * vkp - sn * vkq;
                    V[lane * 3 + q] = sn * vkp + c * vkq;
                }
                __syncwarp();
            }
    }
    if (lane < 3)
        ev[lane] = A[lane * 3 + lane];
    __syncwarp();
    for (int i = 0; i < 3; ++i) {   // selection sort, ascending (the same choice on every lane)
        int mi = i;
        for (int j = i + 1; j < 3; ++j)
            if (ev[j] < ev[mi])
                mi = j;
        __syncwarp();
        if (mi != i) {
            if (lane < 3) {
                const double v = V[lane * 3 + i];
                V[lane * 3 + i] = V[lane * 3 + mi];
                V[lane * 3 + mi] = v;
            }
            if (lane == 0) {
                const double t = ev[i];
                ev[i] = ev[mi];
                ev[mi] = t;
            }
        }
        __syncwarp();
    }
}

// The same decomposition on three warps (threads 0-95, which all call it)
// for even n <= 16: the 12 x 12 normal matrix of Eq. 6.  A sweep is n - 1
// rounds of n / 2 disjoint rotations (the round-robin ordering: pairs
// (r, n - 1) and ((r + i) mod (n - 1), (r - i) mod (n - 1)), i = 1 ..
// n/2 - 1); each round's angles come from the matrix before it (the 2 x 2
// subproblems of disjoint pairs are independent), then the columns and the
// eigenvector columns, and then the rows, are updated with one element pair
// per thread.  The three warps run on three schedulers, whose FP64 units
// work in parallel; they meet at named barrier 1.  Same convergence test and
// ascending order as jacobi3_warp; A, V, ev in shared memory.
__device__ __forceinline__ void bar_jacobi()
{
    asm volatile("bar.sync 1, 96;" ::: "memory");
}

// warm: V holds an orthogonal matrix on entry (the eigenvectors of a
// nearby matrix); A is first replaced by V^T A V (T: n x n scratch) and
// the sweeps start from there, so a matrix close to the earlier one needs
// fewer of them.  The result is the same decomposition, to rounding.
__device__ void jacobi_eigen_warps(double *A, double *V, double *ev, int n, bool warm, double *T)
{
    __shared__ double rc[8], rs[8], conv[2];
    __shared__ int rp[8], rq[8];
    const unsigned full = 0xffffffffu;
    const int tid = threadIdx.x, half = n / 2, m = n - 1, np = n * half;
    if (warm) {
        for (int e = tid; e < n * n; e += 96) {   // T = A V
            const int i = e / n, j = e % n;
            double acc = 0.0;
            for (int k = 0; k < n; ++k)
                acc += A[i * n + k] * V[k * n + j];
            T[e] = acc;
        }
        bar_jacobi();
        for (int e = tid; e < n * n; e += 96) {   // A = V^T T, upper triangle
            const int i = e / n, j = e % n;
            if (j < i)
                continue;
            double acc = 0.0;
            for (int k = 0; k < n; ++k)
                acc += V[k * n + i] * T[k * n + j];
            A[i * n + j] = acc;
        }
        bar_jacobi();
        for (int e = tid; e < n * n; e += 96) {   // mirrored: A stays exactly symmetric
            const int i = e / n, j = e % n;
            if (j < i)
                A[e] = A[j * n + i];
        }
    } else {
        for (int e = tid; e < n * n; e += 96)
            V[e] = e / n == e % n ? 1.0 : 0.0;
    }
    bar_jacobi();
    for (int sweep = 0; sweep < 60; ++sweep) {
        if (tid < 32) {   // convergence sums on warp 0
            double off = 0.0, diag = 0.0;
            for (int e = tid; e < n * n; e += 32) {
                const int r = e / n, c = e % n;
                if (r == c)
                    diag += A[e] * A[e];
                else if (r < c)
                    off += A[e] * A[e];
            }
            for (int o = 16; o > 0; o >>= 1) {
                off += __shfl_xor_sync(full, off, o);
                diag += __shfl_xor_sync(full, diag, o);
            }
            if (tid == 0) {
                conv[0] = off;
                conv[1] = diag;
            }
        }
        bar_jacobi();
        const double off = conv[0], diag = conv[1];
        if (off <= 1e-30 * diag || off == 0.0)
            break;
        for (int r = 0; r < m; ++r) {
            if (tid < half) {
                int p = tid == 0 ? r : (r + tid) % m;
                int q = tid == 0 ? m : (r - tid + m) % m;
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                const double apq = A[p * n + q];
                double c = 1.0, sn = 0.0;
                if (apq != 0.0)
                    jacobi_angle(A[p * n + p], A[q * n + q], apq, c, sn);
                rc[tid] = c;
                rs[tid] = sn;
                rp[tid] = p;
                rq[tid] = q;
            }
            bar_jacobi();
            // columns p, q of every row of A, and of V
            for (int e = tid; e < 2 * np; e += 96) {
                double *M = e < np ? A : V;
                const int f = e < np ? e : e - np;
                const int k = f / half, i = f % half, p = rp[i], q = rq[i];
                const double c = rc[i], sn = rs[i];
                const double mkp = M[k * n + p], mkq = M[k * n + q];
                M[k * n + p] = c * mkp - sn * mkq;
                M[k * n + q] = sn * mkp + c * mkq;
            }
            bar_jacobi();
            for (int e = tid; e < np; e += 96) {   // rows p, q of A
                const int i = e / n, k = e % n, p = rp[i], q = rq[i];
                const double c = rc[i], sn = rs[i];
                const double apk = A[p * n + k], aqk = A[q * n + k];
                A[p * n + k] = c * apk - sn * aqk;
                A[q * n + k] = sn * apk + c * aqk;
            }
            bar_jacobi();
        }
    }
    for (int i = tid; i < n; i += 96)
        ev[i] = A[i * n + i];
    bar_jacobi();
    for (int i = 0; i < n; ++i) {   // selection sort, ascending (the same choice on every thread)
        int mi = i;
        for (int j = i + 1; j < n; ++j)
            if (ev[j] < ev[mi])
                mi = j;
        bar_jacobi();
        if (mi != i) {
            if (tid < n) {
                const double v = V[tid * n + i];
                V[tid * n + i] = V[tid * n + mi];
                V[tid * n + mi] = v;
            }
            if (tid == 0) {
                const double t = ev[i];
                ev[i] = ev[mi];
                ev[mi] = t;
            }
        }
        bar_jacobi();
    }
}

// Solves the symmetric positive semi-definite system (A^T A) x = A^T b of a
// least-squares problem given as the normal matrix N (m x m) and right side
// g, by Gaussian elimination with partial pivoting; one thread.
__device__ void solve_small(double *N, double *g, double *x, int m)
{
    for (int c = 0; c < m; ++c) {
        int p = c;
        for (int r = c + 1; r < m; ++r)
            if (fabs(N[r * m + c]) > fabs(N[p * m + c]))
                p = r;
        if (p != c) {
            for (int k = 0; k < m; ++k) {
                const double t = N[c * m + k];
                N[c * m + k] = N[p * m + k];
                N[p * m + k] = t;
            }
            const double t = g[c];
            g[c] = g[p];
            g[p] = t;
        }
        const double d = N[c * m + c];
        if (fabs(d) < 1e-300)
            continue;
        for (int r = c + 1; r < m; ++r) {
            const double f = N[r * m + c] / d;
            for (int k = c; k < m; ++k)
                N[r * m + k] -= f * N[c * m + k];
            g[r] -= f * g[c];
        }
    }
    for (int c = m - 1; c >= 0; --c) {
        double s = g[c];
        for (int k = c + 1; k < m; ++k)
            s -= N[c * m + k] * x[k];
        x[c] = fabs(N[c * m + c]) < 1e-300 ? 0.0 : s / N[c * m + c];
    }
}

struct EpnpArgs {
    const double *P;    // n x 3 world points
    const double *uv;   // n x 2 pixels
    int n;
    double fx, fy, cx, cy;
    double *out;        // R (9, row-major), T (3), mean error of the inliers, inlier count
};

// Independent problems of one launch, one CTA each (the left and right
// poses of a stereo pair run side by side on two SMs).
constexpr int kMaxEpnpJobs = 2;
struct EpnpJobs {
    EpnpArgs job[kMaxEpnpJobs];
};

__constant__ int kPairI[6] = {0, 0, 0, 1, 1, 2};
__constant__ int kPairJ[6] = {1, 2, 3, 2, 3, 3};

// Block-wide sum of `k` per-thread values (k <= 80): red holds k x blockDim
// doubles.  Few values: a tree over the threads; many (the 78 entries of the
// normal matrix): thread i adds up value i of every thread in order, which
// issues fewer FP64 instructions on the busiest scheduler.
__device__ void block_sum(double *vals, int k, double *red)
{
    const int t = threadIdx.x, nt = blockDim.x;
    for (int i = 0; i < k; ++i)
        red[i * nt + t] = vals[i];
    __syncthreads();
    if (k >= 8) {
        if (t < k) {
            double acc = 0.0;
            for (int j = 0; j < nt; ++j)
                acc += red[t * nt + j];
            red[t * nt] = acc;
        }
        __syncthreads();
    } else {
        for (int o = nt / 2; o > 0; o >>= 1) {
            if (t < o)
                for (int i = 0; i < k; ++i)
                    red[i * nt + t] += red[i * nt + t + o];
            __syncthreads();
        }
    }
    for (int i = 0; i < k; ++i)
        vals[i] = red[i * nt];
    __syncthreads();
}

struct EpnpShared {
    double cw[4][3];       // world control points
    double Cinv[3][3];     // inverse of [c1 - c0, c2 - c0, c3 - c0]
    double V4[12][4];      // the four null-space directions
    double dw[6];          // squared control-point distances
    double R[3][9], T[3][3], err[3];   // the pose of each beta candidate
    double bestR[9], bestT[3], besterr;
    double j3[3][21];      // 3 x 3 eigen-solves of warps 0-2: A, V, eigenvalues
    double scratch[144 + 144 + 12 + 144];   // normal matrix, eigenvectors, eigenvalues, temporary
    int ninl;
};

// Orthogonal Procrustes for Eq. 7 from the sums of one candidate (v: the
// sums of the camera points (3), of the world points (3), of their outer
// products (9) and the point count): R, T with camera = R world + T.  One
// warp (every lane holds the same v and computes the same numbers; js: its
// 21 doubles of shared scratch); lane 0 writes R and T.
__device__ void procrustes(const double *v, double *R, double *T, double *js)
{
    const int lane = threadIdx.x & 31;
    const double m = v[15];
    double mc[3], mw[3], H[9];
    for (int c = 0; c < 3; ++c) {
        mc[c] = v[c] / m;
        mw[c] = v[3 + c] / m;
    }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            H[3 * r + c] = v[6 + 3 * r + c] - m * mc[r] * mw[c];
    // H = U S V^T: V from the eigenvectors of H^T H, U = H V / s, R = U D V^T
    if (lane == 0)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                js[3 * r + c] = H[r] * H[c] + H[3 + r] * H[3 + c] + H[6 + r] * H[6 + c];
    __syncwarp();
    jacobi3_warp(js, js + 9, js + 18);
    const double *Vv = js + 9;
    // descending singular values: columns 2, 1, 0 of Vv
    double Vd[9], U[9];
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r)
            Vd[3 * r + k] = Vv[3 * r + (2 - k)];
    for (int k = 0; k < 2; ++k) {
        double u[3], nrm = 0.0;
        for (int r = 0; r < 3; ++r)
            u[r] = H[3 * r] * Vd[k] + H[3 * r + 1] * Vd[3 + k] + H[3 * r + 2] * Vd[6 + k];
        for (int j = 0; j < k; ++j) {   // Gram-Schmidt against the earlier columns
            const double d = u[0] * U[j] + u[1] * U[3 + j] + u[2] * U[6 + j];
            for (int r = 0; r < 3; ++r)
                u[r] -= d * U[3 * r + j];
        }
        for (int r = 0; r < 3; ++r)
            nrm += u[r] * u[r];
        nrm = sqrt(nrm);
        for (int r = 0; r < 3; ++r)
            U[3 * r + k] = nrm > 0.0 ? u[r] / nrm : (r == k ? 1.0 : 0.0);
    }
    // third column: the cross product (a right-handed U), then the determinant of U V^T
    U[2] = U[3] * U[7] - U[6] * U[4];
    U[5] = U[6] * U[1] - U[0] * U[7];
    U[8] = U[0] * U[4] - U[3] * U[1];
    const double detV = Vd[0] * (Vd[4] * Vd[8] - Vd[5] * Vd[7]) - Vd[1] * (Vd[3] * Vd[8] - Vd[5] * Vd[6]) +
                        Vd[2] * (Vd[3] * Vd[7] - Vd[4] * Vd[6]);
    // U right-handed: det(U V^T) = det V; the reflection fix flips the last singular pair
    const double dl = detV >= 0.0 ? 1.0 : -1.0;
    double Rl[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            Rl[3 * r + c] = U[3 * r] * Vd[3 * c] + U[3 * r + 1] * Vd[3 * c + 1] + dl * U[3 * r + 2] * Vd[3 * c + 2];
    if (lane == 0) {
        for (int k = 0; k < 9; ++k)
            R[k] = Rl[k];
        for (int r = 0; r < 3; ++r)
            T[r] = mc[r] - (Rl[3 * r] * mw[0] + Rl[3 * r + 1] * mw[1] + Rl[3 * r + 2] * mw[2]);
    }
}

// The alphas of point i: its barycentric coordinates in the control points.
__device__ __forceinline__ void point_alphas(const EpnpArgs &a, const EpnpShared &sh, int i, double (&al)[4])
{
    const double d[3] = {a.P[3 * i] - sh.cw[0][0], a.P[3 * i + 1] - sh.cw[0][1], a.P[3 * i + 2] - sh.cw[0][2]};
    for (int k = 0; k < 3; ++k)
        al[k + 1] = sh.Cinv[k][0] * d[0] + sh.Cinv[k][1] * d[1] + sh.Cinv[k][2] * d[2];
    al[0] = 1.0 - al[1] - al[2] - al[3];
}

// Poses of the three beta candidates: control points and points in the
// camera frame, orthogonal Procrustes, mean reprojection error -- all
// threads, each pass over the points serving the three candidates (the
// alphas of a point once), the three Procrustes solutions on warps 0-2.
__device__ void pose_from_betas3(const EpnpArgs &a, const unsigned char *inl, const double (*betas)[4],
                                 EpnpShared &sh, double *red)
{
    double cc[3][12];
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 12; ++r)
            cc[c][r] = betas[c][0] * sh.V4[r][0] + betas[c][1] * sh.V4[r][1] + betas[c][2] * sh.V4[r][2] +
                       betas[c][3] * sh.V4[r][3];
    // the sign: most points in front of the camera
    double v[48];
    for (int c = 0; c < 3; ++c)
        v[c] = 0.0;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        if (!inl[i])
            continue;
        double al[4];
        point_alphas(a, sh, i, al);
        for (int c = 0; c < 3; ++c) {
            const double z = al[0] * cc[c][2] + al[1] * cc[c][5] + al[2] * cc[c][8] + al[3] * cc[c][11];
            v[c] += z < 0.0 ? 1.0 : -1.0;
        }
    }
    block_sum(v, 3, red);
    for (int c = 0; c < 3; ++c) {
        const double sgn = v[c] > 0.0 ? -1.0 : 1.0;   // more negative than positive depths: flip
        for (int r = 0; r < 12; ++r)
            cc[c][r] *= sgn;
    }
    // centroids and the cross-covariance of camera and world points
    for (int k = 0; k < 48; ++k)
        v[k] = 0.0;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        if (!inl[i])
            continue;
        double al[4];
        point_alphas(a, sh, i, al);
        const double *pw = a.P + 3 * i;
        for (int c = 0; c < 3; ++c) {
            double pc[3];
            for (int k = 0; k < 3; ++k)
                pc[k] = al[0] * cc[c][k] + al[1] * cc[c][3 + k] + al[2] * cc[c][6 + k] + al[3] * cc[c][9 + k];
            double *w = v + 16 * c;
            for (int k = 0; k < 3; ++k) {
                w[k] += pc[k];
                w[3 + k] += pw[k];
            }
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 3; ++k)
                    w[6 + 3 * r + k] += pc[r] * pw[k];
            w[15] += 1.0;
        }
    }
    block_sum(v, 48, red);
    if (threadIdx.x < 96) {
        const int c = threadIdx.x >> 5;
        procrustes(v + 16 * c, sh.R[c], sh.T[c], sh.j3[c]);
    }
    __syncthreads();
    // mean reprojection errors
    for (int k = 0; k < 6; ++k)
        v[k] = 0.0;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        if (!inl[i])
            continue;
        const double *pw = a.P + 3 * i;
        for (int c = 0; c < 3; ++c) {
            double pc[3];
            for (int r = 0; r < 3; ++r)
                pc[r] = sh.R[c][3 * r] * pw[0] + sh.R[c][3 * r + 1] * pw[1] + sh.R[c][3 * r + 2] * pw[2] + sh.T[c][r];
            const double du = a.fx * pc[0] / pc[2] + a.cx - a.uv[2 * i];
            const double dv = a.fy * pc[1] / pc[2] + a.cy - a.uv[2 * i + 1];
            v[2 * c] += sqrt(du * du + dv * dv);
            v[2 * c + 1] += 1.0;
        }
    }
    block_sum(v, 6, red);
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c)
            sh.err[c] = v[2 * c] / v[2 * c + 1];
    __syncthreads();
}

// Gauss-Newton on the four betas: the six squared control-point distances,
// on one warp (every lane calls it with the same b).  Lane p < 6 forms the
// residual and Jacobian row of pair p; the 10 distinct entries of the
// normal matrix and the 4 right sides are summed over lanes 0-7 (6 and 7
// add zeros) by a butterfly and taken from lane 0, so every lane solves the
// same 4 x 4 system and b stays the same on all of them.
__device__ void gauss_newton_warp(double *b, const EpnpShared &sh)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    double vd[4][3] = {};
    double dwp = 0.0;
    if (lane < 6) {
        const int i = kPairI[lane], j = kPairJ[lane];
        for (int k = 0; k < 4; ++k)
            for (int c = 0; c < 3; ++c)
                vd[k][c] = sh.V4[3 * i + c][k] - sh.V4[3 * j + c][k];
        dwp = sh.dw[lane];
    }
    auto sum8 = [&](double v) {
        v += __shfl_xor_sync(full, v, 1);
        v += __shfl_xor_sync(full, v, 2);
        v += __shfl_xor_sync(full, v, 4);
        return __shfl_sync(full, v, 0);
    };
    for (int it = 0; it < 5; ++it) {
        double J[4] = {0.0, 0.0, 0.0, 0.0}, res = 0.0;
        if (lane < 6) {
            double d[3];
            for (int c = 0; c < 3; ++c)
                d[c] = b[0] * vd[0][c] + b[1] * vd[1][c] + b[2] * vd[2][c] + b[3] * vd[3][c];
            res = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - dwp;
            for (int k = 0; k < 4; ++k)
                J[k] = 2.0 * (d[0] * vd[k][0] + d[1] * vd[k][1] + d[2] * vd[k][2]);
        }
        double N[16], g[4];
        for (int r = 0; r < 4; ++r) {
            for (int c = r; c < 4; ++c) {
                const double v = sum8(J[r] * J[c]);
                N[4 * r + c] = v;
                N[4 * c + r] = v;
            }
            g[r] = sum8(-J[r] * res);
        }
        double step[4];
        solve_small(N, g, step, 4);
        for (int k = 0; k < 4; ++k)
            b[k] += step[k];
    }
}

// One EPnP solve on the points marked in `inl` (all threads); warm: the
// 12 x 12 eigen-solve starts from the eigenvectors of the previous solve.
__device__ void epnp_solve(const EpnpArgs &a, const unsigned char *inl, EpnpShared &sh, double *red, bool warm)
{
    double v[80];
    // centroid and covariance
    for (int k = 0; k < 4; ++k)
        v[k] = 0.0;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x)
        if (inl[i]) {
            v[0] += a.P[3 * i];
            v[1] += a.P[3 * i + 1];
            v[2] += a.P[3 * i + 2];
            v[3] += 1.0;
        }
    block_sum(v, 4, red);
    const double m = v[3];
    const double c0[3] = {v[0] / m, v[1] / m, v[2] / m};
    for (int k = 0; k < 6; ++k)
        v[k] = 0.0;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x)
        if (inl[i]) {
            const double d[3] = {a.P[3 * i] - c0[0], a.P[3 * i + 1] - c0[1], a.P[3 * i + 2] - c0[2]};
            v[0] += d[0] * d[0];
            v[1] += d[0] * d[1];
            v[2] += d[0] * d[2];
            v[3] += d[1] * d[1];
            v[4] += d[1] * d[2];
            v[5] += d[2] * d[2];
        }
    block_sum(v, 6, red);
    if (threadIdx.x < 32) {   // the principal axes on warp 0
        double *Cs = sh.j3[0];
        if (threadIdx.x == 0) {
            const double C[9] = {v[0] / m, v[1] / m, v[2] / m, v[1] / m, v[3] / m, v[4] / m, v[2] / m, v[4] / m, v[5] / m};
            for (int k = 0; k < 9; ++k)
                Cs[k] = C[k];
        }
        __syncwarp();
        jacobi3_warp(Cs, Cs + 9, Cs + 18);
    }
    if (threadIdx.x == 0) {
        double Vv[9], ev[3];
        for (int k = 0; k < 9; ++k)
            Vv[k] = sh.j3[0][9 + k];
        for (int k = 0; k < 3; ++k)
            ev[k] = sh.j3[0][18 + k];
        // each axis with its largest-magnitude component positive (the control
        // points must not depend on the eigen-solver's choice of signs)
        for (int k = 0; k < 3; ++k) {
            int m = 0;
            for (int r = 1; r < 3; ++r)
                if (fabs(Vv[3 * r + k]) > fabs(Vv[3 * m + k]))
                    m = r;
            if (Vv[3 * m + k] < 0.0)
                for (int r = 0; r < 3; ++r)
                    Vv[3 * r + k] = -Vv[3 * r + k];
        }
        for (int c = 0; c < 3; ++c)
            sh.cw[0][c] = c0[c];
        for (int k = 0; k < 3; ++k) {   // largest variance first
            const double s = sqrt(fmax(ev[2 - k], 0.0));
            for (int c = 0; c < 3; ++c)
                sh.cw[k + 1][c] = c0[c] + s * Vv[3 * c + (2 - k)];
        }
        // inverse of the 3 x 3 matrix of control-point offsets (columns)
        double Cm[3][3];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k)
                Cm[r][k] = sh.cw[k + 1][r] - sh.cw[0][r];
        const double det = Cm[0][0] * (Cm[1][1] * Cm[2][2] - Cm[1][2] * Cm[2][1]) -
                           Cm[0][1] * (Cm[1][0] * Cm[2][2] - Cm[1][2] * Cm[2][0]) +
                           Cm[0][2] * (Cm[1][0] * Cm[2][1] - Cm[1][1] * Cm[2][0]);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                const int r1 = (c + 1) % 3, r2 = (c + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
                sh.Cinv[r][c] = (Cm[r1][c1] * Cm[r2][c2] - Cm[r1][c2] * Cm[r2][c1]) / det;
            }
        for (int p = 0; p < 6; ++p) {
            const int i = kPairI[p], j = kPairJ[p];
            double d2 = 0.0;
            for (int c = 0; c < 3; ++c)
                d2 += (sh.cw[i][c] - sh.cw[j][c]) * (sh.cw[i][c] - sh.cw[j][c]);
            sh.dw[p] = d2;
        }
    }
    __syncthreads();
    // the 12 x 12 normal matrix of Eq. 6.  Its 3 x 3 block (j, k) is
    //   sum al_j al_k [[1, 0, -u], [0, 1, -v], [-u, -v, u^2 + v^2]]
    // (u, v: normalised image coordinates), so four sums per pair j <= k of
    // control points -- 40 in all -- give every entry.
    for (int k = 0; k < 40; ++k)
        v[k] = 0.0;
    const double inv_fx = 1.0 / a.fx, inv_fy = 1.0 / a.fy;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        if (!inl[i])
            continue;
        double al[4];
        point_alphas(a, sh, i, al);
        // the two equations of Eq. 6 divided by fx and fy (normalised image coordinates)
        const double un = (a.uv[2 * i] - a.cx) * inv_fx, vn = (a.uv[2 * i + 1] - a.cy) * inv_fy;
        const double w2 = un * un + vn * vn;
        int t = 0;
        for (int j = 0; j < 4; ++j)
            for (int k = j; k < 4; ++k, ++t) {
                const double pjk = al[j] * al[k];
                v[t] += pjk;
                v[10 + t] += pjk * un;
                v[20 + t] += pjk * vn;
                v[30 + t] += pjk * w2;
            }
    }
    block_sum(v, 40, red);
    if (threadIdx.x < 96) {   // warps 0-2
        double *MtM = sh.scratch, *Vm = sh.scratch + 144, *ev = sh.scratch + 288;
        if (threadIdx.x == 0) {
            int t = 0;
            for (int j = 0; j < 4; ++j)
                for (int k = j; k < 4; ++k, ++t) {
                    const double blk[3][3] = {{v[t], 0.0, -v[10 + t]},
                                              {0.0, v[t], -v[20 + t]},
                                              {-v[10 + t], -v[20 + t], v[30 + t]}};
                    for (int r = 0; r < 3; ++r)
                        for (int c = 0; c < 3; ++c) {
                            MtM[12 * (3 * j + r) + 3 * k + c] = blk[r][c];
                            MtM[12 * (3 * k + c) + 3 * j + r] = blk[r][c];
                        }
                }
        }
        bar_jacobi();
        jacobi_eigen_warps(MtM, Vm, ev, 12, warm, sh.scratch + 300);
        if (threadIdx.x == 0) {
            for (int r = 0; r < 12; ++r)
                for (int k = 0; k < 4; ++k)
                    sh.V4[r][k] = Vm[12 * r + k];
            sh.besterr = 1e300;
        }
    }
    __syncthreads();
    // the betas of the three candidates (N = 1, 2, 3), one per warp: their
    // serial FP64 chains run side by side on three schedulers
    __shared__ double betas_c[3][4];
    if (threadIdx.x < 96) {
        const int cand = threadIdx.x >> 5, lane = threadIdx.x & 31;
        double b[4] = {0.0, 0.0, 0.0, 0.0};
        if (lane == 0) {
            double vd[4][6][3];
            for (int k = 0; k < 4; ++k)
                for (int p = 0; p < 6; ++p)
                    for (int c = 0; c < 3; ++c)
                        vd[k][p][c] = sh.V4[3 * kPairI[p] + c][k] - sh.V4[3 * kPairJ[p] + c][k];
            auto dot = [&](int k, int l, int p) {
                return vd[k][p][0] * vd[l][p][0] + vd[k][p][1] * vd[l][p][1] + vd[k][p][2] * vd[l][p][2];
            };
            if (cand == 0) {   // N = 1
                double num = 0.0, den = 0.0;
                for (int p = 0; p < 6; ++p) {
                    const double dv = sqrt(dot(0, 0, p));
                    num += dv * sqrt(sh.dw[p]);
                    den += dv * dv;
                }
                b[0] = num / den;
            } else if (cand == 1) {   // N = 2: unknowns (b1^2, b1 b2, b2^2)
                double N[9] = {0}, g[3] = {0}, s[3];
                for (int p = 0; p < 6; ++p) {
                    const double row[3] = {dot(0, 0, p), 2.0 * dot(0, 1, p), dot(1, 1, p)};
                    for (int r = 0; r < 3; ++r) {
                        for (int c = 0; c < 3; ++c)
                            N[3 * r + c] += row[r] * row[c];
                        g[r] += row[r] * sh.dw[p];
                    }
                }
                solve_small(N, g, s, 3);
                b[0] = sqrt(fabs(s[0]));
                b[1] = (s[1] > 0.0 ? 1.0 : (s[1] < 0.0 ? -1.0 : 0.0)) * sqrt(fabs(s[2]));
            } else {   // N = 3: six products, six equations
                double N[36] = {0}, g[6] = {0}, s[6];
                for (int p = 0; p < 6; ++p) {
                    const double row[6] = {dot(0, 0, p), 2.0 * dot(0, 1, p), dot(1, 1, p),
                                           2.0 * dot(0, 2, p), 2.0 * dot(1, 2, p), dot(2, 2, p)};
                    for (int r = 0; r < 6; ++r) {
                        for (int c = 0; c < 6; ++c)
                            N[6 * r + c] += row[r] * row[c];
                        g[r] += row[r] * sh.dw[p];
                    }
                }
                solve_small(N, g, s, 6);
                b[0] = sqrt(fabs(s[0]));
                if (b[0] > 0.0) {
                    b[1] = s[1] / b[0];
                    b[2] = s[3] / b[0];
                }
            }
        }
        for (int k = 0; k < 4; ++k)
            b[k] = __shfl_sync(0xffffffffu, b[k], 0);
        gauss_newton_warp(b, sh);
        if (lane == 0)
            for (int k = 0; k < 4; ++k)
                betas_c[cand][k] = b[k];
    }
    __syncthreads();
    pose_from_betas3(a, inl, betas_c, sh, red);
    if (threadIdx.x == 0)
        for (int cand = 0; cand < 3; ++cand)   // in order: the first of equal errors wins
            if (sh.err[cand] < sh.besterr) {
                sh.besterr = sh.err[cand];
                for (int k = 0; k < 9; ++k)
                    sh.bestR[k] = sh.R[cand][k];
                for (int k = 0; k < 3; ++k)
                    sh.bestT[k] = sh.T[cand][k];
            }
    __syncthreads();
}

__global__ void __launch_bounds__(kEpnpThreads) k_epnp(const __grid_constant__ EpnpJobs jobs)
{
    pdl_begin();
    const EpnpArgs &a = jobs.job[blockIdx.x];
    __shared__ unsigned char inl[kMaxPts];
    __shared__ EpnpShared sh;
    extern __shared__ double red[];   // 80 x blockDim
    __shared__ double errs[kMaxPts];
    // usable points: finite world point and pixel
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        const double *p = a.P + 3 * i, *u = a.uv + 2 * i;
        inl[i] = isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]) && isfinite(u[0]) && isfinite(u[1]);
    }
    __syncthreads();
    double cnt[1] = {0.0};
    for (int i = threadIdx.x; i < a.n; i += blockDim.x)
        cnt[0] += inl[i];
    block_sum(cnt, 1, red);
    if (cnt[0] < 6.0) {
        if (threadIdx.x == 0)
            for (int k = 0; k < 14; ++k)
                a.out[k] = k < 13 ? __longlong_as_double(0x7FF8000000000000LL) : cnt[0];
        return;
    }
    epnp_solve(a, inl, sh, red, false);
    if (threadIdx.x == 0)
        sh.ninl = (int)cnt[0];
    __syncthreads();
    // inlier rounds: keep the errors below max(2 px, 3 x the median)
    for (int round = 0; round < 2; ++round) {
        for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
            const double *p = a.P + 3 * i, *u = a.uv + 2 * i;
            const bool usable = isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]) && isfinite(u[0]) && isfinite(u[1]);
            double e = INFINITY;
            if (usable) {
                double pc[3];
                for (int r = 0; r < 3; ++r)
                    pc[r] = sh.bestR[3 * r] * p[0] + sh.bestR[3 * r + 1] * p[1] + sh.bestR[3 * r + 2] * p[2] +
                            sh.bestT[r];
                const double du = a.fx * pc[0] / pc[2] + a.cx - u[0], dv = a.fy * pc[1] / pc[2] + a.cy - u[1];
                e = sqrt(du * du + dv * dv);
            }
            errs[i] = e;
        }
        __syncthreads();
        // the median of the usable errors, exact: the errors are >= 0 or +inf
        // (NaN: unusable), whose bit patterns as 64-bit integers order as the
        // numbers do, so they are sorted as integers (a bitonic network over
        // the next power of two, padded with the largest key, in the
        // reduction scratch) and the middle one or two read off
        const long long *ek = reinterpret_cast<const long long *>(errs);
        constexpr long long kInfBits = 0x7FF0000000000000LL;
        __shared__ int nusable;
        if (threadIdx.x == 0)
            nusable = 0;
        long long *key = reinterpret_cast<long long *>(red);   // 80 x blockDim doubles >= kMaxPts
        int N = 1;
        while (N < a.n)
            N <<= 1;
        for (int i = threadIdx.x; i < N; i += blockDim.x)
            key[i] = i < a.n ? ek[i] : LLONG_MAX;
        __syncthreads();
        {
            int cnt_u = 0;
            for (int i = threadIdx.x; i < a.n; i += blockDim.x)
                cnt_u += ek[i] < kInfBits;
            atomicAdd(&nusable, cnt_u);
        }
        for (int k = 2; k <= N; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < N; i += blockDim.x) {
                    const int l = i ^ j;
                    if (l > i) {
                        const long long x = key[i], y = key[l];
                        if ((x > y) == ((i & k) == 0)) {
                            key[i] = y;
                            key[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        const int n = nusable;
        const double med = __longlong_as_double(key[(n - 1) / 2]), med_hi = __longlong_as_double(key[n / 2]);
        __syncthreads();   // the scratch is the reductions' again
        const double thr = fmax(2.0, 3.0 * (0.5 * (med + med_hi)));
        int changed = 0;
        for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
            const unsigned char m = errs[i] < thr;
            changed |= m != inl[i];
            inl[i] = m;
        }
        // the same points as the last solve give the same pose, whose errors
        // give the same points again: nothing is left to do
        if (!__syncthreads_or(changed))
            break;
        cnt[0] = 0.0;
        for (int i = threadIdx.x; i < a.n; i += blockDim.x)
            cnt[0] += inl[i];
        block_sum(cnt, 1, red);
        if (cnt[0] < 6.0)
            break;
        epnp_solve(a, inl, sh, red, true);   // the inliers: a nearby normal matrix
        if (threadIdx.x == 0)
            sh.ninl = (int)cnt[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 9; ++k)
            a.out[k] = sh.bestR[k];
        for (int k = 0; k < 3; ++k)
            a.out[9 + k] = sh.bestT[k];
        a.out[12] = sh.besterr;
        a.out[13] = (double)sh.ninl;
    }
}

// ---------------------------------------------------------------------------
// the whole pose step: points of the frame-1 corners from its cloud

struct GatherArgs {
    const int32_t *corners;
    const float *xyz;
    const double *pos;
    int W, n;
    double *P;
    double *uv;
};

__global__ void k_pose_gather(GatherArgs a)
{
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n)
        return;
    const double nan = __longlong_as_double(0x7FF8000000000000LL);
    const int x = a.corners[2 * i], y = a.corners[2 * i + 1];
    double p[3] = {nan, nan, nan};
    if (x >= 0) {
        const float *q = a.xyz + ((size_t)y * a.W + x) * 3;
        p[0] = q[0];
        p[1] = q[1];
        p[2] = q[2];
    }
    a.P[3 * i] = p[0];
    a.P[3 * i + 1] = p[1];
    a.P[3 * i + 2] = p[2];
    a.uv[2 * i] = a.pos[2 * i];
    a.uv[2 * i + 1] = a.pos[2 * i + 1];
}

bool pose_params_ok(int W, int H, const vs_pose_params *p)
{
    return p && W > 0 && H > 0 && (long long)W * H <= (1LL << 27) && p->grid >= 1 && p->grid <= kMaxGrid &&
           p->radius >= 1 && p->radius <= kMaxRadius && p->search >= 0 && p->search <= kMaxSearch &&
           p->margin >= p->radius + 1 && 2 * p->margin < W && 2 * p->margin < H;
}

// ---------------------------------------------------------------------------
// Section 2.3: the left and right poses of a later stereo pair, averaged

struct AvgArgs {
    const double *left, *right;   // 14 doubles each: R (9), T (3), error, inliers
    double baseline;
    double *out;
};

// One warp.  The right estimate is moved to the left camera through the
// rig (T + (baseline, 0, 0)); R is the polar factor of M = R_left + R_right,
// sum_i d_i (M v_i / s_i) v_i^T over the eigenvectors v_i of M^T M (s_i the
// square roots of its eigenvalues), with d = -1 on the smallest pair when
// det M < 0 (never for two rotations less than 180 degrees apart).
__global__ void __launch_bounds__(32) k_pose_average(AvgArgs a)
{
    pdl_begin();
    __shared__ double js[21];
    const int lane = threadIdx.x;
    const double nan = __longlong_as_double(0x7FF8000000000000LL);
    double RL[9], TL[3], RR[9], TR[3];
    bool okL = true, okR = true;
    for (int k = 0; k < 9; ++k) {
        RL[k] = a.left[k];
        RR[k] = a.right[k];
        okL = okL && isfinite(RL[k]);
        okR = okR && isfinite(RR[k]);
    }
    for (int k = 0; k < 3; ++k) {
        TL[k] = a.left[9 + k];
        TR[k] = a.right[9 + k] + (k == 0 ? a.baseline : 0.0);
        okL = okL && isfinite(TL[k]);
        okR = okR && isfinite(TR[k]);
    }
    if (!okL || !okR) {   // one estimate or none
        if (lane == 0) {
            const double *R = okL ? RL : RR, *T = okL ? TL : TR;
            const double *src = okL ? a.left : a.right;
            for (int k = 0; k < 9; ++k)
                a.out[k] = okL || okR ? R[k] : nan;
            for (int k = 0; k < 3; ++k)
                a.out[9 + k] = okL || okR ? T[k] : nan;
            a.out[12] = okL || okR ? src[12] : nan;
            a.out[13] = okL || okR ? src[13] : 0.0;
        }
        return;
    }
    double M[9];
    for (int k = 0; k < 9; ++k)
        M[k] = RL[k] + RR[k];
    if (lane == 0)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                js[3 * r + c] = M[r] * M[c] + M[3 + r] * M[3 + c] + M[6 + r] * M[6 + c];
    __syncwarp();
    jacobi3_warp(js, js + 9, js + 18);
    const double *V = js + 9, *ev = js + 18;
    const double detM = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                        M[2] * (M[3] * M[7] - M[4] * M[6]);
    double R[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 3; ++i) {   // eigenvalues ascending: i = 0 is the smallest pair
        const double s = sqrt(fmax(ev[i], 0.0));
        const double d = (i == 0 && detM < 0.0) ? -1.0 : 1.0;
        double u[3];
        for (int r = 0; r < 3; ++r)
            u[r] = (M[3 * r] * V[i] + M[3 * r + 1] * V[3 + i] + M[3 * r + 2] * V[6 + i]) / s;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                R[3 * r + c] += d * u[r] * V[3 * c + i];
    }
    if (lane == 0) {
        for (int k = 0; k < 9; ++k)
            a.out[k] = R[k];
        for (int k = 0; k < 3; ++k)
            a.out[9 + k] = 0.5 * (TL[k] + TR[k]);
        a.out[12] = 0.5 * (a.left[12] + a.right[12]);
        a.out[13] = a.left[13] + a.right[13];
    }
}

struct PoseLayout {
    size_t r25, corners, pos, cost, P, uv, total;
};

PoseLayout pose_layout(int W, int H, const vs_pose_params *p)
{
    PoseLayout l;
    const size_t nc = (size_t)p->grid * p->grid;
    size_t off = 0;
    l.r25 = off;
    off = align_up(off + (size_t)W * H * sizeof(int64_t), 256);
    l.corners = off;
    off = align_up(off + nc * 2 * sizeof(int32_t), 256);
    l.pos = off;
    off = align_up(off + nc * 2 * sizeof(double), 256);
    l.cost = off;
    off = align_up(off + nc * sizeof(int64_t), 256);
    l.P = off;
    off = align_up(off + nc * 3 * sizeof(double), 256);
    l.uv = off;
    off = align_up(off + nc * 2 * sizeof(double), 256);
    l.total = off;
    return l;
}

int launch_harris(const uint8_t *rgb, int W, int H, int pitch, int64_t *r25, cudaStream_t st)
{
    HarrisArgs a{rgb, W, H, pitch, r25};
    launch_pdl(k_harris_r25, dim3((W + kHarrisTx - 1) / kHarrisTx, (H + kHarrisTy - 1) / kHarrisTy),
               dim3(kHarrisTx, kHarrisTy), st, a);
    note_launch();
    return launch_status();
}

int launch_cells(const int64_t *r25, int W, int H, const vs_pose_params *p, int32_t *corners, cudaStream_t st)
{
    CellArgs a{r25, W, H, p->grid, p->margin, (long long)p->threshold25, corners};
    launch_pdl(k_harris_cells, dim3(p->grid * p->grid), dim3(256), st, a);
    note_launch();
    return launch_status();
}

int launch_zssd(const uint8_t *rgb1, const uint8_t *rgb2, int W, int H, int pitch, const int32_t *corners, int n,
                const vs_pose_params *p, double *pos, int64_t *cost, cudaStream_t st)
{
    ZssdArgs a{rgb1, rgb2, W, H, pitch, p->radius, p->search, corners, pos, cost};
    launch_pdl(k_zssd, dim3(n), dim3(256), st, a);
    note_launch();
    return launch_status();
}

// njobs (1 or 2) problems in one launch.
int launch_epnp_jobs(const EpnpJobs &jobs, int njobs, cudaStream_t st)
{
    launch_pdl_smem(k_epnp, dim3((unsigned)njobs), dim3(kEpnpThreads), (size_t)80 * kEpnpThreads * sizeof(double),
                    st, jobs);
    note_launch();
    return launch_status();
}

EpnpArgs epnp_args(const double *P, const double *uv, int n, const vs_camera *cam, double *out)
{
    return EpnpArgs{P, uv, n, cam->fx, cam->fy, cam->cx, cam->cy, out};
}

int launch_epnp(const double *P, const double *uv, int n, const vs_camera *cam, double *out, cudaStream_t st)
{
    EpnpJobs jobs{};
    jobs.job[0] = epnp_args(P, uv, n, cam, out);
    return launch_epnp_jobs(jobs, 1, st);
}

// ZSSD matches of the corners of frame 1 in frame 2 and their points from
// frame 1's cloud (P, uv: the EPnP input).
int match_points(const uint8_t *rgb1, const uint8_t *rgb2, const float *xyz1, int W, int H, int pitch,
                 const vs_pose_params *p, const int32_t *corners, int n, double *pos, int64_t *cost, double *P,
                 double *uv, cudaStream_t st)
{
    int rc = launch_zssd(rgb1, rgb2, W, H, pitch, corners, n, p, pos, cost, st);
    if (rc == VS_OK) {
        GatherArgs g{corners, xyz1, pos, W, n, P, uv};
        launch_pdl(k_pose_gather, dim3((n + 127) / 128), dim3(128), st, g);
        note_launch();
        rc = launch_status();
    }
    return rc;
}

// The matches, then EPnP with its inlier rounds into out (14 doubles).
int pose_from_corners(const uint8_t *rgb1, const uint8_t *rgb2, const float *xyz1, int W, int H, int pitch,
                      const vs_camera *cam, const vs_pose_params *p, const int32_t *corners, int n, double *pos,
                      int64_t *cost, double *P, double *uv, double *out, cudaStream_t st)
{
    int rc = match_points(rgb1, rgb2, xyz1, W, H, pitch, p, corners, n, pos, cost, P, uv, st);
    if (rc == VS_OK)
        rc = launch_epnp(P, uv, n, cam, out, st);
    return rc;
}

int launch_average(const double *left, const double *right, double baseline, double *out, cudaStream_t st)
{
    AvgArgs a{left, right, baseline, out};
    launch_pdl(k_pose_average, dim3(1), dim3(32), st, a);
    note_launch();
    return launch_status();
}

// vs_pose_estimate_stereo: the single-pose layout, then the second set of
// matches and points and the two estimates.
struct StereoLayout {
    PoseLayout base;
    size_t pos2, cost2, P2, uv2, outL, outR, total;
};

StereoLayout stereo_layout(int W, int H, const vs_pose_params *p)
{
    StereoLayout l;
    l.base = pose_layout(W, H, p);
    const size_t nc = (size_t)p->grid * p->grid;
    size_t off = l.base.total;
    l.pos2 = off;
    off = align_up(off + nc * 2 * sizeof(double), 256);
    l.cost2 = off;
    off = align_up(off + nc * sizeof(int64_t), 256);
    l.P2 = off;
    off = align_up(off + nc * 3 * sizeof(double), 256);
    l.uv2 = off;
    off = align_up(off + nc * 2 * sizeof(double), 256);
    l.outL = off;
    off = align_up(off + 14 * sizeof(double), 256);
    l.outR = off;
    off = align_up(off + 14 * sizeof(double), 256);
    l.total = off;
    return l;
}

// The EPnP kernel's reduction space (160 KB) is dynamic shared memory: allowed
// once per device.
bool epnp_ready()
{
    constexpr int kMaxDev = 64;
    static bool done[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev)
        return false;
    if (!done[dev]) {
        if (cudaFuncSetAttribute(k_epnp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 80 * kEpnpThreads * (int)sizeof(double)) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        done[dev] = true;
    }
    return true;
}

}  // namespace
}  // namespace vs

extern "C" size_t vs_pose_workspace_size(int W, int H, const vs_pose_params *p)
{
    return vs::pose_params_ok(W, H, p) ? vs::pose_layout(W, H, p).total : 0;
}

extern "C" size_t vs_pose_stereo_workspace_size(int W, int H, const vs_pose_params *p)
{
    return vs::pose_params_ok(W, H, p) ? vs::stereo_layout(W, H, p).total : 0;
}

extern "C" int vs_pose_average(const double *left, const double *right, double baseline, double *out, void *stream)
{
    vs::NvtxRange nvtx_range("vs_pose_average");
    if (!left || !right || !out || !std::isfinite(baseline))
        return VS_EINVAL;
    return vs::launch_average(left, right, baseline, out, (cudaStream_t)stream);
}

extern "C" int vs_harris_response(const uint8_t *rgb, int W, int H, int pitch, int64_t *r25, void *stream)
{
    vs::NvtxRange nvtx_range("vs_harris_response");
    if (!rgb || !r25 || W <= 0 || H <= 0 || pitch < 3 * W || (long long)W * H > (1LL << 27))
        return VS_EINVAL;
    return vs::launch_harris(rgb, W, H, pitch, r25, (cudaStream_t)stream);
}

extern "C" int vs_harris_corners(const uint8_t *rgb, int W, int H, int pitch, const vs_pose_params *p,
                                 int32_t *corners, void *workspace, size_t ws_bytes, void *stream)
{
    using namespace vs;
    NvtxRange nvtx_range("vs_harris_corners");
    if (!rgb || !corners || pitch < 3 * W || !pose_params_ok(W, H, p))
        return VS_EINVAL;
    const PoseLayout l = pose_layout(W, H, p);
    if (!workspace || !aligned(workspace, 256) || ws_bytes < l.total)
        return VS_EWORKSPACE;
    int64_t *r25 = reinterpret_cast<int64_t *>(static_cast<uint8_t *>(workspace) + l.r25);
    const int rc = launch_harris(rgb, W, H, pitch, r25, (cudaStream_t)stream);
    if (rc != VS_OK)
        return rc;
    return launch_cells(r25, W, H, p, corners, (cudaStream_t)stream);
}

extern "C" int vs_zssd_match(const uint8_t *rgb1, const uint8_t *rgb2, int W, int H, int pitch,
                             const int32_t *corners, int n, const vs_pose_params *p, double *pos, int64_t *cost,
                             void *stream)
{
    using namespace vs;
    NvtxRange nvtx_range("vs_zssd_match");
    if (!rgb1 || !rgb2 || !corners || !pos || !cost || n < 0 || n > kMaxPts || pitch < 3 * W ||
        !pose_params_ok(W, H, p))
        return VS_EINVAL;
    if (n == 0)
        return VS_OK;
    return launch_zssd(rgb1, rgb2, W, H, pitch, corners, n, p, pos, cost, (cudaStream_t)stream);
}

extern "C" int vs_epnp(const double *points, const double *uv, int n, const vs_camera *cam, double *out,
                       void *stream)
{
    using namespace vs;
    NvtxRange nvtx_range("vs_epnp");
    if (!points || !uv || !cam || !out || n < 6 || n > kMaxPts || !(cam->fx > 0.0f) || !(cam->fy > 0.0f))
        return VS_EINVAL;
    if (!epnp_ready())
        return VS_ECUDA;
    return launch_epnp(points, uv, n, cam, out, (cudaStream_t)stream);
}

extern "C" int vs_pose_estimate(const uint8_t *rgb1, const uint8_t *rgb2, const float *xyz1, int W, int H,
                                int pitch, const vs_camera *cam, const vs_pose_params *p, double *out,
                                void *workspace, size_t ws_bytes, void *stream)
{
    using namespace vs;
    NvtxRange nvtx_range("vs_pose_estimate");
    if (!rgb1 || !rgb2 || !xyz1 || !cam || !out || pitch < 3 * W || !pose_params_ok(W, H, p) ||
        !(cam->fx > 0.0f) || !(cam->fy > 0.0f))
        return VS_EINVAL;
    const PoseLayout l = pose_layout(W, H, p);
    if (!workspace || !aligned(workspace, 256) || ws_bytes < l.total)
        return VS_EWORKSPACE;
    if (!epnp_ready())
        return VS_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t *ws = static_cast<uint8_t *>(workspace);
    int64_t *r25 = reinterpret_cast<int64_t *>(ws + l.r25);
    int32_t *corners = reinterpret_cast<int32_t *>(ws + l.corners);
    double *pos = reinterpret_cast<double *>(ws + l.pos);
    int64_t *cost = reinterpret_cast<int64_t *>(ws + l.cost);
    double *P = reinterpret_cast<double *>(ws + l.P), *uv = reinterpret_cast<double *>(ws + l.uv);
    const int n = p->grid * p->grid;
    int rc = launch_harris(rgb1, W, H, pitch, r25, st);
    if (rc == VS_OK)
        rc = launch_cells(r25, W, H, p, corners, st);
    if (rc == VS_OK)
        rc = pose_from_corners(rgb1, rgb2, xyz1, W, H, pitch, cam, p, corners, n, pos, cost, P, uv, out, st);
    return rc;
}

extern "C" int vs_pose_estimate_stereo(const uint8_t *left1, const uint8_t *left2, const uint8_t *right2,
                                       const float *xyz1, int W, int H, int pitch, const vs_camera *cam,
                                       double baseline, const vs_pose_params *p, double *out, void *workspace,
                                       size_t ws_bytes, void *stream)
{
    using namespace vs;
    NvtxRange nvtx_range("vs_pose_estimate_stereo");
    if (!left1 || !left2 || !right2 || !xyz1 || !cam || !out || pitch < 3 * W || !pose_params_ok(W, H, p) ||
        !(cam->fx > 0.0f) || !(cam->fy > 0.0f) || !std::isfinite(baseline))
        return VS_EINVAL;
    const StereoLayout l = stereo_layout(W, H, p);
    if (!workspace || !aligned(workspace, 256) || ws_bytes < l.total)
        return VS_EWORKSPACE;
    if (!epnp_ready())
        return VS_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t *ws = static_cast<uint8_t *>(workspace);
    auto at = [&](size_t off) { return ws + off; };
    int64_t *r25 = reinterpret_cast<int64_t *>(at(l.base.r25));
    int32_t *corners = reinterpret_cast<int32_t *>(at(l.base.corners));
    double *outL = reinterpret_cast<double *>(at(l.outL)), *outR = reinterpret_cast<double *>(at(l.outR));
    const int n = p->grid * p->grid;
    int rc = launch_harris(left1, W, H, pitch, r25, st);
    if (rc == VS_OK)
        rc = launch_cells(r25, W, H, p, corners, st);
    double *PL = reinterpret_cast<double *>(at(l.base.P)), *uvL = reinterpret_cast<double *>(at(l.base.uv));
    double *PR = reinterpret_cast<double *>(at(l.P2)), *uvR = reinterpret_cast<double *>(at(l.uv2));
    if (rc == VS_OK)
        rc = match_points(left1, left2, xyz1, W, H, pitch, p, corners, n, reinterpret_cast<double *>(at(l.base.pos)),
                          reinterpret_cast<int64_t *>(at(l.base.cost)), PL, uvL, st);
    if (rc == VS_OK)
        rc = match_points(left1, right2, xyz1, W, H, pitch, p, corners, n, reinterpret_cast<double *>(at(l.pos2)),
                          reinterpret_cast<int64_t *>(at(l.cost2)), PR, uvR, st);
    if (rc == VS_OK) {   // the two poses side by side, one CTA each
        EpnpJobs jobs{};
        jobs.job[0] = epnp_args(PL, uvL, n, cam, outL);
        jobs.job[1] = epnp_args(PR, uvR, n, cam, outR);
        rc = launch_epnp_jobs(jobs, 2, st);
    }
    if (rc == VS_OK)
        rc = launch_average(outL, outR, baseline, out, st);
    return rc;
}
