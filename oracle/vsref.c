/*
 * vsref.c -- plain, slow CPU oracle for the virtual-stereo hot path of
 * "Towards Real-time 3D Reconstruction using Consumer UAVs" (arXiv 1902.09733).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA
 * library.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may build, load or call it.  It shares no code, header, table or
 * constant generator with the CUDA path, and the CUDA path never calls it.
 *
 * Every function follows one step of the method, in the paper's order:
 *   Section 2.1            undistort / rectify remap (radial model, bilinear)
 *   Section 2.2            downsample to the stereo resolution (box mean, luma)
 *   Eq. 1                  data cost, hierarchical min-sum belief propagation,
 *                          per-pixel label = argmin of E_X(d)
 *   Eq. 2                  joint bilateral upsampling of the disparity
 *   Eq. 3                  reprojection to camera-frame (x, y, z)
 * Integer stages use int32/int64; floating-point stages use double.
 * Where the paper is silent the chosen reading is stated beside the code.
 * Built with OpenMP, the rows of a stage are shared among threads where no
 * row reads what another row writes (every loop below says so); the
 * arithmetic and its order per element are the same with one thread or many,
 * so results do not depend on the thread count.
 *
 * Status codes: 0 ok, -1 invalid argument, -2 out of memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads for the row loops (1 without OpenMP); n <= 0 keeps the current
 * setting.  Returns the number the next parallel loop will use. */
int vsref_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static int thread_slot(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

static int max_slots(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define VSREF_OK 0
#define VSREF_EINVAL (-1)
#define VSREF_ENOMEM (-2)

/* ------------------------------------------------------------------------- */
/* Section 2.1 -- undistort + rectify remap.                                  */
/* ------------------------------------------------------------------------- */

/* Value of source channel ch at integer pixel (x, y); pixels outside the
 * frame read as 0 (constant border). */
static double src_tap(const uint8_t *src, int W, int H, int pitch, int x, int y, int ch)
{
    if (x < 0 || y < 0 || x >= W || y >= H)
        return 0.0;
    return (double)src[(size_t)y * pitch + (size_t)x * 3 + ch];
}

/*
 * For every destination (undistorted, rectified) pixel (u, v):
 *   normalised ray       (xn, yn) = ((u - cx) / fx, (v - cy) / fy)
 *   rectification        [X Y Z]^T = R^T [xn yn 1]^T, xn = X/Z, yn = Y/Z
 *                        (R == NULL means R = I: extrinsics are ignored)
 *   radial distortion    r2 = xn^2 + yn^2, xd = xn (1 + k1 r2 + k2 r2^2)
 *                        (radial only, no tangential term)
 *   source pixel         (sx, sy) = (fx xd + cx, fy yd + cy)
 * then a bilinear sample of each of the 3 channels, rounded half-to-even and
 * clamped to 0..255.  Rays with Z <= 0 give 0.
 * cam = {fx, fy, cx, cy, k1, k2}.  Images are interleaved RGB, row pitch in
 * bytes.  dst_f (nullable) receives the value before rounding, W*H*3 doubles.
 */
int vsref_rectify_remap(const uint8_t *src, int W, int H, int src_pitch,
                        const double *cam, const double *R9,
                        uint8_t *dst, int dst_pitch, double *dst_f)
{
    if (!src || !dst || !cam || W <= 0 || H <= 0 || src_pitch < 3 * W || dst_pitch < 3 * W)
        return VSREF_EINVAL;
    const double fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3], k1 = cam[4], k2 = cam[5];
    /* rows are independent: each writes only its own destination row */
#pragma omp parallel for schedule(static)
    for (int v = 0; v < H; ++v) {
        for (int u = 0; u < W; ++u) {
            double xn = (u - cx) / fx;
            double yn = (v - cy) / fy;
            int valid = 1;
            if (R9) {
                double X = R9[0] * xn + R9[3] * yn + R9[6];
                double Y = R9[1] * xn + R9[4] * yn + R9[7];
                double Z = R9[2] * xn + R9[5] * yn + R9[8];
                if (Z <= 0.0) {
                    valid = 0;
                } else {
                    xn = X / Z;
                    yn = Y / Z;
                }
            }
            double val[3] = {0.0, 0.0, 0.0};
            if (valid) {
                double r2 = xn * xn + yn * yn;
                double radial = 1.0 + k1 * r2 + k2 * r2 * r2;
                double sx = fx * (xn * radial) + cx;
                double sy = fy * (yn * radial) + cy;
                if (sx > -1.0 && sx < (double)W && sy > -1.0 && sy < (double)H) {
                    double fx0 = floor(sx), fy0 = floor(sy);
                    int x0 = (int)fx0, y0 = (int)fy0;
                    double ax = sx - fx0, ay = sy - fy0;
                    for (int ch = 0; ch < 3; ++ch) {
                        val[ch] = (1.0 - ax) * (1.0 - ay) * src_tap(src, W, H, src_pitch, x0, y0, ch)
                                + ax * (1.0 - ay) * src_tap(src, W, H, src_pitch, x0 + 1, y0, ch)
                                + (1.0 - ax) * ay * src_tap(src, W, H, src_pitch, x0, y0 + 1, ch)
                                + ax * ay * src_tap(src, W, H, src_pitch, x0 + 1, y0 + 1, ch);
                    }
                }
            }
            for (int ch = 0; ch < 3; ++ch) {
                double r = nearbyint(val[ch]); /* round half to even */
                if (r < 0.0) r = 0.0;
                if (r > 255.0) r = 255.0;
                dst[(size_t)v * dst_pitch + (size_t)u * 3 + ch] = (uint8_t)r;
                if (dst_f)
                    dst_f[((size_t)v * W + u) * 3 + ch] = val[ch];
            }
        }
    }
    return VSREF_OK;
}

/* ------------------------------------------------------------------------- */
/* Section 2.2 -- downsample the rectified frame to the stereo resolution.    */
/* ------------------------------------------------------------------------- */

/*
 * Low-resolution size w = ceil(W / s), h = ceil(H / s).  Each low-res pixel is
 * the mean of the in-frame pixels of its s x s block, per channel, rounded half
 * up in integers: (sum + n/2) / n.  Grey = (77 R + 150 G + 29 B + 128) >> 8 of
 * the low-res colour.  low_rgb is w*h*3 contiguous, low_gray w*h contiguous;
 * either may be NULL.
 */
int vsref_downsample_luma(const uint8_t *rgb, int W, int H, int pitch, int s,
                          uint8_t *low_rgb, uint8_t *low_gray)
{
    if (!rgb || W <= 0 || H <= 0 || s <= 0 || pitch < 3 * W)
        return VSREF_EINVAL;
    int w = (W + s - 1) / s, h = (H + s - 1) / s;
#pragma omp parallel for schedule(static)
    for (int yl = 0; yl < h; ++yl) {
        for (int xl = 0; xl < w; ++xl) {
            int64_t sum[3] = {0, 0, 0};
            int64_t n = 0;
            for (int j = 0; j < s; ++j) {
                for (int i = 0; i < s; ++i) {
                    int x = xl * s + i, y = yl * s + j;
                    if (x >= W || y >= H)
                        continue;
                    for (int ch = 0; ch < 3; ++ch)
                        sum[ch] += rgb[(size_t)y * pitch + (size_t)x * 3 + ch];
                    ++n;
                }
            }
            int64_t mean[3];
            for (int ch = 0; ch < 3; ++ch)
                mean[ch] = (sum[ch] + n / 2) / n;
            if (low_rgb)
                for (int ch = 0; ch < 3; ++ch)
                    low_rgb[((size_t)yl * w + xl) * 3 + ch] = (uint8_t)mean[ch];
            if (low_gray)
                low_gray[(size_t)yl * w + xl] = (uint8_t)((77 * mean[0] + 150 * mean[1] + 29 * mean[2] + 128) >> 8);
        }
    }
    return VSREF_OK;
}

/* ------------------------------------------------------------------------- */
/* Eq. 1 -- data term E_D and its coarse-to-fine pyramid.                     */
/* ------------------------------------------------------------------------- */

/*
 * Level-0 data cost, the truncated absolute difference:
 *   D0(x, y, d) = min(|IL(x, y) - IR(x - d, y)|, Td)   if x - d >= 0
 *               = Td                                    otherwise.
 * Labels d are left-image disparities.  Output layout [y][x][d], int32.
 */
void vsref_cost_level0(const uint8_t *left, const uint8_t *right, int w, int h, int L, int Td, int32_t *D0)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x)
            for (int d = 0; d < L; ++d) {
                int32_t c = Td;
                if (x - d >= 0) {
                    int32_t diff = abs((int32_t)left[(size_t)y * w + x] - (int32_t)right[(size_t)y * w + x - d]);
                    c = diff < Td ? diff : Td;
                }
                D0[((size_t)y * w + x) * L + d] = c;
            }
}

/*
 * One coarser level of the hierarchical cost (reading of "hierarchical"):
 * dimensions halve rounding up, and the coarse cost of a label is the sum of
 * the costs of the (up to four) in-frame children.  The label set is the same
 * at every level.
 */
void vsref_cost_coarsen(const int32_t *fine, int wf, int hf, int L, int32_t *coarse)
{
    int wc = (wf + 1) / 2, hc = (hf + 1) / 2;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < hc; ++y)
        for (int x = 0; x < wc; ++x)
            for (int d = 0; d < L; ++d) {
                int32_t s = 0;
                for (int j = 0; j < 2; ++j)
                    for (int i = 0; i < 2; ++i) {
                        int xf = 2 * x + i, yf = 2 * y + j;
                        if (xf < wf && yf < hf)
                            s += fine[((size_t)yf * wf + xf) * L + d];
                    }
                coarse[((size_t)y * wc + x) * L + d] = s;
            }
}

/* ------------------------------------------------------------------------- */
/* Eq. 1 -- one min-sum message M_{Y,X}(d).                                   */
/* ------------------------------------------------------------------------- */

#define VSREF_MSG_BRUTE 0 /* O(L^2): the plain definition */
#define VSREF_MSG_DT 1    /* O(L): two-pass distance transform, same result */

/*
 * Given h(d') = data term of the sender plus the messages it received from its
 * other neighbours, the outgoing message is
 *   m(d) = min_{d'} [ h(d') + min(c |d - d'|, Ts) ]
 * with the truncated-linear smoothness term, then normalised so that its
 * minimum over d is 0 (m - min m).
 * Mode BRUTE evaluates the minimum over all d' directly.  Mode DT uses the
 * lower envelope of the linear cost (a forward and a backward pass) and caps
 * it at min(h) + Ts; the two agree exactly because a minimum distributes over
 * the two branches of the truncation:
 *   min_{d'} [h(d') + min(c|d-d'|, Ts)]
 *     = min( min_{d'} [h(d') + c|d-d'|],  min_{d'} h(d') + Ts ).
 */
void vsref_message(const int32_t *hv, int L, int c, int Ts, int mode, int32_t *out)
{
    if (mode == VSREF_MSG_BRUTE) {
        for (int d = 0; d < L; ++d) {
            int32_t best = INT32_MAX;
            for (int dp = 0; dp < L; ++dp) {
                int32_t lin = c * abs(d - dp);
                int32_t v = hv[dp] + (lin < Ts ? lin : Ts);
                if (v < best)
                    best = v;
            }
            out[d] = best;
        }
    } else {
        int32_t hmin = INT32_MAX;
        for (int d = 0; d < L; ++d) {
            out[d] = hv[d];
            if (hv[d] < hmin)
                hmin = hv[d];
        }
        for (int d = 1; d < L; ++d)
            if (out[d - 1] + c < out[d])
                out[d] = out[d - 1] + c;
        for (int d = L - 2; d >= 0; --d)
            if (out[d + 1] + c < out[d])
                out[d] = out[d + 1] + c;
        for (int d = 0; d < L; ++d)
            if (hmin + Ts < out[d])
                out[d] = hmin + Ts;
    }
    int32_t mmin = INT32_MAX;
    for (int d = 0; d < L; ++d)
        if (out[d] < mmin)
            mmin = out[d];
    for (int d = 0; d < L; ++d)
        out[d] -= mmin;
}

/* ------------------------------------------------------------------------- */
/* Eq. 1 -- hierarchical loopy min-sum belief propagation.                    */
/* ------------------------------------------------------------------------- */

/* Neighbour directions.  in[k] at pixel p holds the message p received from
 * its neighbour in direction k. */
static const int DX[4] = {-1, +1, 0, 0}; /* 0 left, 1 right, 2 up, 3 down */
static const int DY[4] = {0, 0, -1, +1};
static const int OPP[4] = {1, 0, 3, 2};

/*
 * Runs the whole stereo step on one rectified, downsampled grey pair of size
 * w x h and writes one label per pixel (row-major, w*h bytes).
 *
 * Schedule (readings where the paper defers to its citation):
 *  - levels: level 0 is w x h, each coarser level halves rounding up; the
 *    coarsest level starts from all-zero messages; the first iteration of every
 *    finer level starts from the messages of the parent pixel (x>>1, y>>1),
 *    copied direction by direction.
 *  - iterations: at iteration t (counted from 0 at each level) every pixel with
 *    (x + y + t) even sends a message to each in-frame 4-neighbour.  A pixel
 *    only reads its own incoming messages and only writes those of its
 *    neighbours, which have the other colour, so updating in place reads
 *    exactly the messages as they were at the start of the iteration.
 *  - frame border: a missing neighbour contributes nothing and receives
 *    nothing; border pixels are updated like every other pixel.
 *  - label: after the last iteration of level 0, E_X(d) = D0(X, d) + sum of the
 *    four incoming messages (Eq. 1); the smallest d that minimises it wins.
 * msg_mode selects BRUTE or DT for every message.  msgs_out (nullable)
 * receives the final level-0 incoming messages, layout [k][y][x][d] int32.
 */
int vsref_bp(const uint8_t *left, const uint8_t *right, int w, int h, int L, int levels, int iters,
             int Td, int c, int Ts, int msg_mode, uint8_t *labels, int32_t *msgs_out)
{
    if (!left || !right || !labels || w <= 0 || h <= 0 || L < 2 || L > 256 || levels < 1 || iters < 1 ||
        Td < 0 || c < 0 || Ts < 0)
        return VSREF_EINVAL;

    int lw[32], lh[32];
    lw[0] = w;
    lh[0] = h;
    for (int l = 1; l < levels; ++l) {
        lw[l] = (lw[l - 1] + 1) / 2;
        lh[l] = (lh[l - 1] + 1) / 2;
    }

    /* cost pyramid */
    int32_t *cost[32];
    memset(cost, 0, sizeof(cost));
    int rc = VSREF_OK;
    for (int l = 0; l < levels; ++l) {
        cost[l] = (int32_t *)malloc(sizeof(int32_t) * (size_t)lw[l] * lh[l] * L);
        if (!cost[l]) {
            rc = VSREF_ENOMEM;
            goto done_cost;
        }
    }
    vsref_cost_level0(left, right, w, h, L, Td, cost[0]);
    for (int l = 1; l < levels; ++l)
        vsref_cost_coarsen(cost[l - 1], lw[l - 1], lh[l - 1], L, cost[l]);

    {
        int32_t *msg = NULL, *parent = NULL;
        /* one h and one message buffer per thread */
        const int nslots = max_slots();
        int32_t *hv_all = (int32_t *)malloc(sizeof(int32_t) * L * (size_t)nslots);
        int32_t *mv_all = (int32_t *)malloc(sizeof(int32_t) * L * (size_t)nslots);
        if (!hv_all || !mv_all) {
            rc = VSREF_ENOMEM;
            free(hv_all);
            free(mv_all);
            goto done_cost;
        }
        for (int l = levels - 1; l >= 0; --l) {
            int cw = lw[l], ch = lh[l];
            size_t plane = (size_t)cw * ch * L;
            msg = (int32_t *)calloc(4 * plane, sizeof(int32_t));
            if (!msg) {
                rc = VSREF_ENOMEM;
                free(parent);
                free(hv_all);
                free(mv_all);
                goto done_cost;
            }
            if (parent) { /* coarse-to-fine initialisation */
                int pw = lw[l + 1], ph = lh[l + 1];
                size_t pplane = (size_t)pw * ph * L;
                for (int k = 0; k < 4; ++k)
                    for (int y = 0; y < ch; ++y)
                        for (int x = 0; x < cw; ++x)
                            memcpy(&msg[k * plane + ((size_t)y * cw + x) * L],
                                   &parent[k * pplane + ((size_t)(y >> 1) * pw + (x >> 1)) * L],
                                   sizeof(int32_t) * L);
                free(parent);
                parent = NULL;
            }
            const int32_t *D = cost[l];
            for (int t = 0; t < iters; ++t) {
                /* rows are independent within an iteration: a pixel reads only
                 * its own incoming messages and writes only its neighbours',
                 * which are inactive (the other colour) in this iteration */
#pragma omp parallel for schedule(static)
                for (int y = 0; y < ch; ++y) {
                    int32_t *hv = hv_all + (size_t)thread_slot() * L;
                    int32_t *mv = mv_all + (size_t)thread_slot() * L;
                    for (int x = 0; x < cw; ++x) {
                        if (((x + y + t) & 1) != 0)
                            continue;
                        size_t p = (size_t)y * cw + x;
                        for (int k = 0; k < 4; ++k) {
                            int qx = x + DX[k], qy = y + DY[k];
                            if (qx < 0 || qy < 0 || qx >= cw || qy >= ch)
                                continue;
                            for (int d = 0; d < L; ++d) {
                                int32_t s = D[p * L + d];
                                for (int j = 0; j < 4; ++j) {
                                    if (j == k)
                                        continue; /* exclude what q sent to p */
                                    int nx = x + DX[j], ny = y + DY[j];
                                    if (nx < 0 || ny < 0 || nx >= cw || ny >= ch)
                                        continue; /* missing neighbour */
                                    s += msg[j * plane + p * L + d];
                                }
                                hv[d] = s;
                            }
                            vsref_message(hv, L, c, Ts, msg_mode, mv);
                            size_t q = (size_t)qy * cw + qx;
                            memcpy(&msg[OPP[k] * plane + q * L], mv, sizeof(int32_t) * L);
                        }
                    }
                }
            }
            parent = msg;
        }
        /* labels from the level-0 beliefs */
        {
            size_t plane = (size_t)w * h * L;
#pragma omp parallel for schedule(static)
            for (int y = 0; y < h; ++y)
                for (int x = 0; x < w; ++x) {
                    size_t p = (size_t)y * w + x;
                    int64_t best = INT64_MAX;
                    int bestd = 0;
                    for (int d = 0; d < L; ++d) {
                        int64_t b = cost[0][p * L + d];
                        for (int j = 0; j < 4; ++j) {
                            int nx = x + DX[j], ny = y + DY[j];
                            if (nx < 0 || ny < 0 || nx >= w || ny >= h)
                                continue;
                            b += parent[j * plane + p * L + d];
                        }
                        if (b < best) {
                            best = b;
                            bestd = d;
                        }
                    }
                    labels[p] = (uint8_t)bestd;
                }
            if (msgs_out)
                memcpy(msgs_out, parent, sizeof(int32_t) * 4 * plane);
        }
        free(parent);
        free(hv_all);
        free(mv_all);
    }
done_cost:
    for (int l = 0; l < levels; ++l)
        free(cost[l]);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Eq. 2 -- joint bilateral upsampling.                                       */
/* ------------------------------------------------------------------------- */

/*
 * Full-resolution pixel p = (x, y) of a W x H frame, scale s, low-res size
 * w x h.  Its low-res position is the centre-aligned p_down =
 * ((x + 0.5)/s - 0.5, (y + 0.5)/s - 0.5).  The window W of Eq. 2 is the
 * (2r+1)^2 low-res pixels q_down around round-half-up(p_down), clipped to the
 * low-res frame.  With the Gaussian kernels
 *   s(t) = exp(-t^2 / (2 sigma_s^2))   (t in low-res pixels)
 *   g(t) = exp(-t^2 / (2 sigma_r^2))   (t = Euclidean RGB distance, 0..255)
 * between the full-res colour I_p and the low-res (box-mean) colour of q,
 *   D_p = s * sum_q D'(q) s(|p_down - q_down|) g(|I_p - I_q|) / K_p,
 * K_p the sum of the weights (the factor s converts low-res labels to
 * full-res pixels).  Every weight is divided by the largest one before
 * normalising, which leaves D_p unchanged and keeps K_p >= 1.
 * labels w*h bytes, guide_low w*h*3, guide_full W*H*3, disp W*H doubles.
 */
int vsref_guided_upsample(const uint8_t *labels, int w, int h, const uint8_t *guide_low,
                          const uint8_t *guide_full, int W, int H, int s, int r,
                          double sigma_s, double sigma_r, double *disp)
{
    if (!labels || !guide_low || !guide_full || !disp || w <= 0 || h <= 0 || W <= 0 || H <= 0 || s <= 0 ||
        r < 0 || !(sigma_s > 0.0) || !(sigma_r > 0.0))
        return VSREF_EINVAL;
    int nt = (2 * r + 1) * (2 * r + 1);
    /* one pair of tap buffers per thread; rows are independent */
    const int nslots = max_slots();
    double *ex_all = (double *)malloc(sizeof(double) * nt * (size_t)nslots);
    double *dv_all = (double *)malloc(sizeof(double) * nt * (size_t)nslots);
    if (!ex_all || !dv_all) {
        free(ex_all);
        free(dv_all);
        return VSREF_ENOMEM;
    }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        double *ex = ex_all + (size_t)thread_slot() * nt;
        double *dv = dv_all + (size_t)thread_slot() * nt;
        for (int x = 0; x < W; ++x) {
            double px = (x + 0.5) / s - 0.5, py = (y + 0.5) / s - 0.5;
            int cxl = (int)floor(px + 0.5), cyl = (int)floor(py + 0.5);
            const uint8_t *Ip = &guide_full[((size_t)y * W + x) * 3];
            int n = 0;
            double emax = -INFINITY;
            for (int qy = cyl - r; qy <= cyl + r; ++qy) {
                for (int qx = cxl - r; qx <= cxl + r; ++qx) {
                    if (qx < 0 || qy < 0 || qx >= w || qy >= h)
                        continue;
                    const uint8_t *Iq = &guide_low[((size_t)qy * w + qx) * 3];
                    double ds2 = (px - qx) * (px - qx) + (py - qy) * (py - qy);
                    double dr2 = 0.0;
                    for (int ch = 0; ch < 3; ++ch) {
                        double t = (double)Ip[ch] - (double)Iq[ch];
                        dr2 += t * t;
                    }
                    ex[n] = -ds2 / (2.0 * sigma_s * sigma_s) - dr2 / (2.0 * sigma_r * sigma_r);
                    dv[n] = (double)labels[(size_t)qy * w + qx];
                    if (ex[n] > emax)
                        emax = ex[n];
                    ++n;
                }
            }
            double num = 0.0, K = 0.0;
            for (int i = 0; i < n; ++i) {
                double wt = exp(ex[i] - emax);
                num += wt * dv[i];
                K += wt;
            }
            disp[(size_t)y * W + x] = (double)s * num / K;
        }
    }
    free(ex_all);
    free(dv_all);
    return VSREF_OK;
}

/* ------------------------------------------------------------------------- */
/* Eq. 3 -- reprojection of the full-resolution disparity.                    */
/* ------------------------------------------------------------------------- */

/*
 * With f/du = fx, f/dv = fy (so dv/du = fx/fy), principal point (u0, v0) =
 * (cx, cy) and baseline B (metres), Eq. 3 read as
 *   z = fx B / d,  x = (u - cx) B / d,  y = (v - cy) (fx / fy) B / d.
 * Pixels with d <= 0 (or NaN) have no point and get NaN in all three.
 * cam = {fx, fy, cx, cy}; disp W*H doubles; xyz W*H*3 doubles.
 */
void vsref_reproject(const double *disp, int W, int H, const double *cam, double B, double *xyz)
{
    const double fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
#pragma omp parallel for schedule(static)
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            size_t p = (size_t)v * W + u;
            double d = disp[p];
            if (d > 0.0) {
                xyz[3 * p + 0] = (u - cx) * B / d;
                xyz[3 * p + 1] = (v - cy) * (fx / fy) * B / d;
                xyz[3 * p + 2] = fx * B / d;
            } else {
                xyz[3 * p + 0] = NAN;
                xyz[3 * p + 1] = NAN;
                xyz[3 * p + 2] = NAN;
            }
        }
}
