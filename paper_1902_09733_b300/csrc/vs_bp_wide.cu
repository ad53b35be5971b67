// Eq. 1, general path: hierarchical min-sum BP for the parameters the
// byte-message kernels of vs_bp.cu cannot hold -- up to 256 labels,
// truncations up to 65535, coarse data terms up to 2^28.  Same schedule and
// readings as vs_bp.cu (red-black iterations with (x + y + t) even active,
// missing neighbours contribute 0, coarse data term = sum of the in-frame
// 2 x 2 children, coarse-to-fine copy from the parent (x>>1, y>>1), labels =
// smallest argmin of the final belief).
//
// Layout (caller's workspace, every array 256-byte aligned), per level:
//   cost_l[c][y][x >> 1][Lp]     int32 data term (padding labels: kWBig)
//   msg_l [c][k][y][x >> 1][Lp]  uint16 incoming message from direction k
// with c = (x + y) & 1, k = 0 left, 1 right, 2 up, 3 down, and Lp = 32 LPL
// labels, LPL = 1, 2, 4 or 8 per lane.  A padding label's data term is large
// enough never to be a minimum, so the lower envelope and its minimum over
// the real labels come out exactly as over the labels alone.
//
// k_wsweep: one warp per active pixel, lane j owning labels j LPL .. j LPL +
// LPL - 1.  For each outgoing direction the lane runs the two passes of the
// truncated-linear distance transform over its labels, and the blocks are
// joined by min-plus scans across the warp:
//   F(end of block j) = min over i <= j of (E_i + c LPL (j - i)),
// E_i the block's own end value (shuffle-up doubling), F(d) = min(f(d),
// F(end of block j - 1) + c (d - j LPL + 1)), and the mirror image for the
// backward pass; the minimum over the labels is a warp reduction.
#include "vs_bp_wide.cuh"
#include "vs_check.cuh"

#include <algorithm>

namespace vs {
namespace {

constexpr int kWMaxLevels = 8;
constexpr int32_t kWBig = 1 << 29;   // data term of a padding label
constexpr int kWThreads = 128;       // four warps: four active pixels per CTA

struct WideLayout {
    int L, Lp, lpl, levels;
    int w[kWMaxLevels], h[kWMaxLevels], wh[kWMaxLevels];
    size_t cost_off[kWMaxLevels], msg_off[kWMaxLevels];
    size_t status_off, total;
};

WideLayout wide_layout(int w, int h, const vs_bp_params *p)
{
    WideLayout lay;
    lay.L = p->labels;
    lay.lpl = 1;
    while (32 * lay.lpl < p->labels)
        lay.lpl *= 2;
    lay.Lp = 32 * lay.lpl;
    lay.levels = p->levels;
    size_t off = 0;
    for (int l = 0; l < p->levels; ++l) {
        lay.w[l] = l == 0 ? w : (lay.w[l - 1] + 1) / 2;
        lay.h[l] = l == 0 ? h : (lay.h[l - 1] + 1) / 2;
        lay.wh[l] = (lay.w[l] + 1) / 2;
        const size_t slots = (size_t)2 * lay.h[l] * lay.wh[l];
        lay.cost_off[l] = off;
        off = align_up(off + slots * lay.Lp * sizeof(int32_t), 256);
        lay.msg_off[l] = off;
        off = align_up(off + slots * 4 * lay.Lp * sizeof(uint16_t), 256);
    }
    lay.status_off = off;
    lay.total = align_up(off + sizeof(int), 256);
    return lay;
}

// --------------------------------------------------------------------------
// data term

struct WCost0Args {
    const uint8_t *left, *right;
    int pitch, w, h, wh, L, Lp, Td;
    int32_t *cost;
    int *status;   // reset to VS_OK: the first kernel of every call
};

// D0(x, y, d) = min(|IL(x,y) - IR(x-d,y)|, Td), Td where x - d < 0; one
// thread per (slot, label).
__global__ void k_wcost0(WCost0Args a)
{
    pdl_begin();
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx == 0 && chk(a.status, 4, kSiteStatus))
        *a.status = VS_OK;
    if (idx >= (size_t)2 * a.h * a.wh * a.Lp)
        return;
    const int d = (int)(idx % (unsigned)a.Lp);
    const size_t slot = idx / (unsigned)a.Lp;
    const int xh = (int)(slot % (unsigned)a.wh);
    const size_t row = slot / (unsigned)a.wh;
    const int y = (int)(row % (unsigned)a.h), c = (int)(row / (unsigned)a.h);
    const int x = 2 * xh + ((c + y) & 1);
    if (x >= a.w)
        return;
    int32_t v = kWBig;
    if (d < a.L) {
        v = a.Td;
        const uint8_t *pl = a.left + (size_t)y * a.pitch + x, *pr = a.right + (size_t)y * a.pitch + x - d;
        if (x - d >= 0 && chk(pl, 1, kSiteImage) && chk(pr, 1, kSiteImage))
            v = min(abs((int)*pl - (int)*pr), a.Td);
    }
    if (chk(a.cost + idx, 4, kSiteWideStore))
        a.cost[idx] = v;
}

struct WCostDownArgs {
    const int32_t *fine;
    int32_t *coarse;
    int wf, hf, whf, wc, hc, whc, L, Lp;
};

// Coarse data term: the sum over the in-frame 2 x 2 children; child
// (2x+i, 2y+j) has colour (i+j) & 1 and column slot x.
__global__ void k_wcost_down(WCostDownArgs a)
{
    pdl_begin();
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)2 * a.hc * a.whc * a.Lp)
        return;
    const int d = (int)(idx % (unsigned)a.Lp);
    const size_t slot = idx / (unsigned)a.Lp;
    const int xh = (int)(slot % (unsigned)a.whc);
    const size_t row = slot / (unsigned)a.whc;
    const int y = (int)(row % (unsigned)a.hc), c = (int)(row / (unsigned)a.hc);
    const int x = 2 * xh + ((c + y) & 1);
    if (x >= a.wc)
        return;
    int32_t v = kWBig;
    if (d < a.L) {
        v = 0;
        for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i) {
                const int xf = 2 * x + i, yf = 2 * y + j;
                const int32_t *q = a.fine + ((size_t)(((i + j) & 1) * a.hf + yf) * a.whf + x) * a.Lp + d;
                if (xf < a.wf && yf < a.hf && chk(q, 4, kSiteWideLoad))
                    v += *q;
            }
    }
    if (chk(a.coarse + idx, 4, kSiteWideStore))
        a.coarse[idx] = v;
}

// --------------------------------------------------------------------------
// sweep

struct WSweepArgs {
    const int32_t *cost;
    uint16_t *msg;
    const uint16_t *pmsg;    // parent level (coarse-to-fine initialisation)
    int w, h, wh, pw, ph, pwh, Lp;
    int color;               // active colour, = t & 1
    int from_parent;         // incoming = the parent's messages (first iteration below the coarsest level)
    int zero_in;             // incoming = 0 (first iteration of the coarsest level)
    int materialize;         // also store the incoming used into this pixel's own slots
    int32_t c, ts;           // slope (at most ts: the same V) and truncation
};

template <int N>
__device__ __forceinline__ void ld_u16(const uint16_t *p, int32_t (&v)[N])
{
    if (!chk(p, 2 * N, kSiteWideLoad)) {
#pragma unroll
        for (int i = 0; i < N; ++i)
            v[i] = 0;
        return;
    }
    if constexpr (N == 8) {
        const uint4 q = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            v[2 * i] = (int32_t)(w[i] & 0xFFFFu);
            v[2 * i + 1] = (int32_t)(w[i] >> 16);
        }
    } else if constexpr (N == 4) {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        v[0] = (int32_t)(q.x & 0xFFFFu);
        v[1] = (int32_t)(q.x >> 16);
        v[2] = (int32_t)(q.y & 0xFFFFu);
        v[3] = (int32_t)(q.y >> 16);
    } else if constexpr (N == 2) {
        const uint32_t q = *reinterpret_cast<const uint32_t *>(p);
        v[0] = (int32_t)(q & 0xFFFFu);
        v[1] = (int32_t)(q >> 16);
    } else {
        v[0] = (int32_t)p[0];
    }
}

template <int N>
__device__ __forceinline__ void st_u16(uint16_t *p, const int32_t (&v)[N])
{
    if (!chk(p, 2 * N, kSiteWideStore))
        return;
    if constexpr (N == 8) {
        uint4 q;
        q.x = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
        q.y = (uint32_t)v[2] | ((uint32_t)v[3] << 16);
        q.z = (uint32_t)v[4] | ((uint32_t)v[5] << 16);
        q.w = (uint32_t)v[6] | ((uint32_t)v[7] << 16);
        *reinterpret_cast<uint4 *>(p) = q;
    } else if constexpr (N == 4) {
        *reinterpret_cast<uint2 *>(p) =
            make_uint2((uint32_t)v[0] | ((uint32_t)v[1] << 16), (uint32_t)v[2] | ((uint32_t)v[3] << 16));
    } else if constexpr (N == 2) {
        *reinterpret_cast<uint32_t *>(p) = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
    } else {
        p[0] = (uint16_t)v[0];
    }
}

template <int N>
__device__ __forceinline__ void ld_i32(const int32_t *p, int32_t (&v)[N])
{
    if (!chk(p, 4 * N, kSiteWideLoad)) {
#pragma unroll
        for (int i = 0; i < N; ++i)
            v[i] = 0;
        return;
    }
    if constexpr (N >= 4) {
#pragma unroll
        for (int i = 0; i < N; i += 4) {
            const int4 q = *reinterpret_cast<const int4 *>(p + i);
            v[i] = q.x;
            v[i + 1] = q.y;
            v[i + 2] = q.z;
            v[i + 3] = q.w;
        }
    } else if constexpr (N == 2) {
        const int2 q = *reinterpret_cast<const int2 *>(p);
        v[0] = q.x;
        v[1] = q.y;
    } else {
        v[0] = p[0];
    }
}

__device__ __forceinline__ size_t wslot(int c, int k, int y, int xh, int h, int wh)
{
    return ((size_t)(c * 4 + k) * h + y) * wh + xh;
}

template <int LPL>
__global__ void __launch_bounds__(kWThreads) k_wsweep(WSweepArgs a)
{
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const unsigned wid = (blockIdx.x * kWThreads + threadIdx.x) >> 5;   // slot of the active colour
    if (wid >= (unsigned)a.h * (unsigned)a.wh)
        return;
    const int y = (int)(wid / (unsigned)a.wh), xh = (int)(wid % (unsigned)a.wh);
    const int x = 2 * xh + ((a.color + y) & 1);
    if (x >= a.w)
        return;   // the whole warp: one pixel per warp
    const bool has[4] = {x > 0, x < a.w - 1, y > 0, y < a.h - 1};
    const int d0 = lane * LPL;
    int32_t m[4][LPL];
    {
        const int px = x >> 1, py = y >> 1;
        const bool phas[4] = {px > 0, px < a.pw - 1, py > 0, py < a.ph - 1};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool use = has[k] && !a.zero_in && (!a.from_parent || phas[k]);
            if (use) {
                const uint16_t *src = a.from_parent
                                          ? a.pmsg + wslot((px + py) & 1, k, py, px >> 1, a.ph, a.pwh) * a.Lp
                                          : a.msg + wslot(a.color, k, y, xh, a.h, a.wh) * a.Lp;
                ld_u16<LPL>(src + d0, m[k]);
            } else {
#pragma unroll
                for (int i = 0; i < LPL; ++i)
                    m[k][i] = 0;
            }
            if (a.materialize)
                st_u16<LPL>(a.msg + wslot(a.color, k, y, xh, a.h, a.wh) * a.Lp + d0, m[k]);
        }
    }
    int32_t S[LPL];
    ld_i32<LPL>(a.cost + ((size_t)a.color * a.h * a.wh + (size_t)y * a.wh + xh) * a.Lp + d0, S);
#pragma unroll
    for (int i = 0; i < LPL; ++i)
        S[i] += m[0][i] + m[1][i] + m[2][i] + m[3][i];

    const int dx[4] = {-1, 1, 0, 0}, dy[4] = {0, 0, -1, 1}, opp[4] = {1, 0, 3, 2};
    const int32_t c = a.c;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (!has[k])
            continue;   // uniform over the warp
        int32_t f[LPL];
        int32_t hmin = 0x7FFFFFFF;
#pragma unroll
        for (int i = 0; i < LPL; ++i) {
            const int32_t hv = S[i] - m[k][i];   // data term + the other incoming messages
            hmin = min(hmin, hv);
            f[i] = i == 0 ? hv : min(hv, f[i - 1] + c);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            hmin = min(hmin, __shfl_xor_sync(0xffffffffu, hmin, o));
        // forward carry: min-plus scan of the blocks' end values
        int32_t A = f[LPL - 1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, A, o);
            if (lane >= o)
                A = min(A, t + c * LPL * o);
        }
        const int32_t cin = __shfl_up_sync(0xffffffffu, A, 1);
        if (lane > 0) {
#pragma unroll
            for (int i = 0; i < LPL; ++i)
                f[i] = min(f[i], cin + c * (i + 1));
        }
        // backward pass, then the carry from the blocks to the right
#pragma unroll
        for (int i = LPL - 2; i >= 0; --i)
            f[i] = min(f[i], f[i + 1] + c);
        int32_t B = f[0];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_down_sync(0xffffffffu, B, o);
            if (lane + o < 32)
                B = min(B, t + c * LPL * o);
        }
        const int32_t cout = __shfl_down_sync(0xffffffffu, B, 1);
        if (lane < 31) {
#pragma unroll
            for (int i = 0; i < LPL; ++i)
                f[i] = min(f[i], cout + c * (LPL - i));
        }
        // cap at min + Ts and shift to minimum 0
#pragma unroll
        for (int i = 0; i < LPL; ++i)
            f[i] = min(f[i] - hmin, a.ts);
        const int xq = x + dx[k], yq = y + dy[k];
        st_u16<LPL>(a.msg + wslot(a.color ^ 1, opp[k], yq, xq >> 1, a.h, a.wh) * a.Lp + d0, f);
    }
}

// --------------------------------------------------------------------------
// labels and read-out

struct WLabelArgs {
    const int32_t *cost;
    const uint16_t *msg;
    uint8_t *labels;
    int labels_pitch, w, h, wh, L, Lp;
};

// d* = argmin_d D0(d) + the in-frame incoming messages, smallest d on ties;
// one warp per pixel of either colour.
template <int LPL>
__global__ void __launch_bounds__(kWThreads) k_wlabels(WLabelArgs a)
{
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const unsigned wid = (blockIdx.x * kWThreads + threadIdx.x) >> 5;
    if (wid >= 2u * (unsigned)a.h * (unsigned)a.wh)
        return;
    const int c = (int)(wid / ((unsigned)a.h * (unsigned)a.wh));
    const unsigned r = wid - (unsigned)c * a.h * a.wh;
    const int y = (int)(r / (unsigned)a.wh), xh = (int)(r % (unsigned)a.wh);
    const int x = 2 * xh + ((c + y) & 1);
    if (x >= a.w)
        return;
    const bool has[4] = {x > 0, x < a.w - 1, y > 0, y < a.h - 1};
    const int d0 = lane * LPL;
    int32_t b[LPL];
    ld_i32<LPL>(a.cost + ((size_t)c * a.h * a.wh + (size_t)y * a.wh + xh) * a.Lp + d0, b);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (!has[k])
            continue;
        int32_t m[LPL];
        ld_u16<LPL>(a.msg + wslot(c, k, y, xh, a.h, a.wh) * a.Lp + d0, m);
#pragma unroll
        for (int i = 0; i < LPL; ++i)
            b[i] += m[i];
    }
    int32_t best = 0x7FFFFFFF, bestd = 0;
#pragma unroll
    for (int i = 0; i < LPL; ++i)
        if (d0 + i < a.L && b[i] < best) {
            best = b[i];
            bestd = d0 + i;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int32_t ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int32_t od = __shfl_xor_sync(0xffffffffu, bestd, o);
        if (ob < best || (ob == best && od < bestd)) {
            best = ob;
            bestd = od;
        }
    }
    if (lane == 0 && chk(a.labels + (size_t)y * a.labels_pitch + x, 1, kSiteLabel))
        a.labels[(size_t)y * a.labels_pitch + x] = (uint8_t)bestd;
}

struct WExportArgs {
    const uint16_t *msg;
    int32_t *out;
    int w, h, wh, L, Lp;
};

__global__ void k_wexport(WExportArgs a)
{
    pdl_begin();
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)4 * a.h * a.w * a.L)
        return;
    const int d = (int)(idx % (unsigned)a.L);
    const size_t px = idx / (unsigned)a.L;
    const int x = (int)(px % (unsigned)a.w);
    const int y = (int)((px / (unsigned)a.w) % (unsigned)a.h);
    const int k = (int)(px / ((size_t)a.w * a.h));
    const bool has = k == 0 ? x > 0 : k == 1 ? x < a.w - 1 : k == 2 ? y > 0 : y < a.h - 1;
    const uint16_t *src = a.msg + wslot((x + y) & 1, k, y, x >> 1, a.h, a.wh) * a.Lp + d;
    const int32_t v = has && chk(src, 2, kSiteExport) ? (int32_t)*src : 0;
    if (chk(a.out + idx, 4, kSiteExport))
        a.out[idx] = v;
}

template <typename Args>
void launch_lpl(int lpl, void (*k1)(Args), void (*k2)(Args), void (*k4)(Args), void (*k8)(Args), unsigned grid,
                cudaStream_t st, const Args &a)
{
    switch (lpl) {
    case 1: launch_pdl(k1, dim3(grid), dim3(kWThreads), st, a); break;
    case 2: launch_pdl(k2, dim3(grid), dim3(kWThreads), st, a); break;
    case 4: launch_pdl(k4, dim3(grid), dim3(kWThreads), st, a); break;
    default: launch_pdl(k8, dim3(grid), dim3(kWThreads), st, a); break;
    }
}

}  // namespace

bool bp_wide_params_ok(int w, int h, const vs_bp_params *p)
{
    if (!p || w <= 0 || h <= 0 || (long long)w * h > (1LL << 26))
        return false;
    if (p->labels < 2 || p->labels > 256 || p->levels < 1 || p->levels > kWMaxLevels)
        return false;
    if (p->iters < 1 || p->iters > 1000 || p->iters_per_tile < 0 || p->iters_per_tile > 64)
        return false;
    if (p->data_trunc < 0 || p->smooth_slope < 0 || p->smooth_trunc < 0 || p->smooth_trunc > 65535)
        return false;
    return ((long long)p->data_trunc << (2 * (p->levels - 1))) <= (1LL << 28);
}

size_t bp_wide_workspace_size(int w, int h, const vs_bp_params *p)
{
    return bp_wide_params_ok(w, h, p) ? wide_layout(w, h, p).total : 0;
}

size_t bp_wide_status_offset(int w, int h, const vs_bp_params *p)
{
    return wide_layout(w, h, p).status_off;
}

void bp_wide_run(const uint8_t *left, const uint8_t *right, int w, int h, int pitch, const vs_bp_params *p,
                 uint8_t *labels, int labels_pitch, uint8_t *ws, cudaStream_t st, size_t check_shrink)
{
    const WideLayout lay = wide_layout(w, h, p);
    if (check_shrink != kCheckKeepRanges)
        check_ranges(st, {{left, (size_t)(h - 1) * pitch + w}, {right, (size_t)(h - 1) * pitch + w},
                          {labels, (size_t)(h - 1) * labels_pitch + w}, {ws, lay.total}},
                     check_shrink);
    {
        WCost0Args a{left, right, pitch, w, h, lay.wh[0], lay.L, lay.Lp, p->data_trunc,
                     reinterpret_cast<int32_t *>(ws + lay.cost_off[0]), reinterpret_cast<int *>(ws + lay.status_off)};
        const size_t n = (size_t)2 * h * lay.wh[0] * lay.Lp;
        const int slot = prof_begin(kProfBpOther, st);
        launch_pdl(k_wcost0, dim3((unsigned)((n + 255) / 256)), dim3(256), st, a);
        prof_end(slot, st);
        note_launch();
    }
    for (int l = 1; l < lay.levels; ++l) {
        WCostDownArgs a{reinterpret_cast<const int32_t *>(ws + lay.cost_off[l - 1]),
                        reinterpret_cast<int32_t *>(ws + lay.cost_off[l]),
                        lay.w[l - 1], lay.h[l - 1], lay.wh[l - 1], lay.w[l], lay.h[l], lay.wh[l], lay.L, lay.Lp};
        const size_t n = (size_t)2 * lay.h[l] * lay.wh[l] * lay.Lp;
        const int slot = prof_begin(kProfBpOther, st);
        launch_pdl(k_wcost_down, dim3((unsigned)((n + 255) / 256)), dim3(256), st, a);
        prof_end(slot, st);
        note_launch();
    }
    const int32_t ceff = std::min(p->smooth_slope, p->smooth_trunc);   // the same V for any larger slope
    for (int l = lay.levels - 1; l >= 0; --l) {
        for (int t = 0; t < p->iters; ++t) {
            WSweepArgs a;
            a.cost = reinterpret_cast<const int32_t *>(ws + lay.cost_off[l]);
            a.msg = reinterpret_cast<uint16_t *>(ws + lay.msg_off[l]);
            a.pmsg = l + 1 < lay.levels ? reinterpret_cast<const uint16_t *>(ws + lay.msg_off[l + 1]) : nullptr;
            a.w = lay.w[l];
            a.h = lay.h[l];
            a.wh = lay.wh[l];
            a.pw = l + 1 < lay.levels ? lay.w[l + 1] : 0;
            a.ph = l + 1 < lay.levels ? lay.h[l + 1] : 0;
            a.pwh = l + 1 < lay.levels ? lay.wh[l + 1] : 0;
            a.Lp = lay.Lp;
            a.color = t & 1;
            a.from_parent = t == 0 && l + 1 < lay.levels;
            a.zero_in = t == 0 && l + 1 == lay.levels;
            a.materialize = t == 0 && p->iters == 1;
            a.c = ceff;
            a.ts = p->smooth_trunc;
            const unsigned warps = (unsigned)lay.h[l] * (unsigned)lay.wh[l];
            const unsigned grid = (warps * 32u + kWThreads - 1) / kWThreads;
            const int slot = prof_begin(l == 0 ? kProfSweepL0 : kProfSweepCoarse, st);
            launch_lpl<WSweepArgs>(lay.lpl, k_wsweep<1>, k_wsweep<2>, k_wsweep<4>, k_wsweep<8>, grid, st, a);
            prof_end(slot, st);
            note_launch();
        }
    }
    WLabelArgs la{reinterpret_cast<const int32_t *>(ws + lay.cost_off[0]),
                  reinterpret_cast<const uint16_t *>(ws + lay.msg_off[0]), labels, labels_pitch, w, h, lay.wh[0],
                  lay.L, lay.Lp};
    const unsigned warps = 2u * (unsigned)h * (unsigned)lay.wh[0];
    const int slot = prof_begin(kProfBpOther, st);
    launch_lpl<WLabelArgs>(lay.lpl, k_wlabels<1>, k_wlabels<2>, k_wlabels<4>, k_wlabels<8>,
                           (warps * 32u + kWThreads - 1) / kWThreads, st, la);
    prof_end(slot, st);
    note_launch();
}

void bp_wide_export(const uint8_t *ws, int w, int h, const vs_bp_params *p, int32_t *out, cudaStream_t st)
{
    const WideLayout lay = wide_layout(w, h, p);
    check_ranges(st, {{ws, lay.total}, {out, (size_t)16 * h * w * p->labels}});
    WExportArgs a{reinterpret_cast<const uint16_t *>(ws + lay.msg_off[0]), out, w, h, lay.wh[0], lay.L, lay.Lp};
    const size_t n = (size_t)4 * h * w * lay.L;
    launch_pdl(k_wexport, dim3((unsigned)((n + 255) / 256)), dim3(256), st, a);
    note_launch();
}

#ifdef VS_CHECKED
unsigned long long bp_wide_check_take(unsigned long long *addr) { return check_take(addr); }
void bp_wide_check_ranges(cudaStream_t st, const std::vector<std::pair<const void *, size_t>> &bufs)
{
    check_ranges_list(st, bufs);
}
#endif

}  // namespace vs
