// Eq. 1: hierarchical loopy min-sum belief propagation on the downsampled
// grey pair, red-black schedule, truncated-linear smoothness.
//
// Data layout (all in the caller's workspace, every array 256-byte aligned):
//   every level splits its pixels by colour c = (x + y) & 1, so that one
//   iteration reads one colour and writes the other, both contiguously:
//     cost_l[c][y][x >> 1][Lp]     uint8 while data_trunc * 4^l <= 255, else uint16
//     msg_l [c][k][y][x >> 1][Lp]  uint8 incoming message from direction k
//   with k = 0 left, 1 right, 2 up, 3 down and Lp = labels rounded up to one
//   of the compiled sizes 16, 32, 48, 64, 96, 128.  Within a row the slots
//   are interleaved in groups of 16: the 16-byte piece p (16 labels in bytes,
//   8 in uint16) of the 16 slots of a group lies in one 256-byte block, so a
//   warp reading or writing piece p of 16 consecutive slots touches whole
//   32-byte sectors (slot_base below).
//   Messages live in [0, smooth_trunc] after normalisation, so 8 bits hold
//   them exactly; all message arithmetic is integer.
//
// Kernels per call: k_cost01 (level-0 data term and its level-1 sums; it
// also resets the call's status word and zeroes the border message slots
// of levels 0 and 1), k_cost_down per further coarse level, one sweep per
// iteration and level (k_bp_sweep, k_bp_sweep_split on small levels,
// k_bp_sweep_staged on large byte-lane levels) or, where iters_per_tile
// asks for it or the autotuner measured it faster, k_bp_fused launches of
// several iterations each on shared-memory tiles, and k_bp_labels_bytes /
// k_bp_labels for the colour the last sweep did not label.
//
// k_bp_sweep: two threads per active pixel, each owning a pair of outgoing
// directions (left/right or up/down); the two pairs of a CTA's 64 pixels run
// in different warps (threads 0-63 left/right, 64-127 up/down), so a warp's
// choice of operands is fixed at compile time.  A thread packs the pair into the two
// 16-bit halves of 32-bit words, one word per label, and runs the O(L)
// distance transform of the truncated-linear cost (forward pass, backward
// pass, cap at min + Ts, shift to min 0) for both directions at once with
// packed 16-bit add-min (DPX) operations; the forward results stay in
// registers.  All lane values stay below 2^15 (ABI limits), so the packed
// adds never carry across lanes and the signed form is exact too.
#include "vs_bp_wide.cuh"
#include "vs_check.cuh"
#include "vs_common.cuh"
#include "vs_tcgen05.cuh"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

namespace vs {
namespace {

constexpr int kMaxLevels = 8;
constexpr uint32_t kBig2 = 0x7FFF7FFFu;   // "label does not exist" in both halves
constexpr int kSweepThreads = 128;        // 64 pixels x 2 direction pairs per CTA

struct BpLayout {
    int wide;                  // the general path (vs_bp_wide.cu) runs this pair; only w[0], h[0],
                               // L, levels, status_off and total are set then
    int L, Lp, levels;
    int w[kMaxLevels], h[kMaxLevels], wh[kMaxLevels];
    int wg[kMaxLevels];        // 16-slot groups per row
    int cost_u8[kMaxLevels];   // level cost fits a byte: data_trunc * 4^l <= 255
    int bytes[kMaxLevels];     // level belief sums fit a byte: + 4 smooth_trunc <= 255
    size_t cost_off[kMaxLevels], msg_off[kMaxLevels];
    size_t msg_bytes[kMaxLevels];
    size_t fused_off;          // second message buffer of the fused sweeps (0 bytes when none)
    size_t fused_bytes;
    int fused_min_level;       // levels >= this one may run fused sweeps (levels: none)
    size_t status_off;         // int: VS_OK, or VS_ETIMEOUT from a kernel of the last call
    size_t total;
};

// Parameters of the byte-message kernels in this file; anything else that
// bp_wide_params_ok accepts runs the general path.
bool narrow_ok(int w, int h, const vs_bp_params *p)
{
    if (!p || w <= 0 || h <= 0)
        return false;
    if (p->labels < 2 || p->labels > 128 || p->levels < 1 || p->levels > kMaxLevels)
        return false;
    if (p->iters < 1 || p->iters > 1000)
        return false;
    if (p->iters_per_tile < 0 || p->iters_per_tile > 64)
        return false;
    if (p->data_trunc < 0 || p->data_trunc > 127 || p->smooth_slope < 0 || p->smooth_trunc < 0 ||
        p->smooth_trunc > 127)
        return false;
    const long long coarse = (long long)p->data_trunc << (2 * (p->levels - 1));
    if (coarse + 4LL * p->smooth_trunc > 32767)
        return false;
    if ((long long)w * h > (1LL << 26))   // keeps every thread index below 2^31
        return false;
    return true;
}

bool params_ok(int w, int h, const vs_bp_params *p)
{
    return narrow_ok(w, h, p) || bp_wide_params_ok(w, h, p);
}

BpLayout make_layout(int w, int h, const vs_bp_params *p)
{
    BpLayout lay;
    lay.wide = !narrow_ok(w, h, p);
    if (lay.wide) {
        lay.L = p->labels;
        lay.Lp = 0;
        lay.levels = p->levels;
        lay.w[0] = w;
        lay.h[0] = h;
        lay.fused_min_level = p->levels;
        lay.fused_bytes = 0;
        lay.status_off = bp_wide_status_offset(w, h, p);
        lay.total = bp_wide_workspace_size(w, h, p);
        return lay;
    }
    lay.L = p->labels;
    // padded label count: one of the compiled sizes 16, 32, 48, 64, 96, 128
    lay.Lp = p->labels <= 64 ? (p->labels + 15) / 16 * 16 : (p->labels <= 96 ? 96 : 128);
    lay.levels = p->levels;
    size_t off = 0;
    for (int l = 0; l < p->levels; ++l) {
        lay.w[l] = l == 0 ? w : (lay.w[l - 1] + 1) / 2;
        lay.h[l] = l == 0 ? h : (lay.h[l - 1] + 1) / 2;
        lay.wh[l] = (lay.w[l] + 1) / 2;
        lay.wg[l] = (lay.wh[l] + 15) / 16;
        const size_t slots = (size_t)2 * lay.h[l] * lay.wg[l] * 16;   // both colours, rows padded to groups
        const long long cmax = (long long)p->data_trunc << (2 * l);
        lay.cost_u8[l] = l == 0 || cmax <= 255;
        lay.bytes[l] = lay.cost_u8[l] && cmax + 4LL * p->smooth_trunc <= 255;
        lay.cost_off[l] = off;
        off = align_up(off + slots * lay.Lp * (lay.cost_u8[l] ? 1 : 2), 256);
        lay.msg_off[l] = off;
        lay.msg_bytes[l] = slots * 4 * lay.Lp;
        off = align_up(off + lay.msg_bytes[l], 256);
    }
    // iters_per_tile 1: every sweep unfused; >= 2: fused on every level; 0
    // (automatic): fused only where chosen, on the coarse levels
    lay.fused_min_level = p->iters_per_tile == 1 ? p->levels : (p->iters_per_tile >= 2 ? 0 : 1);
    lay.fused_bytes = 0;
    for (int l = lay.fused_min_level; l < p->levels; ++l)
        lay.fused_bytes = std::max(lay.fused_bytes, lay.msg_bytes[l]);
    lay.fused_off = off;
    off = align_up(off + lay.fused_bytes, 256);
    lay.status_off = off;
    off = align_up(off + sizeof(int), 256);
    lay.total = off;
    return lay;
}

// Byte offset of piece 0 of slot (row, xh) in an array with wg groups per
// row and np 16-byte pieces per slot; piece p lies kPieceStride * p further.
constexpr int kPieceStride = 256;
__host__ __device__ __forceinline__ size_t slot_base(int row, int xh, int wg, int np)
{
    return ((((size_t)row * wg + (xh >> 4)) * np) * 16 + (xh & 15)) * 16;
}
// n / d for 0 <= n < 2^31 and a divisor fixed for the launch, as one wide
// multiply and a shift instead of a division sequence.  With l = ceil(log2 d),
// p = 31 + l and m = ceil(2^p / d): 0 <= m d - 2^p < d <= 2^l, so
// n m / 2^p = n / d + n (m d - 2^p) / (d 2^p) lies in [n / d, n / d + 1 / d)
// for every n < 2^31 and its floor is floor(n / d) (Granlund and Montgomery,
// division by invariant integers using multiplication, 1994); m < 2^32.
struct FastDiv {
    uint32_t m, p;
};
inline FastDiv fast_div(uint32_t d)
{
    d = d ? d : 1u;   // every divisor here counts slots, groups or rows of a level: never 0
    uint32_t l = 0;
    while ((1ull << l) < d)
        ++l;
    const uint32_t p = 31 + l;
    return FastDiv{(uint32_t)(((1ull << p) + d - 1) / d), p};
}
__device__ __forceinline__ uint32_t div_by(uint32_t n, const FastDiv &f)
{
    return (uint32_t)(((uint64_t)n * f.m) >> f.p);
}

// Every global 16-byte piece goes through these (bounds-checked in the
// checked build; shared-memory copies use them too, and chk() accepts none
// of those addresses, so the sweeps that read shared memory pass SMEM to
// sweep_pixel and load directly).
__device__ __forceinline__ uint4 ld_piece(const uint8_t *base, int p)
{
    const uint8_t *q = base + (size_t)p * kPieceStride;
    if (!chk(q, 16, kSitePieceLoad))
        return make_uint4(0, 0, 0, 0);
    return *reinterpret_cast<const uint4 *>(q);
}
__device__ __forceinline__ void st_piece(uint8_t *base, int p, const uint4 &v)
{
    uint8_t *q = base + (size_t)p * kPieceStride;
    if (chk(q, 16, kSitePieceStore))
        *reinterpret_cast<uint4 *>(q) = v;
}
// The same without the check, for shared memory.
__device__ __forceinline__ uint4 ld_piece_smem(const uint8_t *base, int p)
{
    return *reinterpret_cast<const uint4 *>(base + (size_t)p * kPieceStride);
}

// The level being swept reads and rewrites its message arrays every
// iteration; marking those accesses evict-last keeps more of them in L2
// (a per-instruction hint, no device setting).
__device__ __forceinline__ uint64_t l2_evict_last_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint4 ld_piece_keep(const uint8_t *base, int p, uint64_t pol)
{
    uint4 v;
    const uint8_t *ptr = base + (size_t)p * kPieceStride;
    if (!chk(ptr, 16, kSitePieceLoad))
        return make_uint4(0, 0, 0, 0);
    asm volatile("ld.global.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_piece_keep(uint8_t *base, int p, const uint4 &v, uint64_t pol)
{
    uint8_t *ptr = base + (size_t)p * kPieceStride;
    if (!chk(ptr, 16, kSitePieceStore))
        return;
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(ptr), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
}

// ---------------------------------------------------------------------------
// data term

struct Cost01Args {
    const uint8_t *left, *right;
    int pitch, L, Lp, Td;
    int w0, h0, wg0;        // level 0
    int w1, h1, wg1;        // level 1 (its size even when levels == 1)
    uint8_t *cost0;
    uint8_t *cost1;         // null when there is no level 1
    int cost1_u8;
    int *status;            // reset to VS_OK: the first kernel of every call
    uint8_t *msg0, *msg1;   // levels 0 and 1 (msg1 null without level 1): the incoming
                            // slots no neighbour ever writes are zeroed
};

// D0(x, y, d) = min(|IL(x,y) - IR(x-d,y)|, Td), Td where x - d < 0, 0 on
// padding labels, for labels 16 j .. 16 j + 15 of pixel (x, y); also added
// into acc (8 words of 2 x u16, label k in half k & 1 of word k >> 1).
// Byte loads: the left edge, the right edge, the last label chunk.
__device__ __forceinline__ uint4 cost0_chunk_slow(const Cost01Args &a, const uint8_t *rowL, const uint8_t *rowR,
                                                  int x, int j, uint32_t (&acc)[8])
{
    const int il = chk(rowL + x, 1, kSiteImage) ? __ldg(rowL + x) : 0;
    uint32_t wv[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int d = 16 * j + i;
        int v = 0;
        if (d < a.L) {
            v = a.Td;
            if (x - d >= 0 && chk(rowR + x - d, 1, kSiteImage))
                v = min(abs(il - (int)__ldg(rowR + x - d)), a.Td);
        }
        wv[i >> 2] |= (uint32_t)v << (8 * (i & 3));
        acc[i >> 1] += (uint32_t)v << (16 * (i & 1));
    }
    return make_uint4(wv[0], wv[1], wv[2], wv[3]);
}

// Level-0 data term and its level-1 2x2 sums in one pass.  A thread owns the
// level-1 pixel (X, Y) and 16 labels; its children (2X+i, 2Y+j) have colour
// (i+j) & 1 and level-0 column slot X, so a warp of 32 consecutive X writes
// whole 256-byte blocks on both levels.  Inside the frame the 17 right-image
// bytes that the two children of a row need are 5 aligned words, shifted into
// place with funnel shifts; per 4 labels one byte permute reverses them, one
// SIMD absolute difference forms |IL - IR|, and the truncation runs on 2 x u16
// lanes (no byte-lane minimum in hardware).
__device__ __forceinline__ void cost01_pixel(const Cost01Args &a, int X, int Y, int j, int chunks);

// Block (32, Lp / 16): threadIdx.y is the label chunk; grid (X tiles of 32,
// rows), the rows strided by gridDim.y (at most 65535).
__global__ void __launch_bounds__(256) k_cost01(Cost01Args a)
{
    pdl_begin();
    const int chunks = a.Lp / 16;
    if ((blockIdx.x | blockIdx.y | threadIdx.x | threadIdx.y) == 0 && chk(a.status, 4, kSiteStatus))
        *a.status = VS_OK;
    const int j = (int)threadIdx.y;
    const int X = 32 * (int)blockIdx.x + (int)threadIdx.x;
    if (X >= a.w1)
        return;
    for (int Y = (int)blockIdx.y; Y < a.h1; Y += (int)gridDim.y)
        cost01_pixel(a, X, Y, j, chunks);
}

// The level-1 pixel (X, Y) and its four level-0 children, labels 16 j ..
// 16 j + 15.
__device__ __forceinline__ void cost01_pixel(const Cost01Args &a, int X, int Y, int j, int chunks)
{
    uint32_t acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const uint32_t td2 = (uint32_t)a.Td * 0x00010001u;
    const int s0 = 2 * X - 16 * j - 15;   // first right-image column of the row window
    // fast: both children in the frame, a full label chunk, and the 20 bytes
    // of the aligned words inside the row
    const bool fast = 2 * X + 1 < a.w0 && 16 * j + 15 < a.L && s0 >= 3 && s0 + 20 <= a.w0;
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
        const int yf = 2 * Y + jj;
        if (yf >= a.h0)
            break;
        const uint8_t *rowL = a.left + (size_t)yf * a.pitch;
        const uint8_t *rowR = a.right + (size_t)yf * a.pitch;
        uint4 out[2];
        if (fast) {
            // bytes s0 .. s0 + 16 of the row: W[k] = bytes s0 + 4k .. s0 + 4k + 3
            const uintptr_t addr = reinterpret_cast<uintptr_t>(rowR + s0);
            const uint32_t *q = reinterpret_cast<const uint32_t *>(addr & ~(uintptr_t)3);
            const uint32_t sh = 8u * (uint32_t)(addr & 3u);
            uint32_t w[5], W[5];
#pragma unroll
            for (int k = 0; k < 5; ++k)
                w[k] = chk(q + k, 4, kSiteImage) ? __ldg(q + k) : 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                W[k] = __funnelshift_r(w[k], w[k + 1], sh);
            W[4] = w[4] >> sh;
            const uint32_t il2 = chk(rowL + 2 * X, 2, kSiteImage)
                                     ? (uint32_t)__ldg(reinterpret_cast<const uint8_t *>(rowL + 2 * X)) |
                                           ((uint32_t)__ldg(rowL + 2 * X + 1) << 8)
                                     : 0u;
#pragma unroll
            for (int ii = 0; ii < 2; ++ii) {
                const uint32_t il4 = ((il2 >> (8 * ii)) & 0xFFu) * 0x01010101u;
                uint32_t wv[4];
#pragma unroll
                for (int qd = 0; qd < 4; ++qd) {
                    // labels 16j + 4qd + r sit at window offsets 15 + ii - 4qd - r
                    const uint32_t rev = ii == 0 ? prmt(W[3 - qd], 0u, 0x0123u) : prmt(W[3 - qd], W[4 - qd], 0x1234u);
                    const uint32_t ad = __vabsdiffu4(il4, rev);
                    const uint32_t lo = min_u16x2(prmt(ad, 0u, 0x4140u), td2);
                    const uint32_t hi = min_u16x2(prmt(ad, 0u, 0x4342u), td2);
                    wv[qd] = prmt(lo, hi, 0x6420u);
                    acc[2 * qd] += lo;
                    acc[2 * qd + 1] += hi;
                }
                out[ii] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
        } else {
#pragma unroll
            for (int ii = 0; ii < 2; ++ii)
                if (2 * X + ii < a.w0)
                    out[ii] = cost0_chunk_slow(a, rowL, rowR, 2 * X + ii, j, acc);
        }
#pragma unroll
        for (int ii = 0; ii < 2; ++ii) {
            const int xf = 2 * X + ii, cf = (ii + jj) & 1;
            if (xf >= a.w0)
                continue;
            st_piece(a.cost0 + slot_base(cf * a.h0 + yf, X, a.wg0, chunks), j, out[ii]);
            // incoming slots of a missing neighbour (frame border) read as 0
            const uint4 z = make_uint4(0, 0, 0, 0);
            const bool border[4] = {xf == 0, xf == a.w0 - 1, yf == 0, yf == a.h0 - 1};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (border[k])
                    st_piece(a.msg0 + slot_base((cf * 4 + k) * a.h0 + yf, X, a.wg0, chunks), j, z);
        }
    }
    if (!a.cost1)
        return;
    {
        const uint4 z = make_uint4(0, 0, 0, 0);
        const bool border[4] = {X == 0, X == a.w1 - 1, Y == 0, Y == a.h1 - 1};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (border[k])
                st_piece(a.msg1 + slot_base((((X + Y) & 1) * 4 + k) * a.h1 + Y, X >> 1, a.wg1, chunks), j, z);
    }
    const int row1 = ((X + Y) & 1) * a.h1 + Y;
    if (a.cost1_u8) {   // every sum is <= 4 Td <= 255 here
        st_piece(a.cost1 + slot_base(row1, X >> 1, a.wg1, chunks), j,
                 make_uint4(prmt(acc[0], acc[1], 0x6420u), prmt(acc[2], acc[3], 0x6420u),
                            prmt(acc[4], acc[5], 0x6420u), prmt(acc[6], acc[7], 0x6420u)));
    } else {
        uint8_t *b = a.cost1 + slot_base(row1, X >> 1, a.wg1, 2 * chunks);
        st_piece(b, 2 * j, make_uint4(acc[0], acc[1], acc[2], acc[3]));
        st_piece(b, 2 * j + 1, make_uint4(acc[4], acc[5], acc[6], acc[7]));
    }
}

struct CostDownArgs {
    const void *fine;      // level l-1, uint8 or uint16
    void *coarse;          // level l, uint8 (when the sums fit) or uint16
    int fine_is_u8, coarse_is_u8;
    int wf, hf, wgf;       // fine dims (width, height, slot groups per row)
    int wc, hc, wgc;       // coarse dims
    int Lp;
    FastDiv div_chunks, div_wgc, div_hc;   // by Lp / 8, wgc, hc
};

// Coarse data term: the sum over the in-frame 2x2 children.  Child
// (2x+i, 2y+j) has colour (i+j)&1 and column slot x.  8 labels per thread.
__global__ void k_cost_down(CostDownArgs a)
{
    // threads in memory order: (row, group, 8-label chunk j, slot in group)
    const unsigned chunks = (unsigned)a.Lp / 8u;
    const int np16 = a.Lp / 16;
    const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2u * a.hc * a.wgc * chunks * 16u)
        return;
    const int lane = (int)(idx & 15u);
    unsigned t = idx >> 4;
    const unsigned t1 = div_by(t, a.div_chunks);
    const int j = (int)(t - t1 * chunks);
    t = t1;
    const unsigned row = div_by(t, a.div_wgc);
    const int g = (int)(t - row * (unsigned)a.wgc);
    const int c = (int)div_by(row, a.div_hc);
    const int y = (int)(row - (unsigned)c * (unsigned)a.hc);
    const int xh = 16 * g + lane;
    const int x = 2 * xh + ((c + y) & 1);
    if (x >= a.wc)
        return;
    pdl_begin();   // the index work above overlaps the previous kernel's last wave
    uint32_t acc[4] = {0, 0, 0, 0};   // 8 x u16
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
#pragma unroll
        for (int ii = 0; ii < 2; ++ii) {
            const int xf = 2 * x + ii, yf = 2 * y + jj;
            if (xf >= a.wf || yf >= a.hf)
                continue;
            const int cf = (ii + jj) & 1;   // child slot: row cf*hf + yf, column slot x
            const int frow = cf * a.hf + yf;
            if (a.fine_is_u8) {
                const uint8_t *b = reinterpret_cast<const uint8_t *>(a.fine) + slot_base(frow, x, a.wgf, np16);
                const uint8_t *q = b + (j >> 1) * kPieceStride + (j & 1) * 8;
                const uint2 v = chk(q, 8, kSiteCostWord) ? *reinterpret_cast<const uint2 *>(q) : make_uint2(0, 0);
                // widen 8 bytes to 8 u16 lanes
                acc[0] += prmt(v.x, 0, 0x4140);
                acc[1] += prmt(v.x, 0, 0x4342);
                acc[2] += prmt(v.y, 0, 0x4140);
                acc[3] += prmt(v.y, 0, 0x4342);
            } else {
                const uint8_t *b = reinterpret_cast<const uint8_t *>(a.fine) + slot_base(frow, x, a.wgf, 2 * np16);
                const uint4 v = ld_piece(b, j);
                acc[0] += v.x;
                acc[1] += v.y;
                acc[2] += v.z;
                acc[3] += v.w;
            }
        }
    }
    uint8_t *cb = reinterpret_cast<uint8_t *>(a.coarse);
    if (a.coarse_is_u8) {   // every lane is <= 255 here: narrow back to bytes
        uint8_t *b = cb + slot_base((int)row, xh, a.wgc, np16) + (j >> 1) * kPieceStride + (j & 1) * 8;
        if (chk(b, 8, kSiteCostWord))
            *reinterpret_cast<uint2 *>(b) = make_uint2(prmt(acc[0], acc[1], 0x6420u), prmt(acc[2], acc[3], 0x6420u));
    } else {
        st_piece(cb + slot_base((int)row, xh, a.wgc, 2 * np16), j, make_uint4(acc[0], acc[1], acc[2], acc[3]));
    }
}

// ---------------------------------------------------------------------------
// message sweep

struct SweepArgs {
    const void *cost;       // this level
    uint8_t *msg;           // this level
    const uint8_t *pmsg;    // parent level (coarse-to-fine initialisation)
    int w, h, wh, wg, L;
    int pw, ph, pwh, pwg;
    int color;              // active colour, = t & 1
    int from_parent;        // incoming = parent's messages (first iteration, not coarsest)
    int zero_in;            // incoming = 0 (first iteration of the coarsest level)
    int materialize;        // also store the incoming used into the own slots
    uint32_t c2, ts2;       // (c, c) and (Ts, Ts) packed
    uint32_t k256;          // 256 as a run-time value: x + y * k256 stays one integer multiply-add
    FastDiv div_rowslots;   // by 16 wg, the slots of a padded row
    uint8_t *labels;        // last level-0 iteration: labels of the active colour
    int labels_pitch;
    int *status;            // set to VS_ETIMEOUT by a kernel that gives up a bounded wait
    int zero_border;        // this level's never-written incoming slots hold 0 (levels 0, 1)
    int withhold_copies;    // test aid: the staged sweep expects its tile bytes but issues no copy
};

// Byte i of word a in the low half and byte i of word b in the high half,
// each zero-extended to 16 bits (the bytes are < 128, so sign fill is 0).
__device__ __forceinline__ uint32_t pair_bytes(uint32_t a, uint32_t b, int i)
{
    const uint32_t sel = (uint32_t)i | ((uint32_t)(8 | i) << 4) | ((uint32_t)(4 + i) << 8) |
                         ((uint32_t)(12 + i) << 12);
    return prmt(a, b, sel);
}

template <typename CostT>
struct CostChunk;

template <>
struct CostChunk<uint8_t> {
    uint4 v;
    __device__ __forceinline__ void load(const uint8_t *base, int j) { v = ld_piece(base, j); }
    __device__ __forceinline__ void load_smem(const uint8_t *base, int j) { v = ld_piece_smem(base, j); }
    // shared-memory copy with `ps` pieces between consecutive pieces of a slot
    __device__ __forceinline__ void load_s(const uint4 *base, int j, int ps) { v = base[j * ps]; }
    __device__ __forceinline__ uint32_t word(int wi) const { return (&v.x)[wi]; }
    __device__ __forceinline__ void zero() { v = make_uint4(0, 0, 0, 0); }
    __device__ __forceinline__ uint32_t dup(int i) const
    {
        // byte i & 3 zero-extended into both 16-bit halves (byte 4 of {0:wv} is 0)
        const uint32_t wv = (&v.x)[i >> 2];
        const uint32_t b = (uint32_t)(i & 3);
        return prmt(wv, 0u, b | (4u << 4) | (b << 8) | (4u << 12));
    }
};

template <>
struct CostChunk<uint16_t> {
    uint4 v0, v1;
    __device__ __forceinline__ void load(const uint8_t *base, int j)
    {
        v0 = ld_piece(base, 2 * j);
        v1 = ld_piece(base, 2 * j + 1);
    }
    __device__ __forceinline__ void load_smem(const uint8_t *base, int j)
    {
        v0 = ld_piece_smem(base, 2 * j);
        v1 = ld_piece_smem(base, 2 * j + 1);
    }
    __device__ __forceinline__ void load_s(const uint4 *base, int j, int ps)
    {
        v0 = base[2 * j * ps];
        v1 = base[(2 * j + 1) * ps];
    }
    __device__ __forceinline__ uint32_t word(int) const { return 0u; }   // byte-lane path never uses 16-bit costs
    __device__ __forceinline__ void zero()
    {
        v0 = make_uint4(0, 0, 0, 0);
        v1 = v0;
    }
    __device__ __forceinline__ uint32_t dup(int i) const
    {
        const uint32_t wv = i < 8 ? (&v0.x)[i >> 1] : (&v1.x)[(i - 8) >> 1];
        return prmt(wv, wv, (i & 1) ? 0x3232u : 0x1010u);
    }
};

// BYTES: level 0 with data_trunc + 4 smooth_trunc <= 255, so the belief sum
// of four labels fits four byte lanes of one 32-bit add.  FULL: labels == LP,
// no padding labels to mask.
// LABELS: the last level-0 iteration also writes the labels of its active
// pixels (their incoming messages are final): argmin_d of the belief sum S(d)
// taken as the minimum of S(d) * 256 + d, so ties go to the smallest d.
// PRELOAD: issue every load of the pixel before the arithmetic (levels too
// small to fill the GPU, where one thread's latency is the sweep's time).
// The sweep of one level-iteration for the CTA `block` of a launch; the
// plain kernel passes blockIdx.x, the batched kernel its position within
// its job.
template <int LP, typename CostT, bool BYTES, bool FULL, bool LABELS, bool PRELOAD, bool SMEM, int PAIR, typename Dsts>
__device__ __forceinline__ void sweep_pixel(const SweepArgs &a, int x, int y, const uint8_t *const (&in)[4],
                                            const bool (&use)[4], const uint8_t *cost, uint8_t *own,
                                            const Dsts &dsts);

// Where pixel (x, y) sends the two messages of direction pair PAIR: A = the
// left / up neighbour's slot, B = the right / down neighbour's, in the other
// colour's arrays; null where the neighbour is missing.
template <int LP, int PAIR>
__device__ __forceinline__ void sweep_dsts(const SweepArgs &a, int x, int y, const bool (&has)[4], uint8_t *&dstA,
                                           uint8_t *&dstB)
{
    const int ncolor = a.color ^ 1;
    dstA = dstB = nullptr;
    if (PAIR == 0) {
        if (has[0])
            dstA = a.msg + slot_base((ncolor * 4 + 1) * a.h + y, (x - 1) >> 1, a.wg, LP / 16);
        if (has[1])
            dstB = a.msg + slot_base((ncolor * 4 + 0) * a.h + y, (x + 1) >> 1, a.wg, LP / 16);
    } else {
        if (has[2])
            dstA = a.msg + slot_base((ncolor * 4 + 3) * a.h + (y - 1), x >> 1, a.wg, LP / 16);
        if (has[3])
            dstB = a.msg + slot_base((ncolor * 4 + 2) * a.h + (y + 1), x >> 1, a.wg, LP / 16);
    }
}

template <int LP, typename CostT, bool BYTES, bool FULL, bool LABELS, bool PRELOAD>
__device__ __forceinline__ void sweep_body(const SweepArgs &a, unsigned block)
{
    // slots over rows padded to whole 16-slot groups; direction pair by warp
    constexpr int kSlots = kSweepThreads / 2;
    const int pair = (int)(threadIdx.x / kSlots);
    const unsigned slot = block * kSlots + (threadIdx.x & (kSlots - 1));
    const unsigned rowslots = 16u * (unsigned)a.wg;
    if (slot >= (unsigned)a.h * rowslots)
        return;
    const int y = (int)div_by(slot, a.div_rowslots);
    const int xh = (int)(slot - (unsigned)y * rowslots);
    const int x = 2 * xh + ((a.color + y) & 1);
    if (x >= a.w)
        return;
    const bool has[4] = {x > 0, x < a.w - 1, y > 0, y < a.h - 1};

    // where the incoming messages of this pixel are read from
    const uint8_t *in[4];
    {
        if (a.from_parent) {
            const int px = x >> 1, py = y >> 1, pc = (px + py) & 1;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                in[k] = a.pmsg + slot_base((pc * 4 + k) * a.ph + py, px >> 1, a.pwg, LP / 16);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                in[k] = a.msg + slot_base((a.color * 4 + k) * a.h + y, xh, a.wg, LP / 16);
        }
    }
    // a slot is read only if the neighbour exists here and, when the messages
    // come from the parent, the parent has that neighbour too (otherwise the
    // parent never received from it and its message is 0)
    bool use[4];
    {
        const int px = x >> 1, py = y >> 1;
        const bool phas[4] = {px > 0, px < a.pw - 1, py > 0, py < a.ph - 1};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            use[k] = has[k] && !a.zero_in && (!a.from_parent || phas[k]);
    }
    const uint8_t *cost = reinterpret_cast<const uint8_t *>(a.cost) +
                          slot_base(a.color * a.h + y, xh, a.wg, (LP / 16) * (int)sizeof(CostT));
    uint8_t *own = a.msg + slot_base(a.color * 4 * a.h + y, xh, a.wg, LP / 16);
    // only now wait for the previous kernel: the index work above overlaps
    // its last wave (nothing above reads memory it writes)
    pdl_begin();
    if (pair == 0)
        sweep_pixel<LP, CostT, BYTES, FULL, LABELS, PRELOAD, false, 0>(
            a, x, y, in, use, cost, own, [&](uint8_t *&A, uint8_t *&B) { sweep_dsts<LP, 0>(a, x, y, has, A, B); });
    else
        sweep_pixel<LP, CostT, BYTES, FULL, LABELS, PRELOAD, false, 1>(
            a, x, y, in, use, cost, own, [&](uint8_t *&A, uint8_t *&B) { sweep_dsts<LP, 1>(a, x, y, has, A, B); });
}

// The message update of one pixel for one direction pair (PAIR 0: left /
// right, 1: up / down) once the sources are known: in[k] = piece 0 of the
// incoming message from direction k (read only where use[k]), cost = piece 0
// of the data term, own = this pixel's slot of direction 0 (for
// materialize), dsts(A, B) sets the two destination slots (called after the
// forward pass).  SMEM: the sources are a shared-memory copy (plain loads,
// no L2 hint).
template <int LP, typename CostT, bool BYTES, bool FULL, bool LABELS, bool PRELOAD, bool SMEM, int PAIR, typename Dsts>
__device__ __forceinline__ void sweep_pixel(const SweepArgs &a, int x, int y, const uint8_t *const (&in)[4],
                                            const bool (&use)[4], const uint8_t *cost, uint8_t *own,
                                            const Dsts &dsts)
{
    constexpr int pair = PAIR;
    const size_t dir_stride = (size_t)a.h * a.wg * (LP / 16) * kPieceStride;   // bytes between directions

    constexpr int NPRE = PRELOAD ? LP / 16 : 1;
    uint4 mpre[NPRE][4];
    CostChunk<CostT> cpre[NPRE];
    if (PRELOAD) {
#pragma unroll
        for (int j = 0; j < NPRE; ++j) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mpre[j][k] = use[k] ? ld_piece(in[k], j) : make_uint4(0, 0, 0, 0);
            cpre[j].load(cost, j);
        }
    }

    const uint64_t pol = l2_evict_last_policy();
    uint32_t F[LP];
    uint32_t H2 = kBig2;
    uint32_t best_key = 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < LP / 16; ++j) {
        uint4 m[4];
        CostChunk<CostT> cc;
        if (PRELOAD) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                m[k] = mpre[PRELOAD ? j : 0][k];
            cc = cpre[PRELOAD ? j : 0];
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                m[k] = !use[k] ? make_uint4(0, 0, 0, 0) : (SMEM ? ld_piece_smem(in[k], j) : ld_piece_keep(in[k], j, pol));
            if (SMEM)
                cc.load_smem(cost, j);
            else
                cc.load(cost, j);
        }
        if (a.materialize) {
            const size_t k0 = 2 * pair;
            st_piece(own + k0 * dir_stride, j, pair ? m[2] : m[0]);
            st_piece(own + (k0 + 1) * dir_stride, j, pair ? m[3] : m[1]);
        }
        if (BYTES) {
            // four labels per word: S = D + L + R + U + D in byte lanes, then
            // h_A = S - in_A, h_B = S - in_B, interleaved and widened to
            // (h_A, h_B) 16-bit pairs
#pragma unroll
            for (int wi = 0; wi < 4; ++wi) {
                // A, B = directions 2 PAIR, 2 PAIR + 1; the other pair's two
                // incoming are summed once for both
                const uint32_t c4 = cc.word(wi);
                const uint32_t mA = (&m[2 * PAIR].x)[wi], mB = (&m[2 * PAIR + 1].x)[wi];
                const uint32_t oth = (&m[2 - 2 * PAIR].x)[wi] + (&m[3 - 2 * PAIR].x)[wi];
                const uint32_t a4 = c4 + oth + mB;
                const uint32_t b4 = c4 + oth + mA;
                const uint32_t s4 = a4 + mA;   // the belief sum (labels only)
                const uint32_t x01 = prmt(a4, b4, 0x5140u);    // A0 B0 A1 B1
                const uint32_t x23 = prmt(a4, b4, 0x7362u);    // A2 B2 A3 B3
                uint32_t wq[4] = {prmt(x01, 0u, 0x4140u), prmt(x01, 0u, 0x4342u), prmt(x23, 0u, 0x4140u),
                                  prmt(x23, 0u, 0x4342u)};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int d = 16 * j + 4 * wi + q;
                    if (LABELS && PAIR == 0 && (FULL || d < a.L))
                        best_key = min(best_key, (((s4 >> (8 * q)) & 0xFFu) << 8) | (uint32_t)d);
                    uint32_t wv = wq[q];
                    if (!FULL && d >= a.L)
                        wv = kBig2;
                    F[d] = d == 0 ? wv : __viaddmin_u16x2(F[d - 1], a.c2, wv);   // min(F + c, h)
                    H2 = min_u16x2(H2, wv);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int d = 16 * j + i;
                const int wi = i >> 2;
                const uint32_t plr = pair_bytes((&m[0].x)[wi], (&m[1].x)[wi], i & 3);
                const uint32_t pud = pair_bytes((&m[2].x)[wi], (&m[3].x)[wi], i & 3);
                const uint32_t t = plr + pud;                       // (L+U, R+D), no carry
                const uint32_t s2 = t + prmt(t, t, 0x1032u) + cc.dup(i);   // (S, S)
                if (LABELS && PAIR == 0 && (FULL || d < a.L))
                    best_key = min(best_key, ((s2 & 0xFFFFu) << 8) | (uint32_t)d);
                uint32_t wv = s2 - (pair ? pud : plr);              // (h_A, h_B)
                if (!FULL && d >= a.L)
                    wv = kBig2;
                F[d] = d == 0 ? wv : __viaddmin_u16x2(F[d - 1], a.c2, wv);   // min(F + c, h)
                H2 = min_u16x2(H2, wv);
            }
        }
    }

    if (LABELS && pair == 0 && chk(a.labels + (size_t)y * a.labels_pitch + x, 1, kSiteLabel))
        a.labels[(size_t)y * a.labels_pitch + x] = (uint8_t)(best_key & 0xFFu);

    // destinations (after the forward pass: fewer live registers during it)
    uint8_t *dstA, *dstB;
    dsts(dstA, dstB);

    // -H in both 16-bit lanes, for the fused add-min of the output
    const uint32_t negH2 = ((0u - (H2 & 0xFFFFu)) & 0xFFFFu) | ((0u - (H2 >> 16)) << 16);
    uint32_t G = F[LP - 1];
#pragma unroll
    for (int j = LP / 16 - 1; j >= 0; --j) {
        uint32_t o[16];
#pragma unroll
        for (int i = 15; i >= 0; --i) {
            const int d = 16 * j + i;
            if (d < LP - 1)
                G = __viaddmin_u16x2(G, a.c2, F[d]);           // min(G + c, F)
            o[i] = __viaddmin_s16x2(G, negH2, a.ts2);   // (m_A(d), m_B(d)) = min(G - H, Ts)
        }
        uint32_t oa[4], ob[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // outputs are in [0, Ts], Ts <= 127: o0 + 256 o1 = (A0 A1 B0 B1)
            // without carries, one multiply-add off the integer ALU pipe
            const uint32_t t01 = o[4 * q] + o[4 * q + 1] * a.k256;
            const uint32_t t23 = o[4 * q + 2] + o[4 * q + 3] * a.k256;
            oa[q] = prmt(t01, t23, 0x5410u);
            ob[q] = prmt(t01, t23, 0x7632u);
        }
        if (dstA)
            st_piece_keep(dstA, j, make_uint4(oa[0], oa[1], oa[2], oa[3]), pol);
        if (dstB)
            st_piece_keep(dstB, j, make_uint4(ob[0], ob[1], ob[2], ob[3]), pol);
    }
}

// ---------------------------------------------------------------------------
// message sweep, labels split across NS = 2 or 4 lanes (small levels)
//
// On the coarse levels there are too few pixels to fill the GPU, so a sweep
// is as long as one thread's serial label chain.  Here each direction pair
// is shared by NS adjacent lanes, one per block of HL = LP / NS labels.  Each
// lane runs the forward and backward lower-envelope passes over its block;
// the blocks are joined exactly by
//   F(d) = min(F_blk(d), F(s_j - 1) + c (d - s_j + 1))   forward, block j > 0
//   G(d) = min(G_blk(d), G(s_{j+1}) + c (s_{j+1} - d))    backward, block j < NS-1
// (s_j = first label of block j).  The carries are min-plus scans over the
// lane group: F(end of block j) = min over i <= j of (E_i + c HL (j - i)),
// E_i the block's own end value, and the mirror image backwards -- one
// shuffle step for two lanes, two for four.  The chain per lane is NS times
// shorter; the corrections touch all labels in parallel.

// Threads 0-63 of a CTA take direction pair 0 (left / right) of its pixels,
// 64-127 pair 1 (up / down): PAIR is fixed per warp, as in sweep_body.
template <int LP, typename CostT, bool BYTES, bool FULL, int NS, int PAIR>
__device__ __forceinline__ void sweep_split_pair(const SweepArgs &a, unsigned block)
{
    static_assert(NS == 2 || NS == 4, "label blocks per direction pair");
    constexpr int HL = LP / NS;  // labels per lane
    constexpr int HC = HL / 16;  // 16-label chunks per lane
    static_assert(HC >= 1 && HL % 16 == 0, "whole 16-label chunks per lane");
    constexpr int pair = PAIR;
    constexpr int kHalfThreads = kSweepThreads / 2;
    const int half = (int)(threadIdx.x % NS);   // label block of this lane
    // over rows padded to whole 16-slot groups
    const unsigned slot = block * (kHalfThreads / NS) + (threadIdx.x & (kHalfThreads - 1)) / NS;
    const unsigned rowslots = 16u * (unsigned)a.wg;
    int y = 0, xh = 0, x = 0;
    bool valid = slot < (unsigned)a.h * rowslots;
    if (valid) {
        y = (int)div_by(slot, a.div_rowslots);
        xh = (int)(slot - (unsigned)y * rowslots);
        x = 2 * xh + ((a.color + y) & 1);
        valid = x < a.w;
    }
    const bool has[4] = {x > 0, x < a.w - 1, y > 0, y < a.h - 1};
    const uint8_t *in[4];
    if (a.from_parent) {
        const int px = x >> 1, py = y >> 1, pc = (px + py) & 1;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            in[k] = a.pmsg + slot_base((pc * 4 + k) * a.ph + py, px >> 1, a.pwg, LP / 16);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            in[k] = a.msg + slot_base((a.color * 4 + k) * a.h + y, xh, a.wg, LP / 16);
    }
    bool use[4];
    {
        const int px = x >> 1, py = y >> 1;
        const bool phas[4] = {px > 0, px < a.pw - 1, py > 0, py < a.ph - 1};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            use[k] = valid && has[k] && !a.zero_in && (!a.from_parent || phas[k]);
    }
    const uint8_t *cost = reinterpret_cast<const uint8_t *>(a.cost) +
                          slot_base(a.color * a.h + y, xh, a.wg, (LP / 16) * (int)sizeof(CostT));
    uint8_t *own = a.msg + slot_base(a.color * 4 * a.h + y, xh, a.wg, LP / 16);
    const size_t dir_stride = (size_t)a.h * a.wg * (LP / 16) * kPieceStride;   // bytes between directions
    pdl_begin();   // the index work above overlaps the previous kernel's last wave

    uint32_t F[HL];
    uint32_t H2 = kBig2;
#pragma unroll
    for (int jj = 0; jj < HC; ++jj) {
        const int j = half * HC + jj;   // chunk of the full label range
        uint4 m[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            m[k] = use[k] ? ld_piece(in[k], j) : make_uint4(0, 0, 0, 0);
        CostChunk<CostT> cc;
        if (valid)
            cc.load(cost, j);
        else
            cc.zero();
        if (valid && a.materialize) {
            const size_t k0 = 2 * pair;
            st_piece(own + k0 * dir_stride, j, pair ? m[2] : m[0]);
            st_piece(own + (k0 + 1) * dir_stride, j, pair ? m[3] : m[1]);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int k = 16 * jj + i;           // label within the half
            const int d = half * HL + k;         // label
            uint32_t wv;
            if (BYTES) {
                const int wi = i >> 2, q = i & 3;
                const uint32_t s4 = cc.word(wi) + (&m[0].x)[wi] + (&m[1].x)[wi] + (&m[2].x)[wi] + (&m[3].x)[wi];
                const uint32_t a4 = s4 - (pair ? (&m[2].x)[wi] : (&m[0].x)[wi]);
                const uint32_t b4 = s4 - (pair ? (&m[3].x)[wi] : (&m[1].x)[wi]);
                // (byte q of a4, byte q of b4) as 16-bit lanes: pick, then clear bytes 1 and 3
                wv = prmt(a4, b4, (uint32_t)q | ((uint32_t)(4 + q) << 8)) & 0x00FF00FFu;
            } else {
                const int wi = i >> 2;
                const uint32_t plr = pair_bytes((&m[0].x)[wi], (&m[1].x)[wi], i & 3);
                const uint32_t pud = pair_bytes((&m[2].x)[wi], (&m[3].x)[wi], i & 3);
                const uint32_t t = plr + pud;
                const uint32_t s2 = t + prmt(t, t, 0x1032u) + cc.dup(i);
                wv = s2 - (pair ? pud : plr);
            }
            if (!FULL && d >= a.L)
                wv = kBig2;
            F[k] = k == 0 ? wv : __viaddmin_u16x2(F[k - 1], a.c2, wv);
            H2 = min_u16x2(H2, wv);
        }
    }
    // join the blocks: global minimum over the lane group
#pragma unroll
    for (int o = 1; o < NS; o <<= 1)
        H2 = min_u16x2(H2, __shfl_xor_sync(0xffffffffu, H2, o));
    // forward carry: inclusive min-plus scan of the blocks' end values
    uint32_t A = F[HL - 1];
#pragma unroll
    for (int o = 1; o < NS; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, A, o, NS);
        if (half >= o)
            A = min_u16x2(A, t + a.c2 * (uint32_t)(HL * o));
    }
    const uint32_t c_lo = __shfl_up_sync(0xffffffffu, A, 1, NS);   // F at the end of the previous block
    if (half > 0) {
#pragma unroll
        for (int k = 0; k < HL; ++k)
            F[k] = min_u16x2(F[k], c_lo + a.c2 * (uint32_t)(k + 1));
    }
    // backward pass over the block (G kept in F), then the carry from the right
#pragma unroll
    for (int k = HL - 2; k >= 0; --k)
        F[k] = __viaddmin_u16x2(F[k + 1], a.c2, F[k]);
    uint32_t B = F[0];
#pragma unroll
    for (int o = 1; o < NS; o <<= 1) {
        const uint32_t t = __shfl_down_sync(0xffffffffu, B, o, NS);
        if (half + o < NS)
            B = min_u16x2(B, t + a.c2 * (uint32_t)(HL * o));
    }
    const uint32_t c_hi = __shfl_down_sync(0xffffffffu, B, 1, NS);   // G at the start of the next block
    if (half < NS - 1) {
#pragma unroll
        for (int k = 0; k < HL; ++k)
            F[k] = min_u16x2(F[k], c_hi + a.c2 * (uint32_t)(HL - k));
    }
    if (!valid)
        return;

    const int ncolor = a.color ^ 1;
    uint8_t *dstA = nullptr, *dstB = nullptr;
    if (pair == 0) {
        if (has[0])
            dstA = a.msg + slot_base((ncolor * 4 + 1) * a.h + y, (x - 1) >> 1, a.wg, LP / 16);
        if (has[1])
            dstB = a.msg + slot_base((ncolor * 4 + 0) * a.h + y, (x + 1) >> 1, a.wg, LP / 16);
    } else {
        if (has[2])
            dstA = a.msg + slot_base((ncolor * 4 + 3) * a.h + (y - 1), x >> 1, a.wg, LP / 16);
        if (has[3])
            dstB = a.msg + slot_base((ncolor * 4 + 2) * a.h + (y + 1), x >> 1, a.wg, LP / 16);
    }
    const uint32_t negH2 = ((0u - (H2 & 0xFFFFu)) & 0xFFFFu) | ((0u - (H2 >> 16)) << 16);
#pragma unroll
    for (int jj = 0; jj < HC; ++jj) {
        uint32_t o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i)
            o[i] = __viaddmin_s16x2(F[16 * jj + i], negH2, a.ts2);   // min(G - H, Ts)
        uint32_t oa[4], ob[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t t01 = o[4 * q] + o[4 * q + 1] * a.k256;   // (A0 A1 B0 B1), as in sweep_pixel
            const uint32_t t23 = o[4 * q + 2] + o[4 * q + 3] * a.k256;
            oa[q] = prmt(t01, t23, 0x5410u);
            ob[q] = prmt(t01, t23, 0x7632u);
        }
        const int j = half * HC + jj;
        if (dstA)
            st_piece(dstA, j, make_uint4(oa[0], oa[1], oa[2], oa[3]));
        if (dstB)
            st_piece(dstB, j, make_uint4(ob[0], ob[1], ob[2], ob[3]));
    }
}

template <int LP, typename CostT, bool BYTES, bool FULL, int NS>
__device__ __forceinline__ void sweep_split_body(const SweepArgs &a, unsigned block)
{
    if (threadIdx.x < kSweepThreads / 2)
        sweep_split_pair<LP, CostT, BYTES, FULL, NS, 0>(a, block);
    else
        sweep_split_pair<LP, CostT, BYTES, FULL, NS, 1>(a, block);
}

template <int LP, typename CostT, bool BYTES, bool FULL, bool LABELS, bool PRELOAD>
__global__ void __launch_bounds__(kSweepThreads) k_bp_sweep(SweepArgs a)
{
    sweep_body<LP, CostT, BYTES, FULL, LABELS, PRELOAD>(a, blockIdx.x);
}

template <int LP, typename CostT, bool BYTES, bool FULL, int NS>
__global__ void __launch_bounds__(kSweepThreads) k_bp_sweep_split(SweepArgs a)
{
    sweep_split_body<LP, CostT, BYTES, FULL, NS>(a, blockIdx.x);
}

// ---------------------------------------------------------------------------
// staged sweep: persistent CTAs stream their tiles through shared memory
//
// A tile is 64 consecutive slots of the active colour (4 slot groups, which
// may run across a row end).  Its four incoming-message blocks and its cost
// block are each one contiguous run of 64 LP bytes, so one thread issues five
// bulk asynchronous copies per tile, into one of two shared-memory stages
// tracked by an mbarrier; a CTA works through tiles blockIdx.x,
// blockIdx.x + gridDim.x, ..., with the next tile's copies in flight while it
// computes the current one.  Compute is sweep_pixel reading shared memory;
// the outgoing messages go straight to global memory as in k_bp_sweep.
// Measured on the 2.7K pair (level 0, 64 labels, 740 resident CTAs): 17.3 us
// per sweep against 16.7 for the register-preload kernel, yet four pairs in
// flight run 4110 pairs/s against 3941 (one pair at a time 3015 against
// 3109); since the border slots are zeroed and all four directions are read
// without selects, 16.5 us per sweep and 4107 / 3070-3090 pairs/s.  Reading
// the cost from global memory instead (four blocks per stage, six CTAs per
// SM) measured 3953 / 3015.
// For the iterations that read this level's own messages (not the first of a
// level) with byte costs and byte-lane sums, on levels 0 and 1, whose
// never-written border slots k_cost01 zeroes -- level 0 by default.
constexpr int kStageSlots = kSweepThreads / 2;

template <int LP>
constexpr int staged_smem_bytes()
{
    return 2 * 5 * kStageSlots * LP + 16;   // two stages of 5 blocks, two mbarriers
}

template <int LP, bool FULL, bool LABELS>
__global__ void __launch_bounds__(kSweepThreads) k_bp_sweep_staged(SweepArgs a)
{
    constexpr int NP = LP / 16;
    constexpr int kBlock = kStageSlots * LP;   // one direction (or the cost) of a tile
    constexpr int kStage = 5 * kBlock;
    extern __shared__ __align__(128) uint8_t sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * kStage);
    if (threadIdx.x == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_init(bar + 1, 1);
    }
    __syncthreads();
    const int ngroups = a.h * a.wg;   // 16-slot groups of one colour
    const int ntiles = (ngroups + 3) / 4;
    const size_t arr = (size_t)ngroups * NP * kPieceStride;   // one colour-direction array
    const uint8_t *msg_in = a.msg + (size_t)a.color * 4 * arr;
    uint8_t *const msg_out = a.msg + (size_t)(a.color ^ 1) * 4 * arr;
    const uint8_t *cost_in = static_cast<const uint8_t *>(a.cost) + (size_t)a.color * arr;
    // part 1: the phase's byte count and the data term; part 2: the messages
    auto issue = [&](int tile, int buf, int part) {
        const size_t off = (size_t)tile * 4 * NP * kPieceStride;
        const uint32_t bytes = (uint32_t)min(4, ngroups - 4 * tile) * NP * kPieceStride;
        uint8_t *dst = sm + buf * kStage;
        if (part & 1)
            tc::mbar_expect_tx(bar + buf, 5 * bytes);
        if (a.withhold_copies)   // nothing completes the phase: the bounded wait runs out
            return;
        bool in_range = chk(cost_in + off, bytes, kSiteBulkCopy);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            in_range = in_range && chk(msg_in + k * arr + off, bytes, kSiteBulkCopy);
        if (!in_range)   // (checked build) the wait runs out and the call reports VS_ETIMEOUT
            return;
        if (part & 2) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                tc::bulk_g2s(dst + k * kBlock, msg_in + k * arr + off, bytes, bar + buf);
        }
        if (part & 1)
            tc::bulk_g2s(dst + 4 * kBlock, cost_in + off, bytes, bar + buf);
    };
    // The first tile's data term is copied before the wait for the previous
    // kernel: this kernel runs from a level's second iteration on, so the
    // previous kernel is a sweep of the same level, and this launch is
    // scheduled only once every CTA of that sweep has passed its own wait --
    // the data term's writer (k_cost01) and every other earlier kernel have
    // finished by then, and no sweep writes the data term.
    if (threadIdx.x == 0 && (int)blockIdx.x < ntiles)
        issue(blockIdx.x, 0, 1);
    pdl_begin();
    if (threadIdx.x == 0 && (int)blockIdx.x < ntiles)
        issue(blockIdx.x, 0, 2);
    const int sl = threadIdx.x & (kStageSlots - 1), pair = threadIdx.x / kStageSlots;   // pair by warp
    const unsigned rowslots = 16u * (unsigned)a.wg;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int buf = it & 1;
        const int next = tile + gridDim.x;
        // the stage of `next` was read in the previous round, which every
        // thread has left (the barrier at the end of the loop)
        if (threadIdx.x == 0 && next < ntiles)
            issue(next, buf ^ 1, 3);
        const bool arrived = tc::mbar_wait(bar + buf, (uint32_t)(it >> 1) & 1u);
        if (!__syncthreads_and(arrived)) {
            // The copies did not complete within the bound: report it and issue
            // nothing more.  A CTA must not leave while a bulk copy still
            // writes its shared memory, so thread 0 first waits once more
            // (four seconds each) for the stages whose copies it did issue:
            // this tile's and, if issued above, the next one's.  (The test aid
            // issues none, so nothing is in flight and the CTA leaves at
            // once.)  Only a copy that never lands at all, which no input can
            // cause, would still be pending when that second bound runs out.
            if (threadIdx.x == 0) {
                if (chk(a.status, 4, kSiteStatus))
                    atomicExch(a.status, VS_ETIMEOUT);
                if (!a.withhold_copies) {
                    tc::mbar_wait(bar + buf, (uint32_t)(it >> 1) & 1u, 4000000000ull);
                    if (next < ntiles)
                        tc::mbar_wait(bar + (buf ^ 1), (uint32_t)((it + 1) >> 1) & 1u, 4000000000ull);
                }
            }
            __syncthreads();
            return;
        }
        const unsigned slot = (unsigned)tile * kStageSlots + (unsigned)sl;
        const int y = (int)div_by(slot, a.div_rowslots);
        const int xh = (int)(slot - (unsigned)y * rowslots);
        const int x = 2 * xh + ((a.color + y) & 1);
        if (y < a.h && x < a.w) {
            const bool has[4] = {x > 0, x < a.w - 1, y > 0, y < a.h - 1};
            const uint8_t *base = sm + buf * kStage + (sl >> 4) * NP * kPieceStride + (sl & 15) * 16;
            const uint8_t *const in[4] = {base, base + kBlock, base + 2 * kBlock, base + 3 * kBlock};
            const uint8_t *cost = base + 4 * kBlock;
            // the slots of missing neighbours hold 0 (k_cost01 of this call), so
            // all four directions are read as they are
            const bool all[4] = {true, true, true, true};
            // destinations as 32-bit offsets into the other colour's arrays
            // (each below 2^31 bytes on this kernel)
            auto off = [&](int yy, int xs) {
                return (((uint32_t)yy * (uint32_t)a.wg + ((uint32_t)xs >> 4)) * (uint32_t)(NP * 16) +
                        ((uint32_t)xs & 15u)) *
                       16u;
            };
            if (pair == 0)
                sweep_pixel<LP, uint8_t, true, FULL, LABELS, false, true, 0>(
                    a, x, y, in, all, cost, nullptr, [&](uint8_t *&A, uint8_t *&B) {
                        A = has[0] ? msg_out + arr + off(y, (x - 1) >> 1) : nullptr;
                        B = has[1] ? msg_out + off(y, (x + 1) >> 1) : nullptr;
                    });
            else
                sweep_pixel<LP, uint8_t, true, FULL, LABELS, false, true, 1>(
                    a, x, y, in, all, cost, nullptr, [&](uint8_t *&A, uint8_t *&B) {
                        A = has[2] ? msg_out + 3 * arr + off(y - 1, x >> 1) : nullptr;
                        B = has[3] ? msg_out + 2 * arr + off(y + 1, x >> 1) : nullptr;
                    });
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// fused sweeps: K iterations per launch on shared-memory tiles with a halo
//
// A CTA owns a core tile of TW x TH pixels of the level.  It copies into
// shared memory the data term and the incoming messages (both colours, all
// four directions) of its region -- the core grown by K pixels on every side
// that is not a frame edge -- and runs iterations t0 .. t0 + K - 1 of the
// red-black schedule there, with the global parity ((x + y + t) even), in
// place: an iteration reads the active colour's slots and writes the other
// colour's, as in the global layout.  At fused iteration i only the active
// pixels of the region shrunk by i on its cut sides compute.  Their incoming
// messages are exact: a slot whose sender lies outside the region is never
// refreshed, and each iteration spreads that staleness by at most one pixel
// inward, so the computed set is a trapezoid over the K iterations that ends
// on the core, whose state after K iterations is exact.  The CTA writes the
// core's messages to the level's other message buffer (no CTA reads
// another's results within a launch).  The launch that ends the last
// level-0 iteration also writes every core pixel's label.
//
// Shared memory, 16-byte pieces in planes of rh x rwh slots (row ry of the
// region; slot sx = (x >> 1) - (rx0 >> 1), the global colour split):
//   messages [c][k][j][rh][rwh]    j  < LP / 16
//   cost     [c][jc][rh][rwh]      jc < LP / 16 * sizeof(CostT)
// The lanes of a pixel are 2 NS consecutive threads: direction pair (left /
// right, up / down) times NS blocks of the labels, joined by shuffles as in
// the split sweep; one thread per lane, up to 512 per CTA.

constexpr int kFusedThreads = 512;   // most threads of a fused CTA (a launch may use fewer)

struct FusedArgs {
    const uint8_t *cost;    // this level's data term
    const uint8_t *src;     // incoming messages before iteration t0: this level's, or the parent's
    uint8_t *dst;           // this level's incoming messages after iteration t0 + K - 1
    int w, h, wg, L;
    int pw, ph, pwg;        // parent level (from_parent)
    int t0, K;              // first iteration of the launch, iterations fused
    int TW, TH, tiles_x;    // core tile, tiles per row
    int from_parent;        // t0 == 0 below the coarsest level: start from the parent's messages
    int zero_in;            // t0 == 0 on the coarsest level: start from zero messages
    uint32_t c2, ts2;       // (c, c) and (Ts, Ts) packed
    uint8_t *labels;        // non-null: write the core's labels at the end
    int labels_pitch;
};

__host__ __device__ constexpr int fused_region_rows(int TH, int K) { return TH + 2 * K; }
__host__ __device__ constexpr int fused_region_slots(int TW, int K) { return ((TW + 2 * K + 1) >> 1) + 1; }

// One direction pair (or one label block of it) of one active pixel, its
// sources and destinations in shared memory (`ps` pieces between the pieces
// of a slot).  Every lane of the warp calls this (the label blocks are joined
// by shuffles); lanes with valid == false read zeros and store nothing.
template <int LP, typename CostT, bool BYTES, bool FULL, int NS>
__device__ __forceinline__ void fused_pixel(const FusedArgs &a, int pair, int half, bool valid,
                                            const uint4 *const (&in)[4], const uint4 *cost, int ps, uint4 *dstA,
                                            uint4 *dstB)
{
    constexpr int HL = LP / NS;   // labels per lane
    constexpr int HC = HL / 16;   // 16-label chunks per lane
    static_assert(NS == 1 || NS == 2 || NS == 4, "label blocks per direction pair");
    static_assert(HL % 16 == 0, "whole 16-label chunks per lane");
    uint32_t F[HL];
    uint32_t H2 = kBig2;
#pragma unroll
    for (int jj = 0; jj < HC; ++jj) {
        const int j = half * HC + jj;
        uint4 m[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            m[k] = valid ? in[k][j * ps] : make_uint4(0, 0, 0, 0);
        CostChunk<CostT> cc;
        if (valid)
            cc.load_s(cost, j, ps);
        else
            cc.zero();
        if (BYTES) {
#pragma unroll
            for (int wi = 0; wi < 4; ++wi) {
                const uint32_t s4 = cc.word(wi) + (&m[0].x)[wi] + (&m[1].x)[wi] + (&m[2].x)[wi] + (&m[3].x)[wi];
                const uint32_t a4 = s4 - (pair ? (&m[2].x)[wi] : (&m[0].x)[wi]);
                const uint32_t b4 = s4 - (pair ? (&m[3].x)[wi] : (&m[1].x)[wi]);
                const uint32_t x01 = prmt(a4, b4, 0x5140u);   // A0 B0 A1 B1
                const uint32_t x23 = prmt(a4, b4, 0x7362u);   // A2 B2 A3 B3
                const uint32_t wq[4] = {prmt(x01, 0u, 0x4140u), prmt(x01, 0u, 0x4342u), prmt(x23, 0u, 0x4140u),
                                        prmt(x23, 0u, 0x4342u)};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int kk = 16 * jj + 4 * wi + q;   // label within the lane's block
                    uint32_t wv = wq[q];
                    if (!FULL && half * HL + kk >= a.L)
                        wv = kBig2;
                    F[kk] = kk == 0 ? wv : __viaddmin_u16x2(F[kk - 1], a.c2, wv);   // min(F + c, h)
                    H2 = min_u16x2(H2, wv);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int kk = 16 * jj + i;
                const int wi = i >> 2;
                const uint32_t plr = pair_bytes((&m[0].x)[wi], (&m[1].x)[wi], i & 3);
                const uint32_t pud = pair_bytes((&m[2].x)[wi], (&m[3].x)[wi], i & 3);
                const uint32_t t = plr + pud;                                  // (L+U, R+D), no carry
                const uint32_t s2 = t + prmt(t, t, 0x1032u) + cc.dup(i);      // (S, S)
                uint32_t wv = s2 - (pair ? pud : plr);                         // (h_A, h_B)
                if (!FULL && half * HL + kk >= a.L)
                    wv = kBig2;
                F[kk] = kk == 0 ? wv : __viaddmin_u16x2(F[kk - 1], a.c2, wv);
                H2 = min_u16x2(H2, wv);
            }
        }
    }
    if (NS > 1) {
        // the label blocks of a direction pair are NS consecutive lanes:
        // global minimum, then the forward carry from the blocks to the left
#pragma unroll
        for (int o = 1; o < NS; o <<= 1)
            H2 = min_u16x2(H2, __shfl_xor_sync(0xffffffffu, H2, o));
        uint32_t A = F[HL - 1];
#pragma unroll
        for (int o = 1; o < NS; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, A, o, NS);
            if (half >= o)
                A = min_u16x2(A, t + a.c2 * (uint32_t)(HL * o));
        }
        const uint32_t c_lo = __shfl_up_sync(0xffffffffu, A, 1, NS);
        if (half > 0) {
#pragma unroll
            for (int k = 0; k < HL; ++k)
                F[k] = min_u16x2(F[k], c_lo + a.c2 * (uint32_t)(k + 1));
        }
    }
    // backward pass (G kept in F)
#pragma unroll
    for (int k = HL - 2; k >= 0; --k)
        F[k] = __viaddmin_u16x2(F[k + 1], a.c2, F[k]);
    if (NS > 1) {
        uint32_t B = F[0];
#pragma unroll
        for (int o = 1; o < NS; o <<= 1) {
            const uint32_t t = __shfl_down_sync(0xffffffffu, B, o, NS);
            if (half + o < NS)
                B = min_u16x2(B, t + a.c2 * (uint32_t)(HL * o));
        }
        const uint32_t c_hi = __shfl_down_sync(0xffffffffu, B, 1, NS);
        if (half < NS - 1) {
#pragma unroll
            for (int k = 0; k < HL; ++k)
                F[k] = min_u16x2(F[k], c_hi + a.c2 * (uint32_t)(HL - k));
        }
    }
    if (!valid)
        return;
    const uint32_t negH2 = ((0u - (H2 & 0xFFFFu)) & 0xFFFFu) | ((0u - (H2 >> 16)) << 16);
#pragma unroll
    for (int jj = 0; jj < HC; ++jj) {
        uint32_t o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i)
            o[i] = __viaddmin_s16x2(F[16 * jj + i], negH2, a.ts2);   // min(G - H, Ts)
        uint32_t oa[4], ob[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t t01 = prmt(o[4 * q], o[4 * q + 1], 0x6420u);
            const uint32_t t23 = prmt(o[4 * q + 2], o[4 * q + 3], 0x6420u);
            oa[q] = prmt(t01, t23, 0x6420u);
            ob[q] = prmt(t01, t23, 0x7531u);
        }
        const int j = half * HC + jj;
        if (dstA)
            dstA[j * ps] = make_uint4(oa[0], oa[1], oa[2], oa[3]);
        if (dstB)
            dstB[j * ps] = make_uint4(ob[0], ob[1], ob[2], ob[3]);
    }
}

// 16 bytes from global to shared memory without a register round trip
// (zeros when `valid` is false: no byte is read then).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid)
{
    const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0)
                 : "memory");
}

template <int LP, typename CostT, bool BYTES, bool FULL, int NS>
__global__ void __launch_bounds__(kFusedThreads, 1) k_bp_fused(FusedArgs a)
{
    constexpr int NP = LP / 16;                     // pieces of a message
    constexpr int NPC = NP * (int)sizeof(CostT);    // pieces of a data term
    extern __shared__ __align__(16) uint4 fsm[];
    pdl_begin();
    const int by = (int)(blockIdx.x / (unsigned)a.tiles_x);
    const int bx = (int)blockIdx.x - by * a.tiles_x;
    const int x0 = bx * a.TW, y0 = by * a.TH;
    const int x1 = min(x0 + a.TW, a.w), y1 = min(y0 + a.TH, a.h);
    const int rx0 = max(x0 - a.K, 0), ry0 = max(y0 - a.K, 0);
    const int rx1 = min(x1 + a.K, a.w), ry1 = min(y1 + a.K, a.h);
    const int sx0 = rx0 >> 1;
    const int rwh = ((rx1 - 1) >> 1) - sx0 + 1;
    const int ps = (ry1 - ry0) * rwh;   // slots of a plane = pieces between planes
    uint4 *msg_s = fsm;                 // planes (c * 4 + k) * NP + j
    uint4 *cost_s = fsm + 8 * NP * ps;  // planes c * NPC + jc

    // 1. the region's state, one (colour, direction or data term, slot) per
    //    work item: a slot outside the region, or from a missing neighbour
    //    (or one the parent level lacked), reads 0
    for (int u = threadIdx.x; u < 10 * ps; u += blockDim.x) {
        const int grp = u / ps, r = u - grp * ps;
        const int c = grp >= 5, g = grp - 5 * c;   // g: direction 0..3, or 4 for the data term
        const int ry = r / rwh;
        const int y = ry0 + ry, xh = sx0 + (r - ry * rwh);
        const int x = 2 * xh + ((c + y) & 1);
        const bool in = x >= rx0 && x < rx1;
        if (g < 4) {
            const int k = g;
            const int px = x >> 1, py = y >> 1;
            const bool has = k == 0 ? x > 0 : k == 1 ? x < a.w - 1 : k == 2 ? y > 0 : y < a.h - 1;
            const bool phas = k == 0 ? px > 0 : k == 1 ? px < a.pw - 1 : k == 2 ? py > 0 : py < a.ph - 1;
            const bool use = in && has && !a.zero_in && (!a.from_parent || phas);
            const uint8_t *g0 = !use ? a.cost
                                : a.from_parent
                                    ? a.src + slot_base((((px + py) & 1) * 4 + k) * a.ph + py, px >> 1, a.pwg, NP)
                                    : a.src + slot_base((c * 4 + k) * a.h + y, xh, a.wg, NP);
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                const bool ok = use && chk(g0 + (size_t)j * kPieceStride, 16, kSiteAsyncCopy);
                cp_async16(msg_s + ((c * 4 + k) * NP + j) * ps + r, ok ? g0 + (size_t)j * kPieceStride : a.cost, ok);
            }
        } else {
            const uint8_t *g0 = in ? a.cost + slot_base(c * a.h + y, xh, a.wg, NPC) : a.cost;
#pragma unroll
            for (int jc = 0; jc < NPC; ++jc) {
                const bool ok = in && chk(g0 + (size_t)jc * kPieceStride, 16, kSiteAsyncCopy);
                cp_async16(cost_s + (c * NPC + jc) * ps + r, ok ? g0 + (size_t)jc * kPieceStride : a.cost, ok);
            }
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();

    // 2. K iterations on the shrinking region
    for (int i = 0; i < a.K; ++i) {
        const int c = (a.t0 + i) & 1;
        const int ex0 = rx0 + (rx0 > 0 ? i : 0), ex1 = rx1 - (rx1 < a.w ? i : 0);
        const int ey0 = ry0 + (ry0 > 0 ? i : 0), ey1 = ry1 - (ry1 < a.h ? i : 0);
        const int es0 = ex0 >> 1, ens = ((ex1 - 1) >> 1) - es0 + 1;
        const int items = (ey1 - ey0) * ens * (2 * NS);
        for (int base = 0; base < items; base += blockDim.x) {
            const int u = base + (int)threadIdx.x;
            const int pix = u / (2 * NS), sub = u - pix * (2 * NS);
            const int half = sub % NS, pair = sub / NS;
            const int row = pix / ens;
            const int y = ey0 + row, xh = es0 + (pix - row * ens);
            const int x = 2 * xh + ((c + y) & 1);
            const bool valid = u < items && x >= ex0 && x < ex1;
            const int slot = (y - ry0) * rwh + (xh - sx0);
            const uint4 *in[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                in[k] = msg_s + (c * 4 + k) * NP * ps + slot;
            const uint4 *cost = cost_s + c * NPC * ps + slot;
            // destinations: A = left / up neighbour, B = right / down, inside the region
            uint4 *dstA = nullptr, *dstB = nullptr;
            if (valid) {
                uint4 *o = msg_s + (c ^ 1) * 4 * NP * ps;
                if (pair == 0) {
                    if (x - 1 >= rx0)
                        dstA = o + 1 * NP * ps + (y - ry0) * rwh + ((x - 1) >> 1) - sx0;
                    if (x + 1 < rx1)
                        dstB = o + 0 * NP * ps + (y - ry0) * rwh + ((x + 1) >> 1) - sx0;
                } else {
                    if (y - 1 >= ry0)
                        dstA = o + 3 * NP * ps + slot - rwh;
                    if (y + 1 < ry1)
                        dstB = o + 2 * NP * ps + slot + rwh;
                }
            }
            fused_pixel<LP, CostT, BYTES, FULL, NS>(a, pair, half, valid, in, cost, ps, dstA, dstB);
        }
        __syncthreads();
    }

    // 3. the core's messages out, one (colour, direction, slot) per work item
    const int cs0 = x0 >> 1, cns = ((x1 - 1) >> 1) - cs0 + 1;
    const int n = (y1 - y0) * cns;
    for (int u = threadIdx.x; u < 8 * n; u += blockDim.x) {
        const int plane = u / n, r = u - plane * n;   // plane = c * 4 + k
        const int c = plane >> 2, k = plane & 3;
        const int row = r / cns;
        const int y = y0 + row, xh = cs0 + (r - row * cns);
        const int x = 2 * xh + ((c + y) & 1);
        if (x < x0 || x >= x1)
            continue;
        const int slot = (y - ry0) * rwh + (xh - sx0);
        uint8_t *g = a.dst + slot_base((c * 4 + k) * a.h + y, xh, a.wg, NP);
#pragma unroll
        for (int j = 0; j < NP; ++j)
            st_piece(g, j, msg_s[((c * 4 + k) * NP + j) * ps + slot]);
    }
    if (!a.labels)
        return;
    // labels of the core (the launch that ends level 0): d* = argmin_d D(d)
    // + the four incoming messages (0 from a missing neighbour), the
    // smallest d on ties
    for (int u = threadIdx.x; u < 2 * n; u += blockDim.x) {
        const int c = u >= n, r = u - c * n;
        const int row = r / cns;
        const int y = y0 + row, xh = cs0 + (r - row * cns);
        const int x = 2 * xh + ((c + y) & 1);
        if (x < x0 || x >= x1)
            continue;
        const int slot = (y - ry0) * rwh + (xh - sx0);
        int best = 0x7FFFFFFF, bestd = 0;
        for (int j = 0; j < NP; ++j) {
            uint4 m[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                m[k] = msg_s[((c * 4 + k) * NP + j) * ps + slot];
            CostChunk<CostT> cc;
            cc.load_s(cost_s + c * NPC * ps + slot, j, ps);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int sh = 8 * (i & 3);
                int b = (int)(cc.dup(i) & 0xFFFFu);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    b += (int)(((&m[k].x)[i >> 2] >> sh) & 0xFFu);
                if (16 * j + i < a.L && b < best) {
                    best = b;
                    bestd = 16 * j + i;
                }
            }
        }
        if (chk(a.labels + (size_t)y * a.labels_pitch + x, 1, kSiteLabel))
            a.labels[(size_t)y * a.labels_pitch + x] = (uint8_t)bestd;
    }
}

// ---------------------------------------------------------------------------
// batched sweeps: one launch advances the same level-iteration of many pairs
//
// The jobs of a launch (one per pair, same kernel variant) travel in the
// kernel parameters, so a captured CUDA graph replays them without any
// host-side table; job j owns the launch's CTAs first_block[j] ..
// first_block[j + 1] - 1.

constexpr int kMaxBatch = 64;

struct BatchArgs {
    int njobs;
    unsigned first_block[kMaxBatch + 1];
    SweepArgs job[kMaxBatch];
};

__device__ __forceinline__ int batch_job(const BatchArgs &b, unsigned block)
{
    int lo = 0, hi = b.njobs - 1;   // last job whose first block is <= block
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.first_block[mid] <= block)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <int LP, typename CostT, bool BYTES, bool FULL, bool LABELS, bool PRELOAD>
__global__ void __launch_bounds__(kSweepThreads) k_bp_sweep_batch(const __grid_constant__ BatchArgs b)
{
    const int j = batch_job(b, blockIdx.x);
    sweep_body<LP, CostT, BYTES, FULL, LABELS, PRELOAD>(b.job[j], blockIdx.x - b.first_block[j]);
}

template <int LP, typename CostT, bool BYTES, bool FULL, int NS>
__global__ void __launch_bounds__(kSweepThreads) k_bp_sweep_split_batch(const __grid_constant__ BatchArgs b)
{
    const int j = batch_job(b, blockIdx.x);
    sweep_split_body<LP, CostT, BYTES, FULL, NS>(b.job[j], blockIdx.x - b.first_block[j]);
}

// ---------------------------------------------------------------------------
// labels and read-out

struct LabelArgs {
    const uint8_t *cost;   // level 0
    const uint8_t *msg;    // level 0
    uint8_t *labels;
    int labels_pitch, w, h, wh, wg, L, Lp;
    int color;             // the colour whose labels are still missing
};

// d* = argmin_d D0(d) + sum of the in-frame incoming messages, smallest d
// wins, for the pixels of one colour (the other colour's labels come from
// the last sweep).
__global__ void k_bp_labels(LabelArgs a)
{
    pdl_begin();
    const int xh = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int c = a.color;
    const int x = 2 * xh + ((c + y) & 1);
    if (x >= a.w || y >= a.h)
        return;
    const bool has[4] = {x > 0, x < a.w - 1, y > 0, y < a.h - 1};
    const int np = a.Lp / 16;
    const uint8_t *cost = a.cost + slot_base(c * a.h + y, xh, a.wg, np);
    const uint8_t *in[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        in[k] = a.msg + slot_base((c * 4 + k) * a.h + y, xh, a.wg, np);
    int best = 0x7FFFFFFF, bestd = 0;
    for (int j = 0; j < a.Lp / 16; ++j) {
        uint4 cv = ld_piece(cost, j);
        uint4 m[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            m[k] = has[k] ? ld_piece(in[k], j) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int d = 16 * j + i;
            const int sh = 8 * (i & 3);
            int b = (int)(((&cv.x)[i >> 2] >> sh) & 0xFF);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                b += (int)(((&m[k].x)[i >> 2] >> sh) & 0xFF);
            if (d < a.L && b < best) {
                best = b;
                bestd = d;
            }
        }
    }
    if (chk(a.labels + (size_t)y * a.labels_pitch + x, 1, kSiteLabel))
        a.labels[(size_t)y * a.labels_pitch + x] = (uint8_t)bestd;
}

// k_bp_labels where the belief sum of every label fits a byte (level-0
// costs in bytes, data_trunc + 4 smooth_trunc <= 255): one 32-bit add sums
// four labels, and the argmin runs on 16-bit keys S(d) * 256 + d, two labels
// per packed minimum, so ties still go to the smallest d.  LP labels at
// compile time; FULL: no padding labels to mask.
template <int LP, bool FULL>
__global__ void __launch_bounds__(128) k_bp_labels_bytes(LabelArgs a)
{
    const int xh = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int c = a.color;
    const int x = 2 * xh + ((c + y) & 1);
    if (x >= a.w || y >= a.h)
        return;
    const bool has[4] = {x > 0, x < a.w - 1, y > 0, y < a.h - 1};
    constexpr int NP = LP / 16;
    const uint8_t *cost = a.cost + slot_base(c * a.h + y, xh, a.wg, NP);
    const uint8_t *in[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        in[k] = a.msg + slot_base((c * 4 + k) * a.h + y, xh, a.wg, NP);
    pdl_begin();   // the index work above overlaps the previous kernel's last wave
    uint32_t best2 = 0xFFFFFFFFu;   // smallest key of the even / odd labels of each pair
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const uint4 cv = ld_piece(cost, j);
        uint4 m[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            m[k] = has[k] ? ld_piece(in[k], j) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int wi = 0; wi < 4; ++wi) {
            const uint32_t s4 = (&cv.x)[wi] + (&m[0].x)[wi] + (&m[1].x)[wi] + (&m[2].x)[wi] + (&m[3].x)[wi];
            const uint32_t d0 = (uint32_t)(16 * j + 4 * wi);
            const uint32_t dd = d0 * 0x01010101u + 0x03020100u;   // the four labels as bytes
            uint32_t k01 = prmt(s4, dd, 0x1504u);                 // (S0 << 8 | d0, S1 << 8 | d1)
            uint32_t k23 = prmt(s4, dd, 0x3726u);                 // (S2 << 8 | d2, S3 << 8 | d3)
            if (!FULL && (int)d0 + 3 >= a.L) {
                const int L = a.L - (int)d0;   // labels of this word that exist
                k01 |= (L <= 0 ? 0xFFFFu : 0u) | (L <= 1 ? 0xFFFF0000u : 0u);
                k23 |= (L <= 2 ? 0xFFFFu : 0u) | (L <= 3 ? 0xFFFF0000u : 0u);
            }
            best2 = min_u16x2(best2, min_u16x2(k01, k23));
        }
    }
    const uint32_t best = min(best2 & 0xFFFFu, best2 >> 16);
    if (chk(a.labels + (size_t)y * a.labels_pitch + x, 1, kSiteLabel))
        a.labels[(size_t)y * a.labels_pitch + x] = (uint8_t)(best & 0xFFu);
}

struct ExportArgs {
    const uint8_t *msg;
    int32_t *out;
    int w, h, wh, wg, L, Lp;
};

__global__ void k_bp_export(ExportArgs a)
{
    pdl_begin();
    const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4u * a.h * a.w * a.L)
        return;
    const int d = (int)(idx % (unsigned)a.L);
    const unsigned px = idx / (unsigned)a.L;
    const int x = (int)(px % (unsigned)a.w);
    const int y = (int)((px / (unsigned)a.w) % (unsigned)a.h);
    const int k = (int)(px / ((unsigned)a.w * (unsigned)a.h));
    const bool has = k == 0 ? x > 0 : k == 1 ? x < a.w - 1 : k == 2 ? y > 0 : y < a.h - 1;
    const int c = (x + y) & 1;
    int v = 0;
    const uint8_t *src = a.msg + slot_base((c * 4 + k) * a.h + y, x >> 1, a.wg, a.Lp / 16) +
                         (size_t)(d >> 4) * kPieceStride + (d & 15);
    if (has && chk(src, 1, kSiteExport))
        v = *src;
    if (chk(a.out + idx, 4, kSiteExport))
        a.out[idx] = v;
}

// ---------------------------------------------------------------------------
// host dispatch

// cost8: the level's data term is stored in bytes; bytes: its belief sums
// fit bytes too (byte-lane arithmetic); labels: the last level-0 iteration
// ---------------------------------------------------------------------------
// kernel variant per level: plain, register preload, or labels split over
// two or four lanes.  Defaults by level size (active-colour slots h * wh);
// the autotuner (vs_bp_autotune) measures the variants on a given problem
// and records the fastest per (label count, level size), which then wins.

enum SweepVariant { kVarPlain = 0, kVarPreload = 1, kVarSplit = 2, kVarSplit4 = 3, kVarStaged = 4 };

// Defaults measured on B300 (vs_bp_autotune_times, eager launches, 2.7K
// flight frames at s = 2, 4, 8, 64 and 128 labels): with up to 64 labels the
// register preload wins at every level size (level 0 at 676x380: 12.5 us vs
// 13.1 plain; at 1352x760: 51.8 vs 64.7) except the smallest levels, where
// four lanes per direction pair shorten the serial chain (85x48: 3.07 vs
// 3.28 us); with 96 / 128 labels two lanes win on the largest levels (141.9
// vs 150.1 us at 1352x760), plain in between, four lanes on the smallest.
constexpr unsigned kSplit4MaxSlots = 1u << 12;    // smaller levels: four lanes
constexpr unsigned kSplitMaxSlots = 1u << 14;     // 32 labels, smaller levels: two lanes
constexpr unsigned kWideSplitMinSlots = 1u << 16; // 96 / 128 labels, larger levels: two lanes

struct TuneEntry {
    int Lp;
    unsigned slots;
    int variant;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;
std::vector<float> g_tune_last;   // ms per launch of the last vs_bp_autotune, [level][variant]
int g_force_variant = -1;         // vs_bp_select_sweep: one variant on every level where allowed
std::atomic<int> g_withhold_copies{0};   // vs_bp_test_withhold_copies

bool variant_allowed(int Lp, int variant, bool labels)
{
    if (variant == kVarStaged)   // chosen in launch_sweep, where eligibility is known
        return false;
    if (labels)
        return variant == kVarPlain;   // only the plain kernel writes labels
    if (variant == kVarSplit)
        return Lp % 32 == 0;
    if (variant == kVarSplit4)
        return Lp % 64 == 0;
    if (variant == kVarPreload)
        return Lp <= 64;
    return true;
}

int choose_variant(int Lp, unsigned slots, bool labels)
{
    if (labels)
        return kVarPlain;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (g_force_variant >= 0 && variant_allowed(Lp, g_force_variant, false))
            return g_force_variant;
        for (const TuneEntry &e : g_tune)
            if (e.Lp == Lp && e.slots == slots && variant_allowed(Lp, e.variant, false))
                return e.variant;
    }
    if (Lp % 64 == 0 && slots < kSplit4MaxSlots)
        return kVarSplit4;
    if (Lp <= 64)
        return (Lp == 32 && slots < kSplitMaxSlots) ? kVarSplit : kVarPreload;
    if (slots >= kWideSplitMinSlots || slots < kSplit4MaxSlots)
        return kVarSplit;
    return kVarPlain;
}

unsigned sweep_blocks(const SweepArgs &a, int variant)
{
    const unsigned lanes = variant == kVarSplit4 ? 8u : (variant == kVarSplit ? 4u : 2u);
    const unsigned threads = lanes * (unsigned)a.h * 16u * (unsigned)a.wg;
    return (threads + kSweepThreads - 1) / kSweepThreads;
}

// Launches one sweep kernel: `a` for a single pair, or `b` (njobs >= 1) for
// a batch; cost8 / bytes / full / labels / variant pick the instantiation.
template <int LP, bool FULL>
void launch_sweep_lp(const SweepArgs *a, const BatchArgs *b, unsigned grid, bool cost8, bool bytes, bool labels,
                     int variant, cudaStream_t st)
{
    const dim3 g(grid), blk(kSweepThreads);
#define VS_SWEEP(...)                                                                                         \
    do {                                                                                                      \
        if (b)                                                                                                \
            launch_pdl(k_bp_sweep_batch<__VA_ARGS__>, g, blk, st, *b);                                        \
        else                                                                                                  \
            launch_pdl(k_bp_sweep<__VA_ARGS__>, g, blk, st, *a);                                              \
    } while (0)
#define VS_SPLIT(...)                                                                                         \
    do {                                                                                                      \
        if (b)                                                                                                \
            launch_pdl(k_bp_sweep_split_batch<__VA_ARGS__>, g, blk, st, *b);                                  \
        else                                                                                                  \
            launch_pdl(k_bp_sweep_split<__VA_ARGS__>, g, blk, st, *a);                                        \
    } while (0)
    if constexpr (LP % 32 == 0) {
        if (variant == kVarSplit) {
            if (cost8 && bytes)
                VS_SPLIT(LP, uint8_t, true, FULL, 2);
            else if (cost8)
                VS_SPLIT(LP, uint8_t, false, FULL, 2);
            else
                VS_SPLIT(LP, uint16_t, false, FULL, 2);
            return;
        }
    }
    if constexpr (LP % 64 == 0) {
        if (variant == kVarSplit4) {
            if (cost8 && bytes)
                VS_SPLIT(LP, uint8_t, true, FULL, 4);
            else if (cost8)
                VS_SPLIT(LP, uint8_t, false, FULL, 4);
            else
                VS_SPLIT(LP, uint16_t, false, FULL, 4);
            return;
        }
    }
    constexpr bool kPre = LP <= 64;   // the preload variant exists up to 64 labels
    const bool pre = kPre && variant == kVarPreload;
    if (cost8 && bytes) {
        if (labels)
            VS_SWEEP(LP, uint8_t, true, FULL, true, false);
        else if (pre)
            VS_SWEEP(LP, uint8_t, true, FULL, false, kPre);
        else
            VS_SWEEP(LP, uint8_t, true, FULL, false, false);
    } else if (cost8) {
        if (labels)
            VS_SWEEP(LP, uint8_t, false, FULL, true, false);
        else if (pre)
            VS_SWEEP(LP, uint8_t, false, FULL, false, kPre);
        else
            VS_SWEEP(LP, uint8_t, false, FULL, false, false);
    } else if (pre) {
        VS_SWEEP(LP, uint16_t, false, FULL, false, kPre);
    } else {
        VS_SWEEP(LP, uint16_t, false, FULL, false, false);
    }
#undef VS_SWEEP
#undef VS_SPLIT
}

template <int LP>
void launch_sweep_full(const SweepArgs *a, const BatchArgs *b, unsigned grid, bool full, bool cost8, bool bytes,
                       bool labels, int variant, cudaStream_t st)
{
    if (full)
        launch_sweep_lp<LP, true>(a, b, grid, cost8, bytes, labels, variant, st);
    else
        launch_sweep_lp<LP, false>(a, b, grid, cost8, bytes, labels, variant, st);
}

void launch_sweep_any(int Lp, const SweepArgs *a, const BatchArgs *b, unsigned grid, bool full, bool cost8,
                      bool bytes, bool labels, int variant, cudaStream_t st)
{
    switch (Lp) {
    case 16: launch_sweep_full<16>(a, b, grid, full, cost8, bytes, labels, variant, st); break;
    case 32: launch_sweep_full<32>(a, b, grid, full, cost8, bytes, labels, variant, st); break;
    case 48: launch_sweep_full<48>(a, b, grid, full, cost8, bytes, labels, variant, st); break;
    case 64: launch_sweep_full<64>(a, b, grid, full, cost8, bytes, labels, variant, st); break;
    case 96: launch_sweep_full<96>(a, b, grid, full, cost8, bytes, labels, variant, st); break;
    default: launch_sweep_full<128>(a, b, grid, full, cost8, bytes, labels, variant, st); break;
    }
}

// One pair's sweep with the variant chosen for its level size.
// The staged kernel serves the single-pair sweeps that read the level's own
// messages with byte costs and byte-lane sums, on levels large enough to
// fill the GPU.
constexpr unsigned kStagedMinSlots = 1u << 16;

bool staged_eligible(const SweepArgs &a, bool cost8, bool bytes)
{
    return cost8 && bytes && !a.from_parent && !a.zero_in && !a.materialize && a.zero_border;
}

// Resident CTAs of a staged instantiation on the current device, cached.
template <int LP, bool FULL, bool LABELS>
int staged_grid_cap()
{
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static int cap[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev)
        return -1;
    std::lock_guard<std::mutex> lk(mu);
    if (cap[dev] == 0) {
        auto kern = k_bp_sweep_staged<LP, FULL, LABELS>;
        constexpr int smem = staged_smem_bytes<LP>();
        int sms = 0, per_sm = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSweepThreads, smem) != cudaSuccess ||
            per_sm < 1)
            return -1;
        cap[dev] = sms * per_sm;
    }
    return cap[dev];
}

// False (nothing launched) when the device cannot host the kernel; the
// caller then takes another variant.
template <int LP, bool FULL, bool LABELS>
bool launch_staged_t(const SweepArgs &a, cudaStream_t st)
{
    const int cap = staged_grid_cap<LP, FULL, LABELS>();
    if (cap < 1) {
        (void)cudaGetLastError();   // the failed attribute or occupancy query
        return false;
    }
    const int ntiles = (a.h * a.wg + 3) / 4;
    launch_pdl_smem(k_bp_sweep_staged<LP, FULL, LABELS>, dim3((unsigned)std::min(ntiles, cap)),
                    dim3(kSweepThreads), (size_t)staged_smem_bytes<LP>(), st, a);
    return true;
}

template <int LP>
bool launch_staged_lp(const SweepArgs &a, bool full, bool labels, cudaStream_t st)
{
    if (full)
        return labels ? launch_staged_t<LP, true, true>(a, st) : launch_staged_t<LP, true, false>(a, st);
    return labels ? launch_staged_t<LP, false, true>(a, st) : launch_staged_t<LP, false, false>(a, st);
}

bool launch_staged(int Lp, const SweepArgs &a, cudaStream_t st)
{
    if ((size_t)a.h * a.wg * (size_t)(Lp / 16) * kPieceStride >= (size_t(1) << 31))
        return false;   // the kernel's 32-bit offsets into one colour-direction array
    const bool full = a.L == Lp, labels = a.labels != nullptr;
    switch (Lp) {
    case 16: return launch_staged_lp<16>(a, full, labels, st);
    case 32: return launch_staged_lp<32>(a, full, labels, st);
    case 48: return launch_staged_lp<48>(a, full, labels, st);
    case 64: return launch_staged_lp<64>(a, full, labels, st);
    case 96: return launch_staged_lp<96>(a, full, labels, st);
    default: return launch_staged_lp<128>(a, full, labels, st);
    }
}

void launch_sweep(int Lp, const SweepArgs &a, bool cost8, bool bytes, cudaStream_t st, int variant = -1)
{
    const bool labels = a.labels != nullptr;
    if (variant < 0 && staged_eligible(a, cost8, bytes)) {
        int forced;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            forced = g_force_variant;
        }
        if ((forced == kVarStaged || (forced < 0 && (unsigned)a.h * (unsigned)a.wh >= kStagedMinSlots)) &&
            launch_staged(Lp, a, st))
            return;
    }
    if (variant < 0)
        variant = choose_variant(Lp, (unsigned)a.h * (unsigned)a.wh, labels);
    launch_sweep_any(Lp, &a, nullptr, sweep_blocks(a, variant), a.L == Lp, cost8, bytes, labels, variant, st);
}

// ---------------------------------------------------------------------------
// fused sweeps: plans and launches

struct FusedPlan {
    int K;        // iterations per launch; 0: the level runs one kernel per iteration
    int TW, TH;   // core tile
    int NS;       // lanes per direction pair: 1, 2 (padded labels % 32 == 0) or 4 (% 64)
};

int fused_smem_bytes(int Lp, int cost_bytes, int TW, int TH, int K)
{
    const int NP = Lp / 16;
    return 16 * (8 * NP + 2 * NP * cost_bytes) * fused_region_rows(TH, K) * fused_region_slots(TW, K);
}

// One lane per direction pair keeps the whole label range in registers:
// compiled up to 64 labels (the register budget of 512 threads per CTA).
bool fused_ns_ok(int Lp, int NS)
{
    return (NS == 1 && Lp <= 64) || (NS == 2 && Lp % 32 == 0) || (NS == 4 && Lp % 64 == 0);
}

// Threads of a fused launch: one per lane of the first iteration's active
// pixels (about half the region, two direction pairs, NS lanes each), whole
// warps, at most kFusedThreads.
int fused_threads(int TW, int TH, int K, int NS)
{
    const int items = fused_region_rows(TH, K) * fused_region_slots(TW, K) * 2 * NS;
    return std::min(kFusedThreads, std::max(64, (items + 31) / 32 * 32));
}

struct DeviceInfo {
    int sms = 0, smem_optin = 0, smem_per_sm = 0;
};

// Multiprocessors and shared-memory limits of the current device, cached.
const DeviceInfo *device_info()
{
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static DeviceInfo info[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        (void)cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    DeviceInfo &d = info[dev];
    if (d.sms == 0) {
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
                cudaSuccess) {
            (void)cudaGetLastError();
            d.sms = 0;
            return nullptr;
        }
    }
    return &d;
}

// Tile shape for K fused iterations on level l, from a model of the launch:
// ceil(CTAs / SMs) x the pixel updates of one CTA's trapezoid, tiles that
// fit the shared memory of one CTA.  K is lowered while no 4 x 4 core fits.
// Lanes per direction pair: enough to give every thread work when the
// region is small.  Returns K = 0 if nothing fits.
FusedPlan fused_default(const BpLayout &lay, int l, int K)
{
    const DeviceInfo *dv = device_info();
    if (!dv)
        return FusedPlan{0, 0, 0, 0};
    const int cb = lay.cost_u8[l] ? 1 : 2;
    const int w = lay.w[l], h = lay.h[l];
    K = std::max(1, std::min(K, 64));
    while (K > 1 && fused_smem_bytes(lay.Lp, cb, 4, 4, K) > dv->smem_optin)
        --K;
    if (fused_smem_bytes(lay.Lp, cb, 4, 4, K) > dv->smem_optin)
        return FusedPlan{0, 0, 0, 0};
    double best = 1e300;
    FusedPlan plan{K, 4, 4, 1};
    for (int TH = 2; TH <= std::max(2, std::min(h, 64)); TH += 2) {
        for (int TW = 2; TW <= std::max(2, std::min(w, 128)); TW += 2) {
            const int smem = fused_smem_bytes(lay.Lp, cb, TW, TH, K);
            if (smem > dv->smem_optin)
                break;
            const long long ctas = (long long)((w + TW - 1) / TW) * ((h + TH - 1) / TH);
            double work = 0.0;
            for (int i = 0; i < K; ++i)
                work += (double)std::min(TW + 2 * (K - i), w) * std::min(TH + 2 * (K - i), h);
            const double t = (double)((ctas + dv->sms - 1) / dv->sms) * work;
            if (t < best * 0.999) {
                best = t;
                plan = FusedPlan{K, TW, TH, 1};
            }
        }
    }
    // the fewest lanes per direction pair (measured fastest: the longer
    // chain of one lane costs less than the joins of several)
    for (int NS : {1, 2, 4})
        if (fused_ns_ok(lay.Lp, NS)) {
            plan.NS = NS;
            break;
        }
    return plan;
}

// Test aid (vs_bp_select_fused): force the core tile and the lanes per
// direction pair of every fused launch (0 = the plan's own).
int g_fused_tw = 0, g_fused_th = 0, g_fused_ns = 0;

// Plans recorded by vs_bp_autotune for the automatic mode, per (padded
// labels, level size, iterations, byte costs); guarded by g_tune_mu.
struct FusedTune {
    int Lp, w, h, iters, cost_u8;
    FusedPlan plan;   // K = 0: the level is faster unfused
};
std::vector<FusedTune> g_fused_tune;

// Automatic mode without a recorded plan.  Measured on B300 in graph
// replays (676 x 380, 64 labels, 4 x 10): levels 1 / 2 / 3 take 41 / 29 / 25
// us unfused against 80 / 41 / 25 us for the fastest fused plans -- with
// programmatic dependent launch a coarse sweep costs 2.5-4 us, less than a
// fused tile's repeated halo work and its one CTA per SM.  Fused launches win
// on small levels (16 labels at 80 x 60 to 160 x 90: 10.4 -> 8.3 us per
// level; the 160 x 120, 16-label pair 34.3 -> 32.6 us per call), so a coarse
// level of at most 240 000 label-pixels runs all its iterations fused;
// larger ones run one kernel per iteration unless vs_bp_autotune measured a
// fused plan faster or iters_per_tile asks for one.
constexpr long long kFusedAutoLabelPixels = 240000;
FusedPlan fused_auto_default(const BpLayout &lay, const vs_bp_params *p, int l)
{
    if ((long long)lay.w[l] * lay.h[l] * lay.Lp <= kFusedAutoLabelPixels)
        return fused_default(lay, l, p->iters);
    return FusedPlan{0, 0, 0, 0};
}

// The plan for level l of a pair: K = 0 (one kernel per iteration), or K
// iterations per launch on tiles.
FusedPlan fused_plan(const BpLayout &lay, const vs_bp_params *p, int l)
{
    FusedPlan fp{0, 0, 0, 0};
    if (l < lay.fused_min_level)
        return fp;
    int tw, th, ns;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tw = g_fused_tw;
        th = g_fused_th;
        ns = g_fused_ns;
        if (p->iters_per_tile == 0) {
            bool found = false;
            for (const FusedTune &e : g_fused_tune)
                if (e.Lp == lay.Lp && e.w == lay.w[l] && e.h == lay.h[l] && e.iters == p->iters &&
                    e.cost_u8 == lay.cost_u8[l]) {
                    fp = e.plan;
                    found = true;
                }
            if (found)
                return fp;
        }
    }
    fp = p->iters_per_tile >= 2 ? fused_default(lay, l, std::min(p->iters_per_tile, p->iters))
                                : fused_auto_default(lay, p, l);
    if (fp.K == 0)
        return fp;
    // test overrides of the tile and the lanes, where they fit
    const DeviceInfo *dv = device_info();
    const int cb = lay.cost_u8[l] ? 1 : 2;
    if (tw > 0 && th > 0 && dv && fused_smem_bytes(lay.Lp, cb, tw, th, fp.K) <= dv->smem_optin) {
        fp.TW = tw;
        fp.TH = th;
    }
    if (ns > 0 && fused_ns_ok(lay.Lp, ns))
        fp.NS = ns;
    return fp;
}

template <int LP, typename CostT, bool BYTES, bool FULL, int NS>
bool launch_fused_t(const FusedArgs &a, unsigned grid, int threads, int smem, cudaStream_t st)
{
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static bool ready[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev)
        return false;
    const DeviceInfo *dv = device_info();
    if (!dv || smem > dv->smem_optin)
        return false;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!ready[dev]) {
            if (cudaFuncSetAttribute(k_bp_fused<LP, CostT, BYTES, FULL, NS>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, dv->smem_optin) != cudaSuccess)
                return false;
            ready[dev] = true;
        }
    }
    launch_pdl_smem(k_bp_fused<LP, CostT, BYTES, FULL, NS>, dim3(grid), dim3(threads), (size_t)smem, st, a);
    return true;
}

template <int LP, typename CostT, bool BYTES, bool FULL>
bool launch_fused_ns(int NS, const FusedArgs &a, unsigned grid, int threads, int smem, cudaStream_t st)
{
    if constexpr (LP % 64 == 0)
        if (NS == 4)
            return launch_fused_t<LP, CostT, BYTES, FULL, 4>(a, grid, threads, smem, st);
    if constexpr (LP % 32 == 0)
        if (NS == 2 || LP > 64)
            return launch_fused_t<LP, CostT, BYTES, FULL, 2>(a, grid, threads, smem, st);
    if constexpr (LP <= 64)
        return launch_fused_t<LP, CostT, BYTES, FULL, 1>(a, grid, threads, smem, st);
    return false;
}

template <int LP>
bool launch_fused_lp(int NS, bool full, bool cost8, bool bytes, const FusedArgs &a, unsigned grid, int threads,
                     int smem, cudaStream_t st)
{
    if (cost8 && bytes)
        return full ? launch_fused_ns<LP, uint8_t, true, true>(NS, a, grid, threads, smem, st)
                    : launch_fused_ns<LP, uint8_t, true, false>(NS, a, grid, threads, smem, st);
    if (cost8)
        return full ? launch_fused_ns<LP, uint8_t, false, true>(NS, a, grid, threads, smem, st)
                    : launch_fused_ns<LP, uint8_t, false, false>(NS, a, grid, threads, smem, st);
    return full ? launch_fused_ns<LP, uint16_t, false, true>(NS, a, grid, threads, smem, st)
                : launch_fused_ns<LP, uint16_t, false, false>(NS, a, grid, threads, smem, st);
}

bool launch_fused(int Lp, int NS, bool full, bool cost8, bool bytes, const FusedArgs &a, unsigned grid,
                  int threads, int smem, cudaStream_t st)
{
    switch (Lp) {
    case 16: return launch_fused_lp<16>(NS, full, cost8, bytes, a, grid, threads, smem, st);
    case 32: return launch_fused_lp<32>(NS, full, cost8, bytes, a, grid, threads, smem, st);
    case 48: return launch_fused_lp<48>(NS, full, cost8, bytes, a, grid, threads, smem, st);
    case 64: return launch_fused_lp<64>(NS, full, cost8, bytes, a, grid, threads, smem, st);
    case 96: return launch_fused_lp<96>(NS, full, cost8, bytes, a, grid, threads, smem, st);
    default: return launch_fused_lp<128>(NS, full, cost8, bytes, a, grid, threads, smem, st);
    }
}

// Arguments of the sweep at level l, iteration t of one pair.
SweepArgs sweep_args(const BpLayout &lay, uint8_t *ws, const vs_bp_params *p, int l, int t, uint8_t *labels,
                     int labels_pitch)
{
    SweepArgs a;
    a.cost = ws + lay.cost_off[l];
    a.msg = ws + lay.msg_off[l];
    a.pmsg = l + 1 < lay.levels ? ws + lay.msg_off[l + 1] : nullptr;
    a.w = lay.w[l];
    a.h = lay.h[l];
    a.wh = lay.wh[l];
    a.wg = lay.wg[l];
    a.L = lay.L;
    a.pw = l + 1 < lay.levels ? lay.w[l + 1] : 0;
    a.ph = l + 1 < lay.levels ? lay.h[l + 1] : 0;
    a.pwh = l + 1 < lay.levels ? lay.wh[l + 1] : 0;
    a.pwg = l + 1 < lay.levels ? lay.wg[l + 1] : 0;
    const int ceff = std::min(p->smooth_slope, p->smooth_trunc);   // same V for any larger slope
    a.c2 = (uint32_t)ceff * 0x10001u;
    a.ts2 = (uint32_t)p->smooth_trunc * 0x10001u;
    a.k256 = 256u;
    a.div_rowslots = fast_div(16u * (uint32_t)a.wg);
    a.color = t & 1;
    a.from_parent = (t == 0 && l + 1 < lay.levels);
    a.zero_in = (t == 0 && l + 1 == lay.levels);
    a.materialize = (t == 0 && p->iters == 1);
    const bool last = l == 0 && t == p->iters - 1;
    a.labels = last ? labels : nullptr;
    a.labels_pitch = labels_pitch;
    a.status = reinterpret_cast<int *>(ws + lay.status_off);
    a.zero_border = l <= 1;
    a.withhold_copies = g_withhold_copies.load(std::memory_order_relaxed);
    return a;
}

// Checked build: bytes taken off the end of the workspace's registered range
// (vs_check_test_shrink); set while a batch runs, whose call registered the
// ranges of all its pairs at once.
size_t g_check_shrink = 0;
bool g_check_in_batch = false;

int check_workspace(const BpLayout &lay, const void *ws, size_t ws_bytes)
{
    if (!ws || !aligned(ws, 256) || ws_bytes < lay.total)
        return VS_EWORKSPACE;
    return VS_OK;
}

}  // namespace
}  // namespace vs

extern "C" size_t vs_bp_workspace_size(int w, int h, const vs_bp_params *p)
{
    using namespace vs;
    if (!params_ok(w, h, p))
        return 0;
    return make_layout(w, h, p).total;
}

namespace vs {
namespace {

// Level-0 data term and the coarse pyramid of one pair.
void launch_costs(const BpLayout &lay, uint8_t *ws, const uint8_t *left, const uint8_t *right, int pitch,
                  const vs_bp_params *p, cudaStream_t st)
{
    {
        Cost01Args a;
        a.left = left;
        a.right = right;
        a.pitch = pitch;
        a.L = lay.L;
        a.Lp = lay.Lp;
        a.Td = p->data_trunc;
        a.w0 = lay.w[0];
        a.h0 = lay.h[0];
        a.wg0 = lay.wg[0];
        a.w1 = (lay.w[0] + 1) / 2;
        a.h1 = (lay.h[0] + 1) / 2;
        a.wg1 = lay.levels > 1 ? lay.wg[1] : 0;
        a.cost0 = ws + lay.cost_off[0];
        a.cost1 = lay.levels > 1 ? ws + lay.cost_off[1] : nullptr;
        a.cost1_u8 = lay.levels > 1 ? lay.cost_u8[1] : 1;
        a.status = reinterpret_cast<int *>(ws + lay.status_off);
        a.msg0 = ws + lay.msg_off[0];
        a.msg1 = lay.levels > 1 ? ws + lay.msg_off[1] : nullptr;
        const dim3 grid((unsigned)((a.w1 + 31) / 32), (unsigned)std::min(a.h1, 65535));
        const int slot = prof_begin(kProfBpOther, st);
        launch_pdl(k_cost01, grid, dim3(32, (unsigned)(lay.Lp / 16)), st, a);
        prof_end(slot, st);
        note_launch();
    }
    const int block = 256;
    for (int l = 2; l < lay.levels; ++l) {
        CostDownArgs a;
        a.fine = ws + lay.cost_off[l - 1];
        a.coarse = ws + lay.cost_off[l];
        a.fine_is_u8 = lay.cost_u8[l - 1];
        a.coarse_is_u8 = lay.cost_u8[l];
        a.wf = lay.w[l - 1];
        a.hf = lay.h[l - 1];
        a.wgf = lay.wg[l - 1];
        a.wc = lay.w[l];
        a.hc = lay.h[l];
        a.wgc = lay.wg[l];
        a.Lp = lay.Lp;
        a.div_chunks = fast_div((uint32_t)lay.Lp / 8u);
        a.div_wgc = fast_div((uint32_t)a.wgc);
        a.div_hc = fast_div((uint32_t)a.hc);
        const long long n = 2LL * a.hc * a.wgc * 16 * (lay.Lp / 8);
        const int slot = prof_begin(kProfBpOther, st);
        launch_pdl(k_cost_down, dim3((unsigned)((n + block - 1) / block)), dim3(block), st, a);
        prof_end(slot, st);
        note_launch();
    }
}

// Labels of the colour the last sweep did not label.
void launch_labels(const BpLayout &lay, uint8_t *ws, uint8_t *labels, int labels_pitch, const vs_bp_params *p,
                   cudaStream_t st)
{
    // the last sweep labelled colour (iters - 1) & 1; this pass labels the other
    LabelArgs a{ws + lay.cost_off[0], ws + lay.msg_off[0], labels, labels_pitch, lay.w[0], lay.h[0], lay.wh[0],
                lay.wg[0], lay.L, lay.Lp, (p->iters & 1)};
    dim3 grid((lay.wh[0] + 127) / 128, lay.h[0]);
    const int slot = prof_begin(kProfBpOther, st);
    if (lay.bytes[0]) {
        const bool full = lay.L == lay.Lp;
#define VS_LABELS(LP)                                                                                         \
    do {                                                                                                      \
        if (full)                                                                                             \
            launch_pdl(k_bp_labels_bytes<LP, true>, dim3(grid), dim3(128), st, a);                           \
        else                                                                                                  \
            launch_pdl(k_bp_labels_bytes<LP, false>, dim3(grid), dim3(128), st, a);                          \
    } while (0)
        switch (lay.Lp) {
        case 16: VS_LABELS(16); break;
        case 32: VS_LABELS(32); break;
        case 48: VS_LABELS(48); break;
        case 64: VS_LABELS(64); break;
        case 96: VS_LABELS(96); break;
        default: VS_LABELS(128); break;
        }
#undef VS_LABELS
    } else {
        launch_pdl(k_bp_labels, dim3(grid), dim3(128), st, a);
    }
    prof_end(slot, st);
    note_launch();
}

// Every iteration of level l in fused launches of fp.K iterations: the
// launches alternate between the level's message buffer and the fused
// scratch buffer, the last one writing the level's own, so the finished
// level sits where the unfused path leaves it.  The launch ending level 0
// writes the labels.  False (nothing launched) if the plan cannot run here.
bool run_level_fused(const BpLayout &lay, uint8_t *ws, const vs_bp_params *p, int l, const FusedPlan &fp,
                     uint8_t *labels, int labels_pitch, cudaStream_t st)
{
    const int K = fp.K, iters = p->iters;
    const int nl = (iters + K - 1) / K;
    const int smem = fused_smem_bytes(lay.Lp, lay.cost_u8[l] ? 1 : 2, fp.TW, fp.TH, K);
    const DeviceInfo *dv = device_info();
    if (!dv || smem > dv->smem_optin || (nl > 1 && lay.fused_bytes < lay.msg_bytes[l]))
        return false;
    uint8_t *bufs[2] = {ws + lay.msg_off[l], ws + lay.fused_off};
    int b = (nl & 1) ? 0 : 1;   // the last launch writes bufs[0]
    FusedArgs a;
    a.cost = ws + lay.cost_off[l];
    a.w = lay.w[l];
    a.h = lay.h[l];
    a.wg = lay.wg[l];
    a.L = lay.L;
    a.pw = l + 1 < lay.levels ? lay.w[l + 1] : 0;
    a.ph = l + 1 < lay.levels ? lay.h[l + 1] : 0;
    a.pwg = l + 1 < lay.levels ? lay.wg[l + 1] : 0;
    a.TW = fp.TW;
    a.TH = fp.TH;
    a.tiles_x = (lay.w[l] + fp.TW - 1) / fp.TW;
    const unsigned grid = (unsigned)a.tiles_x * (unsigned)((lay.h[l] + fp.TH - 1) / fp.TH);
    const int ceff = std::min(p->smooth_slope, p->smooth_trunc);   // same V for any larger slope
    a.c2 = (uint32_t)ceff * 0x10001u;
    a.ts2 = (uint32_t)p->smooth_trunc * 0x10001u;
    a.labels_pitch = labels_pitch;
    const bool full = lay.L == lay.Lp;
    for (int q = 0; q < nl; ++q) {
        a.t0 = q * K;
        a.K = std::min(K, iters - a.t0);
        a.from_parent = q == 0 && l + 1 < lay.levels;
        a.zero_in = q == 0 && l + 1 == lay.levels;
        a.src = a.from_parent ? ws + lay.msg_off[l + 1] : bufs[b ^ 1];
        a.dst = bufs[b];
        a.labels = (l == 0 && q == nl - 1) ? labels : nullptr;
        const int slot = prof_begin(l == 0 ? kProfSweepL0 : kProfSweepCoarse, st);
        const bool ok = launch_fused(lay.Lp, fp.NS, full, lay.cost_u8[l], lay.bytes[l], a, grid,
                                     fused_threads(fp.TW, fp.TH, fp.K, fp.NS), smem, st);
        prof_end(slot, st);
        if (!ok)
            return q == 0 ? false : true;   // a later launch cannot fail where the first ran
        note_launch();
        b ^= 1;
    }
    return true;
}

// Eq. 1 for one pair on `st`: costs and pyramid, every level-iteration, labels.
void run_pair(const BpLayout &lay, uint8_t *ws, const uint8_t *left, const uint8_t *right, int pitch,
              const vs_bp_params *p, uint8_t *labels, int labels_pitch, cudaStream_t st)
{
    if (lay.wide) {
        bp_wide_run(left, right, lay.w[0], lay.h[0], pitch, p, labels, labels_pitch, ws, st,
                    g_check_in_batch ? kCheckKeepRanges : g_check_shrink);
        return;
    }
    launch_costs(lay, ws, left, right, pitch, p, st);
    bool labelled = false;
    for (int l = lay.levels - 1; l >= 0; --l) {
        const FusedPlan fp = fused_plan(lay, p, l);
        if (fp.K > 0 && run_level_fused(lay, ws, p, l, fp, labels, labels_pitch, st)) {
            labelled = labelled || l == 0;
            continue;
        }
        for (int t = 0; t < p->iters; ++t) {
            const SweepArgs a = sweep_args(lay, ws, p, l, t, labels, labels_pitch);
            const int slot = prof_begin(l == 0 ? kProfSweepL0 : kProfSweepCoarse, st);
            launch_sweep(lay.Lp, a, lay.cost_u8[l], lay.bytes[l], st);
            prof_end(slot, st);
            note_launch();
        }
    }
    if (!labelled)
        launch_labels(lay, ws, labels, labels_pitch, p, st);
}

}  // namespace
}  // namespace vs

extern "C" int vs_bp_stereo(const uint8_t *left, const uint8_t *right, int w, int h, int pitch,
                            const vs_bp_params *p, uint8_t *labels, int labels_pitch,
                            void *workspace, size_t ws_bytes, void *stream)
{
    using namespace vs;
    if (!params_ok(w, h, p) || !left || !right || !labels || pitch < w || labels_pitch < w)
        return VS_EINVAL;
    const BpLayout lay = make_layout(w, h, p);
    int rc = check_workspace(lay, workspace, ws_bytes);
    if (rc != VS_OK)
        return rc;
    NvtxRange range("vs_bp_stereo");
    check_ranges((cudaStream_t)stream, {{left, (size_t)(h - 1) * pitch + w}, {right, (size_t)(h - 1) * pitch + w},
                                        {labels, (size_t)(h - 1) * labels_pitch + w}, {workspace, ws_bytes}},
                 g_check_shrink);
    run_pair(lay, reinterpret_cast<uint8_t *>(workspace), left, right, pitch, p, labels, labels_pitch,
             (cudaStream_t)stream);
    return launch_status();
}

// ---------------------------------------------------------------------------
// batch of pairs in lockstep

namespace vs {
namespace {

bool batch_layouts(const vs_bp_job *jobs, int n, std::vector<BpLayout> &lays, std::vector<size_t> &offs,
                   size_t &total)
{
    if (!jobs || n < 1 || n > 4096)
        return false;
    lays.resize(n);
    offs.resize(n);
    total = 0;
    for (int i = 0; i < n; ++i) {
        const vs_bp_job &j = jobs[i];
        if (!params_ok(j.w, j.h, &j.params))
            return false;
        if (j.params.levels != jobs[0].params.levels || j.params.iters != jobs[0].params.iters)
            return false;   // the batch advances every pair through the same steps
        lays[i] = make_layout(j.w, j.h, &j.params);
        offs[i] = total;
        total = align_up(total + lays[i].total, 256);
    }
    return true;
}

}  // namespace
}  // namespace vs

extern "C" size_t vs_bp_batch_workspace_size(const vs_bp_job *jobs, int n)
{
    std::vector<vs::BpLayout> lays;
    std::vector<size_t> offs;
    size_t total = 0;
    return vs::batch_layouts(jobs, n, lays, offs, total) ? total : 0;
}

namespace vs {
namespace {

// Lockstep: every level-iteration of all pairs is a few batched launches
// (one per label count and kernel variant), the jobs in the kernel parameters.
void batch_lockstep(const vs_bp_job *jobs, int n, const std::vector<BpLayout> &lays,
                    const std::vector<size_t> &offs, uint8_t *base, cudaStream_t st)
{
    // pairs of the general path run one after another, ahead of the lockstep ones
    for (int i = 0; i < n; ++i)
        if (lays[i].wide)
            run_pair(lays[i], base + offs[i], jobs[i].left, jobs[i].right, jobs[i].pitch, &jobs[i].params,
                     jobs[i].labels, jobs[i].labels_pitch, st);
    for (int i = 0; i < n; ++i)
        if (!lays[i].wide)
            launch_costs(lays[i], base + offs[i], jobs[i].left, jobs[i].right, jobs[i].pitch, &jobs[i].params,
                         st);

    const int levels = jobs[0].params.levels, iters = jobs[0].params.iters;
    struct Group {
        int Lp, full, cost8, bytes, labels, variant;
        std::vector<SweepArgs> args;
    };
    std::vector<Group> groups;
    for (int l = levels - 1; l >= 0; --l) {
        for (int t = 0; t < iters; ++t) {
            groups.clear();
            for (int i = 0; i < n; ++i) {
                const BpLayout &lay = lays[i];
                if (lay.wide)
                    continue;
                const SweepArgs a = sweep_args(lay, base + offs[i], &jobs[i].params, l, t, jobs[i].labels,
                                               jobs[i].labels_pitch);
                const int labels = a.labels != nullptr;
                const int variant = choose_variant(lay.Lp, (unsigned)a.h * (unsigned)a.wh, labels);
                const int full = a.L == lay.Lp;
                Group *gp = nullptr;
                for (Group &g : groups)
                    if (g.Lp == lay.Lp && g.full == full && g.cost8 == lay.cost_u8[l] && g.bytes == lay.bytes[l] &&
                        g.labels == labels && g.variant == variant)
                        gp = &g;
                if (!gp) {
                    groups.push_back(Group{lay.Lp, full, lay.cost_u8[l], lay.bytes[l], labels, variant, {}});
                    gp = &groups.back();
                }
                gp->args.push_back(a);
            }
            for (const Group &g : groups) {
                for (size_t first = 0; first < g.args.size(); first += kMaxBatch) {
                    BatchArgs b;
                    b.njobs = (int)std::min<size_t>(kMaxBatch, g.args.size() - first);
                    unsigned blocks = 0;
                    for (int k = 0; k < b.njobs; ++k) {
                        b.job[k] = g.args[first + k];
                        b.first_block[k] = blocks;
                        blocks += sweep_blocks(b.job[k], g.variant);
                    }
                    b.first_block[b.njobs] = blocks;
                    const int slot = prof_begin(l == 0 ? kProfSweepL0 : kProfSweepCoarse, st);
                    launch_sweep_any(g.Lp, nullptr, &b, blocks, g.full, g.cost8, g.bytes, g.labels, g.variant, st);
                    prof_end(slot, st);
                    note_launch();
                }
            }
        }
    }
    for (int i = 0; i < n; ++i)
        if (!lays[i].wide)
            launch_labels(lays[i], base + offs[i], jobs[i].labels, jobs[i].labels_pitch, &jobs[i].params, st);

}

// Streams: the pairs, balanced by size (w h labels, largest first, each to
// the least loaded stream), run one after another on the library streams
// forked from `st` and joined back to it by events -- capturable.
// Independent pairs then fill each other's gaps: B300, 48 mixed pairs,
// 28.6 ms against 31.8 ms in lockstep and 33.3 ms one after another.
int batch_streams(const vs_bp_job *jobs, int n, const std::vector<BpLayout> &lays, const std::vector<size_t> &offs,
                  uint8_t *base, cudaStream_t st)
{
    const int S = n < kLibStreams ? n : kLibStreams;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i)
        order[i] = i;
    auto work = [&](int i) {
        const int Lp = lays[i].wide ? 2 * jobs[i].params.labels : lays[i].Lp;   // the general path: about 2x a label
        return (double)jobs[i].w * (double)jobs[i].h * (double)Lp;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
    std::vector<std::vector<int>> queue(S);
    std::vector<double> load(S, 0.0);
    for (int i : order) {
        int k = 0;
        for (int j = 1; j < S; ++j)
            if (load[j] < load[k])
                k = j;
        queue[k].push_back(i);
        load[k] += work(i);
    }
    return fork_join(st, S, [&](int k, cudaStream_t side) {
        for (int i : queue[k])
            run_pair(lays[i], base + offs[i], jobs[i].left, jobs[i].right, jobs[i].pitch, &jobs[i].params,
                     jobs[i].labels, jobs[i].labels_pitch, side);
        return VS_OK;
    });
}

int g_batch_mode = 0;   // 0 streams, 1 lockstep

}  // namespace
}  // namespace vs

extern "C" int vs_bp_batch_mode(int mode)
{
    if (mode != 0 && mode != 1)
        return VS_EINVAL;
    vs::g_batch_mode = mode;
    return VS_OK;
}

extern "C" int vs_bp_stereo_batch(const vs_bp_job *jobs, int n, void *workspace, size_t ws_bytes, void *stream)
{
    using namespace vs;
    std::vector<BpLayout> lays;
    std::vector<size_t> offs;
    size_t total = 0;
    if (!batch_layouts(jobs, n, lays, offs, total))
        return VS_EINVAL;
    for (int i = 0; i < n; ++i) {
        const vs_bp_job &j = jobs[i];
        if (!j.left || !j.right || !j.labels || j.pitch < j.w || j.labels_pitch < j.w)
            return VS_EINVAL;
    }
    if (!workspace || !aligned(workspace, 256) || ws_bytes < total)
        return VS_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t *base = reinterpret_cast<uint8_t *>(workspace);
    NvtxRange range("vs_bp_stereo_batch");
#ifdef VS_CHECKED
    {
        // every job's images and labels and the whole workspace (their hull beyond 64 ranges)
        std::vector<std::pair<const void *, size_t>> bufs;
        for (int i = 0; i < n; ++i) {
            const vs_bp_job &j = jobs[i];
            bufs.push_back({j.left, (size_t)(j.h - 1) * j.pitch + j.w});
            bufs.push_back({j.right, (size_t)(j.h - 1) * j.pitch + j.w});
            bufs.push_back({j.labels, (size_t)(j.h - 1) * j.labels_pitch + j.w});
        }
        bufs.push_back({workspace, ws_bytes});
        check_ranges_list(st, bufs);
        bp_wide_check_ranges(st, bufs);
    }
#endif
    g_check_in_batch = true;
    int rc = VS_OK;
    if (g_batch_mode == 0)
        rc = batch_streams(jobs, n, lays, offs, base, st);
    else
        batch_lockstep(jobs, n, lays, offs, base, st);
    g_check_in_batch = false;
    return rc != VS_OK ? rc : launch_status();
}

// ---------------------------------------------------------------------------
// autotuner

namespace vs {
namespace {

std::vector<int> g_fused_last;       // plans of the last vs_bp_autotune: K, TW, TH, NS per level
std::vector<float> g_fused_last_ms;  // and per level: ms unfused, ms of the fastest fused plan (-1: none)

// Milliseconds per run of level l's iterations -- one kernel per iteration
// (fp.K == 0) or fused launches -- replayed from a CUDA graph on the private
// stream `cs`, the way pipelines run them (launches then overlap through
// programmatic dependent launch; eager launches would mostly time the
// launch latency): one eager run first, then 2 warm-up replays and the mean
// of 10.  -1 on an error or when the plan cannot run here.
float time_level(const BpLayout &lay, uint8_t *ws, const vs_bp_params *p, int l, const FusedPlan &fp,
                 cudaStream_t cs, cudaEvent_t e0, cudaEvent_t e1)
{
    auto run = [&]() -> bool {
        if (fp.K > 0)
            return run_level_fused(lay, ws, p, l, fp, nullptr, 0, cs);
        for (int t = 0; t < p->iters; ++t) {
            const SweepArgs a = sweep_args(lay, ws, p, l, t, nullptr, 0);
            launch_sweep(lay.Lp, a, lay.cost_u8[l], lay.bytes[l], cs);
            note_launch();
        }
        return true;
    };
    if (!run() || cudaStreamSynchronize(cs) != cudaSuccess)
        return -1.0f;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return -1.0f;
    const bool ok = run();
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || !ok || !graph)
        return -1.0f;
    float ms = -1.0f;
    if (cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
        const int reps = 10;
        bool good = cudaGraphLaunch(exec, cs) == cudaSuccess && cudaGraphLaunch(exec, cs) == cudaSuccess &&
                    cudaEventRecord(e0, cs) == cudaSuccess;
        for (int r = 0; r < reps && good; ++r)
            good = cudaGraphLaunch(exec, cs) == cudaSuccess;
        float t = 0.0f;
        if (good && cudaEventRecord(e1, cs) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
            ms = t / reps;
        cudaGraphExecDestroy(exec);
    }
    cudaGraphDestroy(graph);
    return ms;
}

// Fused plans for the automatic mode: for every level that may be fused,
// one kernel per iteration against K = 2..10 iterations per launch on the
// model's tile, tiles of half and twice its sides, and every lane count;
// the fastest is recorded for levels of that size.  The coarser levels'
// messages must be in place (a full run first): each level then starts from
// the same parent state every time.  Level 0 writes labels and stays
// unfused in the automatic mode.
int tune_fused(const BpLayout &lay, uint8_t *ws, const vs_bp_params *p, cudaStream_t st, cudaEvent_t e0,
               cudaEvent_t e1, std::vector<int> &plans, std::vector<float> &level_ms)
{
    plans.assign((size_t)lay.levels * 4, 0);
    level_ms.assign((size_t)lay.levels * 2, -1.0f);
    const DeviceInfo *dv = device_info();
    if (!dv)
        return VS_ECUDA;
    // a private stream for the captures, after the caller's stream's work
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return VS_ECUDA;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return VS_ECUDA;
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } guard{cs};
    for (int l = lay.levels - 1; l >= std::max(1, lay.fused_min_level); --l) {
        const int cb = lay.cost_u8[l] ? 1 : 2;
        std::vector<FusedPlan> cands;
        cands.push_back(FusedPlan{0, 0, 0, 0});
        for (int K : {2, 3, 4, 5, 6, 8, 10}) {
            if (K > p->iters)
                break;
            const FusedPlan d = fused_default(lay, l, K);
            if (d.K == 0)
                continue;
            const int sides[7][2] = {{2, 2}, {1, 2}, {2, 1}, {4, 2}, {2, 4}, {1, 1}, {4, 4}};   // halves
            for (const auto &sc : sides) {
                const int TW = std::max(2, d.TW * sc[0] / 4 * 2), TH = std::max(2, d.TH * sc[1] / 4 * 2);
                if (fused_smem_bytes(lay.Lp, cb, TW, TH, d.K) > dv->smem_optin)
                    continue;
                for (int NS : {1, 2, 4}) {
                    if (!fused_ns_ok(lay.Lp, NS))
                        continue;
                    const FusedPlan c{d.K, TW, TH, NS};
                    bool dup = false;
                    for (const FusedPlan &o : cands)
                        dup = dup || (o.K == c.K && o.TW == c.TW && o.TH == c.TH && o.NS == c.NS);
                    if (!dup)
                        cands.push_back(c);
                }
            }
        }
        float best = 3.4e38f, best_fused = -1.0f;
        FusedPlan best_plan{0, 0, 0, 0};
        for (const FusedPlan &c : cands) {
            const float ms = time_level(lay, ws, p, l, c, cs, e0, e1);
            if (ms < 0.0f) {
                if (c.K == 0)
                    return VS_ECUDA;
                (void)cudaGetLastError();
                continue;
            }
            if (c.K == 0)
                level_ms[(size_t)l * 2] = ms;
            else if (best_fused < 0.0f || ms < best_fused)
                best_fused = ms;
            if (ms < best) {
                best = ms;
                best_plan = c;
            }
        }
        level_ms[(size_t)l * 2 + 1] = best_fused;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            bool found = false;
            for (FusedTune &e : g_fused_tune)
                if (e.Lp == lay.Lp && e.w == lay.w[l] && e.h == lay.h[l] && e.iters == p->iters &&
                    e.cost_u8 == lay.cost_u8[l]) {
                    e.plan = best_plan;
                    found = true;
                }
            if (!found)
                g_fused_tune.push_back(FusedTune{lay.Lp, lay.w[l], lay.h[l], p->iters, lay.cost_u8[l], best_plan});
        }
        plans[(size_t)l * 4 + 0] = best_plan.K;
        plans[(size_t)l * 4 + 1] = best_plan.TW;
        plans[(size_t)l * 4 + 2] = best_plan.TH;
        plans[(size_t)l * 4 + 3] = best_plan.NS;
    }
    return VS_OK;
}

}  // namespace
}  // namespace vs

extern "C" int vs_bp_autotune_plans(int *out, int max)
{
    std::lock_guard<std::mutex> lk(vs::g_tune_mu);
    const int n = (int)vs::g_fused_last.size() < max ? (int)vs::g_fused_last.size() : max;
    for (int i = 0; i < n; ++i)
        out[i] = vs::g_fused_last[i];
    return n;
}

extern "C" int vs_bp_autotune_level_times(float *ms, int max)
{
    std::lock_guard<std::mutex> lk(vs::g_tune_mu);
    const int n = (int)vs::g_fused_last_ms.size() < max ? (int)vs::g_fused_last_ms.size() : max;
    for (int i = 0; i < n; ++i)
        ms[i] = vs::g_fused_last_ms[i];
    return n;
}

extern "C" int vs_bp_autotune(const uint8_t *left, const uint8_t *right, int w, int h, int pitch,
                              const vs_bp_params *p, uint8_t *labels, int labels_pitch, void *workspace,
                              size_t ws_bytes, void *stream, int *chosen)
{
    using namespace vs;
    // a full run first leaves valid state in every level's arrays
    int rc = vs_bp_stereo(left, right, w, h, pitch, p, labels, labels_pitch, workspace, ws_bytes, stream);
    if (rc != VS_OK)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const BpLayout lay = make_layout(w, h, p);
    uint8_t *ws = reinterpret_cast<uint8_t *>(workspace);
    if (lay.wide) {   // the general path has one kernel per step: nothing to choose
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_last.clear();
        g_fused_last.assign((size_t)lay.levels * 4, 0);
        g_fused_last_ms.assign((size_t)lay.levels * 2, -1.0f);
        if (chosen)
            for (int l = 0; l < lay.levels; ++l)
                chosen[l] = -1;
        return VS_OK;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess)
        return VS_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return VS_ECUDA;
    }
    rc = VS_OK;
    std::vector<float> times((size_t)lay.levels * 4, -1.0f);
    for (int l = 0; l < lay.levels && rc == VS_OK; ++l) {
        // an interior iteration of the level (t = 2 reads its own arrays)
        const SweepArgs a = sweep_args(lay, ws, p, l, p->iters > 2 ? 2 : 1, nullptr, 0);
        const unsigned slots = (unsigned)a.h * (unsigned)a.wh;
        float best = 3.4e38f;
        int best_v = kVarPlain;
        for (int v = kVarPlain; v <= kVarSplit4; ++v) {
            if (!variant_allowed(lay.Lp, v, false))
                continue;
            for (int rep = 0; rep < 2; ++rep)   // warm-up
                launch_sweep(lay.Lp, a, lay.cost_u8[l], lay.bytes[l], st, v);
            const int reps = 5;
            cudaEventRecord(e0, st);
            for (int rep = 0; rep < reps; ++rep)
                launch_sweep(lay.Lp, a, lay.cost_u8[l], lay.bytes[l], st, v);
            cudaEventRecord(e1, st);
            note_launch(reps + 2);
            float ms = 0.0f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = VS_ECUDA;
                break;
            }
            times[(size_t)l * 4 + v] = ms / reps;
            if (ms < best) {
                best = ms;
                best_v = v;
            }
        }
        if (rc != VS_OK)
            break;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            bool found = false;
            for (TuneEntry &e : g_tune)
                if (e.Lp == lay.Lp && e.slots == slots) {
                    e.variant = best_v;
                    found = true;
                }
            if (!found)
                g_tune.push_back(TuneEntry{lay.Lp, slots, best_v});
        }
        if (chosen)
            chosen[l] = best_v;
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_last = times;
    }
    if (rc == VS_OK && p->iters_per_tile == 0) {
        // the sweep variants are chosen now: time the levels with them
        std::vector<int> plans;
        std::vector<float> level_ms;
        rc = tune_fused(lay, ws, p, st, e0, e1, plans, level_ms);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_fused_last = plans;
        g_fused_last_ms = level_ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != VS_OK)
        return rc;
    // the timing runs changed the message arrays: run once more so that the
    // workspace and labels hold this problem's result again
    return vs_bp_stereo(left, right, w, h, pitch, p, labels, labels_pitch, workspace, ws_bytes, stream);
}

extern "C" int vs_bp_autotune_times(float *ms, int max)
{
    std::lock_guard<std::mutex> lk(vs::g_tune_mu);
    const int n = (int)vs::g_tune_last.size() < max ? (int)vs::g_tune_last.size() : max;
    for (int i = 0; i < n; ++i)
        ms[i] = vs::g_tune_last[i];
    return n;
}

extern "C" int vs_bp_status(const void *workspace, size_t ws_bytes, int w, int h, const vs_bp_params *p,
                            void *stream)
{
    using namespace vs;
    if (!params_ok(w, h, p))
        return VS_EINVAL;
    const BpLayout lay = make_layout(w, h, p);
    const int rc = check_workspace(lay, workspace, ws_bytes);
    if (rc != VS_OK)
        return rc;
    int status = VS_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&status, static_cast<const uint8_t *>(workspace) + lay.status_off, sizeof(int),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return VS_ECUDA;
    return status == VS_ETIMEOUT ? VS_ETIMEOUT : VS_OK;
}

extern "C" int vs_bp_test_withhold_copies(int on)
{
    if (on != 0 && on != 1)
        return VS_EINVAL;
    vs::g_withhold_copies.store(on, std::memory_order_relaxed);
    return VS_OK;
}

extern "C" int vs_bp_select_sweep(int variant)
{
    if (variant < -1 || variant > 4)
        return VS_EINVAL;
    std::lock_guard<std::mutex> lk(vs::g_tune_mu);
    vs::g_force_variant = variant;
    return VS_OK;
}

extern "C" void vs_bp_autotune_reset(void)
{
    std::lock_guard<std::mutex> lk(vs::g_tune_mu);
    vs::g_tune.clear();
    vs::g_fused_tune.clear();
}

extern "C" int vs_check_report(unsigned long long *site_addr)
{
#ifdef VS_CHECKED
    unsigned long long a0 = 0, a1 = 0;
    const unsigned long long s0 = vs::check_take(&a0);
    const unsigned long long s1 = vs::bp_wide_check_take(&a1);
    const unsigned long long site = s0 ? s0 : s1, addr = s0 ? a0 : a1;
    if (site_addr) {
        site_addr[0] = site ? site - 1 : 0;
        site_addr[1] = addr;
    }
    return site ? 1 : 0;
#else
    (void)site_addr;
    return -1;
#endif
}

extern "C" int vs_check_test_shrink(long long bytes)
{
#ifdef VS_CHECKED
    if (bytes < 0)
        return VS_EINVAL;
    vs::g_check_shrink = (size_t)bytes;
    return VS_OK;
#else
    (void)bytes;
    return VS_EINVAL;
#endif
}

extern "C" int vs_bp_select_fused(int tile_w, int tile_h, int lanes)
{
    if (tile_w < 0 || tile_h < 0 || tile_w > 1024 || tile_h > 1024 || (tile_w == 0) != (tile_h == 0) ||
        (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4))
        return VS_EINVAL;
    std::lock_guard<std::mutex> lk(vs::g_tune_mu);
    vs::g_fused_tw = tile_w;
    vs::g_fused_th = tile_h;
    vs::g_fused_ns = lanes;
    return VS_OK;
}

extern "C" int vs_bp_export_messages(const void *workspace, size_t ws_bytes, int w, int h,
                                     const vs_bp_params *p, int32_t *out, void *stream)
{
    using namespace vs;
    if (!params_ok(w, h, p) || !out)
        return VS_EINVAL;
    const BpLayout lay = make_layout(w, h, p);
    int rc = check_workspace(lay, workspace, ws_bytes);
    if (rc != VS_OK)
        return rc;
    const long long n = 4LL * h * w * lay.L;
    if (n >= (1LL << 31))
        return VS_EINVAL;
    if (lay.wide) {
        bp_wide_export(reinterpret_cast<const uint8_t *>(workspace), w, h, p, out, (cudaStream_t)stream);
        return launch_status();
    }
    check_ranges((cudaStream_t)stream, {{workspace, ws_bytes}, {out, (size_t)n * sizeof(int32_t)}});
    ExportArgs a{reinterpret_cast<const uint8_t *>(workspace) + lay.msg_off[0], out, w, h, lay.wh[0], lay.wg[0], lay.L,
                 lay.Lp};
    launch_pdl(k_bp_export, dim3((unsigned)((n + 255) / 256)), dim3(256), (cudaStream_t)stream, a);
    note_launch();
    return launch_status();
}
