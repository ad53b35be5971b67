// Temperature-smoothed (log-domain sum-product) BP and its adjoint: the
// differentiable relaxation of the Eq. 1 messages, in which the minimum over
// d' becomes the soft minimum -tau log sum exp(-x / tau).
//
// One message, from sender r to receiver p, with h = D_r + the messages r
// received from its other in-frame neighbours and a = min h:
//   u(d')  = exp(-(h(d') - a) / tau)                      (in (0, 1], u = 1 at the minimum)
//   S(d)   = sum_d' K(|d - d'|) u(d'),  K(delta) = exp(-min(lambda delta, T) / tau)
//   mt(d)  = a - tau ln S(d)                              (the soft minimum, exactly)
//   m(d)   = mt(d) - mean mt = tau ln2 (mean_d log2 S - log2 S(d))
// K >= exp(-T/tau) and u(argmin h) = 1, so S(d) >= exp(-T/tau) never
// underflows (T/tau <= 50), and S is a sum of positive terms: no cancellation.
//
// The adjoint of one message, with gt = g - mean g the gradient through the
// normalisation and r(d) = gt(d) / S(d):
//   dL/dh(d')   = u(d') sum_d K(|d - d'|) r(d)
//   dL/dlambda += sum_d' u(d') sum_d Kl(|d - d'|) r(d),  Kl = K delta [lambda delta < T]
//   dL/dT      += sum_d' u(d') sum_d Kt(|d - d'|) r(d),  Kt = K [lambda delta >= T]
//   dL/dtau    += (sum_d gt mt - sum_d' (h - a) dL/dh - lambda dL/dlambda_part - T dL/dT_part) / tau
// (the last from Euler's identity: mt is homogeneous of degree 1 in
// (h, lambda, T, tau); sum_d' dL/dh = sum_d gt = 0 removes a).  The two
// bilinear forms r^T Kl u and r^T Kt u are taken through the correlation
// C(delta) of r and u, so one adjoint message costs 3 L^2 multiply-adds
// (K u, C, K r) with only u and r live.
//
// Layout: D and beliefs [h][w][L] floats; a message state is [4][h][w][L],
// slot k of pixel p holding the message from the neighbour p + off(k),
// off = left, right, up, down; the slot of a missing neighbour holds 0.
// Threads: 4 per pixel (one per slot or per outgoing direction), 32 pixels
// per 128-thread CTA, every label vector in registers, the K tables in the
// kernel parameters (constant bank) so each multiply-add is one FFMA.
#include <atomic>
#include <cmath>
#include <cstdio>

#include "vs_common.cuh"
#include "vs_tcgen05.cuh"

namespace vs {
namespace {

constexpr int kSpThreads = 128;
constexpr int kSpMaxLabels = 64;
constexpr unsigned kFull = 0xffffffffu;

struct SpArgs {
    const float *cost;     // D
    const float *min_;     // message state t - 1 (nullptr: all zero)
    float *mout;           // forward: state t
    float *beliefs;        // forward, last iteration: beliefs instead of a state
    const float *gin;      // adjoint: dL/d(state t), or dL/dbeliefs when from_belief
    float *gout;           // adjoint: dL/d(state t - 1) (nullptr at t = 1)
    float *gcost;          // adjoint: dL/dD, accumulated over iterations
    const float *gbel;     // adjoint: dL/dbeliefs (initial value of dL/dD)
    double *partial;       // adjoint: per-CTA (lambda, T, tau) sums, 4 doubles per CTA
    int *err;              // set to 1 by a tensor-core kernel whose MMA wait timed out
    int withhold_mma;      // test aid: the tensor-core kernels issue no MMA and no commit, so every
                           // bounded wait runs out with nothing in flight
    int w, h, npix;
    int from_belief, first;
    float nc;              // -log2(e) / tau
    float tau_ln2;         // tau ln 2
    float lambda, trunc, tau;
    float k[kSpMaxLabels];
    float kl[kSpMaxLabels];
    float kt[kSpMaxLabels];
    // banded form: K(delta) = kinf = exp(-T / tau) for every delta >= band
    // (lambda delta >= T); kd = K - kinf, zero from the band on
    int band;
    float kinf;
    float kd[kSpMaxLabels];
};

// Widest band of the banded kernels: used when the band of K (labels closer
// than T / lambda) is at most this wide; they come in bands of 4, 6 and 8.
constexpr int kSpBand = 8;

__device__ __forceinline__ int neighbour(int p, int dir, int w, int h)
{
    const int x = p % w, y = p / w;
    switch (dir) {
    case 0: return x > 0 ? p - 1 : -1;
    case 1: return x + 1 < w ? p + 1 : -1;
    case 2: return y > 0 ? p - w : -1;
    default: return y + 1 < h ? p + w : -1;
    }
}

__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

__device__ __forceinline__ void st4(float *p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}

// h = D_q + the three slots of q other than `skip` (state may be nullptr).
// SAME_ROWS: the four lanes of a pixel call this for the same q (sender
// form), so every lane reads all four slots in the same order, the skipped
// one with weight 0: each load instruction then touches one row per pixel
// instead of four.  Otherwise only the three slots are read.
template <int L, bool SAME_ROWS>
__device__ __forceinline__ void gather_h(const SpArgs &a, int q, int skip, float (&h)[L])
{
    const float *dq = a.cost + (size_t)q * L;
#pragma unroll
    for (int c = 0; c < L / 4; ++c) {
        const float4 v = ld4(dq + 4 * c);
        h[4 * c] = v.x, h[4 * c + 1] = v.y, h[4 * c + 2] = v.z, h[4 * c + 3] = v.w;
    }
    if (a.min_ != nullptr) {
        const size_t plane = (size_t)a.npix * L;
#pragma unroll
        for (int i = 0; i < (SAME_ROWS ? 4 : 3); ++i) {
            const int j = SAME_ROWS ? i : (skip + 1 + i) & 3;
            const float f = SAME_ROWS && j == skip ? 0.f : 1.f;
            const float *s = a.min_ + (size_t)j * plane + (size_t)q * L;
#pragma unroll
            for (int c = 0; c < L / 4; ++c) {
                const float4 v = ld4(s + 4 * c);
                h[4 * c] = fmaf(f, v.x, h[4 * c]);
                h[4 * c + 1] = fmaf(f, v.y, h[4 * c + 1]);
                h[4 * c + 2] = fmaf(f, v.z, h[4 * c + 2]);
                h[4 * c + 3] = fmaf(f, v.w, h[4 * c + 3]);
            }
        }
    }
}

// e = h - min h (in place); returns min h.
template <int L>
__device__ __forceinline__ float shift_to_min(float (&e)[L])
{
    float m = e[0];
#pragma unroll
    for (int d = 1; d < L; ++d)
        m = fminf(m, e[d]);
#pragma unroll
    for (int d = 0; d < L; ++d)
        e[d] -= m;
    return m;
}

// s(d) = sum_d' K(|d - d'|) u(d').  BW = 0: the whole L x L product.  BW > 0
// (K constant = kinf from distance BW on): the same sum regrouped exactly as
// kinf sum_d' u(d') + sum over |d - d'| < BW of (K - kinf) u(d'), 2 BW - 1
// multiply-adds per label instead of L; for u >= 0 every term is
// non-negative.
template <int L, int BW>
__device__ __forceinline__ void matvec_k(const SpArgs &a, const float (&u)[L], float (&s)[L])
{
    if constexpr (BW == 0) {
#pragma unroll
        for (int d = 0; d < L; ++d)
            s[d] = 0.f;
#pragma unroll
        for (int dd = 0; dd < L; ++dd)
#pragma unroll
            for (int d = 0; d < L; ++d)
                s[d] = fmaf(a.k[d > dd ? d - dd : dd - d], u[dd], s[d]);
    } else {
        float U = 0.f;
#pragma unroll
        for (int d = 0; d < L; ++d)
            U += u[d];
        const float base = a.kinf * U;
#pragma unroll
        for (int d = 0; d < L; ++d) {
            float acc = base;
#pragma unroll
            for (int del = -(BW - 1); del < BW; ++del)
                if (d + del >= 0 && d + del < L)
                    acc = fmaf(a.kd[del < 0 ? -del : del], u[d + del], acc);
            s[d] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Forward iteration.  State t: thread (r, q) sends the message of r to its
// neighbour nb = r + off(q), which receives it in slot q ^ 1, out of state
// t - 1 (h = D_r + the slots of r other than q); the four lanes of r read the
// same rows, so each gather serves four messages.  A lane whose neighbour is
// missing writes the zero message of r's own slot q instead.  In the last
// iteration (BELIEF) the pull form is used: thread (p, k) computes the
// message p receives in slot k, from r = p + off(k), and the four lanes of p
// add their messages to D_p to write the beliefs.
template <int L, bool BELIEF, int BW>
__global__ void __launch_bounds__(kSpThreads, L <= 48 ? 4 : 3) k_sp_fwd(const __grid_constant__ SpArgs a)
{
    pdl_begin();
    const int gid = blockIdx.x * kSpThreads + threadIdx.x;
    const int p = gid >> 2, k = gid & 3;
    const bool valid = p < a.npix;
    // BELIEF: r sends to p; otherwise p sends to r
    const int r = valid ? neighbour(p, k, a.w, a.h) : -1;
    float m[L];
    if (r >= 0) {
        if (BELIEF)
            gather_h<L, false>(a, r, k ^ 1, m);   // r's slot k^1 holds what p sent it
        else
            gather_h<L, true>(a, p, k, m);        // p's slot k holds what r sent it
        shift_to_min<L>(m);
#pragma unroll
        for (int d = 0; d < L; ++d)
            m[d] = exp2f(m[d] * a.nc);   // u
        float s[L];
        matvec_k<L, BW>(a, m, s);
        float lsum = 0.f;
#pragma unroll
        for (int d = 0; d < L; ++d) {
            s[d] = __log2f(s[d]);
            lsum += s[d];
        }
        const float mean = lsum * (1.0f / L);
#pragma unroll
        for (int d = 0; d < L; ++d)
            m[d] = a.tau_ln2 * (mean - s[d]);
    } else {
#pragma unroll
        for (int d = 0; d < L; ++d)
            m[d] = 0.f;
    }
    if constexpr (!BELIEF) {
        if (valid) {
            // to slot k^1 of the receiver, or a zero into p's own slot k
            float *o = r >= 0 ? a.mout + (size_t)(k ^ 1) * a.npix * L + (size_t)r * L
                              : a.mout + (size_t)k * a.npix * L + (size_t)p * L;
#pragma unroll
            for (int c = 0; c < L / 4; ++c)
                st4(o + 4 * c, m[4 * c], m[4 * c + 1], m[4 * c + 2], m[4 * c + 3]);
        }
    } else {
#pragma unroll
        for (int d = 0; d < L; ++d) {
            float t = m[d] + __shfl_xor_sync(kFull, m[d], 1);
            m[d] = t + __shfl_xor_sync(kFull, t, 2);
        }
        if (valid) {
            const float *dp = a.cost + (size_t)p * L;
            float *o = a.beliefs + (size_t)p * L;
#pragma unroll
            for (int c = 0; c < L / 4; ++c)
                if ((c & 3) == k) {
                    const float4 v = ld4(dp + 4 * c);
                    st4(o + 4 * c, v.x + m[4 * c], v.y + m[4 * c + 1], v.z + m[4 * c + 2], v.w + m[4 * c + 3]);
                }
        }
    }
}

// ---------------------------------------------------------------------------
// Adjoint of one iteration, sender form: thread (p, q) takes the gradient of
// the message p sent to nb = p + off(q) (slot q^1 of nb in dL/d(state t), or
// dL/dbeliefs of nb after the last iteration), recomputes that message from
// state t - 1, and forms dL/dh.  The four lanes of p then give
//   dL/d(slot j of p, state t - 1) = sum over q != j of dL/dh_q
//   dL/dD_p                       += sum over q of dL/dh_q
// and the scalar parts are summed per CTA in double.
template <int L, int BW>
__global__ void __launch_bounds__(kSpThreads, L <= 32 ? 4 : (L == 48 ? 3 : 2)) k_sp_adj(const __grid_constant__ SpArgs a)
{
    pdl_begin();
    const int gid = blockIdx.x * kSpThreads + threadIdx.x;
    const int p = gid >> 2, q = gid & 3;
    const bool valid = p < a.npix;
    const int nb = valid ? neighbour(p, q, a.w, a.h) : -1;
    const size_t plane = (size_t)a.npix * L;
    float e[L];   // h - min h, then u, then dL/dh
    float s_lam = 0.f, s_T = 0.f, s_tau = 0.f;
    if (nb >= 0) {
        gather_h<L, true>(a, p, q, e);
        shift_to_min<L>(e);
#pragma unroll
        for (int d = 0; d < L; ++d)
            e[d] = exp2f(e[d] * a.nc);   // u
        float s[L];
        matvec_k<L, BW>(a, e, s);         // S = K u
        const float *g = a.from_belief ? a.gin + (size_t)nb * L : a.gin + (size_t)(q ^ 1) * plane + (size_t)nb * L;
        float gsum = 0.f;
#pragma unroll
        for (int c = 0; c < L / 4; ++c) {
            const float4 v = ld4(g + 4 * c);
            gsum += (v.x + v.y) + (v.z + v.w);
        }
        const float gmean = gsum * (1.0f / L);
        float glog = 0.f;   // sum_d gt(d) log2 S(d)
#pragma unroll
        for (int c = 0; c < L / 4; ++c) {
            const float4 v = ld4(g + 4 * c);
            const float gv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int d = 4 * c + i;
                const float gt = gv[i] - gmean;
                glog = fmaf(gt, __log2f(s[d]), glog);
                s[d] = __fdividef(gt, s[d]);   // r(d)
            }
        }
        // r^T Kl u and r^T Kt u from the correlation C(delta) = sum over
        // |d - d'| = delta of r(d) u(d'); banded, Kl vanishes from the band on
        // and Kt equals kinf there, so the tail is kinf sum over |d - d'| >= BW
        // of r(d) u(d') = kinf sum_d r(d) (P(d - BW) + Q(d + BW)), with P / Q the
        // prefix / suffix sums of u taken as running sums
        constexpr int NDEL = BW == 0 ? L : BW;
#pragma unroll
        for (int del = 0; del < NDEL; ++del) {
            float cr = 0.f;
#pragma unroll
            for (int d = 0; d + del < L; ++d) {
                cr = fmaf(s[d], e[d + del], cr);
                if (del > 0)
                    cr = fmaf(s[d + del], e[d], cr);
            }
            s_lam = fmaf(a.kl[del], cr, s_lam);
            s_T = fmaf(a.kt[del], cr, s_T);
        }
        if constexpr (BW > 0) {
            float run = 0.f, tail = 0.f;
#pragma unroll
            for (int d = BW; d < L; ++d) {
                run += e[d - BW];
                tail = fmaf(s[d], run, tail);
            }
            run = 0.f;
#pragma unroll
            for (int d = L - 1 - BW; d >= 0; --d) {
                run += e[d + BW];
                tail = fmaf(s[d], run, tail);
            }
            s_T = fmaf(a.kinf, tail, s_T);
        }
        // dL/dh(d') = u(d') (K r)(d'), and sum_d' log2 u(d') dL/dh(d'), where
        // h - a = -tau ln2 log2 u (u = 0 contributes nothing)
        float s_lu = 0.f;
        if constexpr (BW == 0) {
#pragma unroll
            for (int dd = 0; dd < L; ++dd) {
                float V = 0.f;
#pragma unroll
                for (int d = 0; d < L; ++d)
                    V = fmaf(a.k[d > dd ? d - dd : dd - d], s[d], V);
                const float hb = e[dd] * V;
                s_lu = fmaf(__log2f(fmaxf(e[dd], 1e-30f)), hb, s_lu);
                e[dd] = hb;
            }
        } else {
            // (K r)(d') = kinf sum_d r(d) + sum over the band of (K - kinf) r(d)
            float R = 0.f;
#pragma unroll
            for (int d = 0; d < L; ++d)
                R += s[d];
            const float base = a.kinf * R;
#pragma unroll
            for (int dd = 0; dd < L; ++dd) {
                float V = base;
#pragma unroll
                for (int del = -(BW - 1); del < BW; ++del)
                    if (dd + del >= 0 && dd + del < L)
                        V = fmaf(a.kd[del < 0 ? -del : del], s[dd + del], V);
                const float hb = e[dd] * V;
                s_lu = fmaf(__log2f(fmaxf(e[dd], 1e-30f)), hb, s_lu);
                e[dd] = hb;
            }
        }
        // tau dL/dtau = sum_d gt mt - sum_d' (h - a) dL/dh - lambda (.) - T (.),
        // sum_d gt mt = -tau ln2 sum_d gt log2 S
        const float ln2 = 0.6931471805599453f;
        s_tau = -ln2 * glog + ln2 * s_lu - (a.lambda * s_lam + a.trunc * s_T) / a.tau;
    } else {
#pragma unroll
        for (int d = 0; d < L; ++d)
            e[d] = 0.f;
    }

    // combine the four senders of p
    float *go = (valid && a.gout != nullptr) ? a.gout + (size_t)q * plane + (size_t)p * L : nullptr;
    float *gc = a.gcost + (size_t)p * L;
    const float *gb = a.gbel + (size_t)p * L;
#pragma unroll
    for (int c = 0; c < L / 4; ++c) {
        float H[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float v = e[4 * c + i];
            const float t = v + __shfl_xor_sync(kFull, v, 1);
            H[i] = t + __shfl_xor_sync(kFull, t, 2);
        }
        if (go != nullptr)
            st4(go + 4 * c, H[0] - e[4 * c], H[1] - e[4 * c + 1], H[2] - e[4 * c + 2], H[3] - e[4 * c + 3]);
        if (valid && (c & 3) == q) {
            const float4 b = a.first ? ld4(gb + 4 * c) : *reinterpret_cast<const float4 *>(gc + 4 * c);
            st4(gc + 4 * c, b.x + H[0], b.y + H[1], b.z + H[2], b.w + H[3]);
        }
    }

    // per-CTA sums of the scalar parts, in double, in a fixed order
    double v0 = s_lam, v1 = s_T, v2 = s_tau;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(kFull, v0, o);
        v1 += __shfl_xor_sync(kFull, v1, o);
        v2 += __shfl_xor_sync(kFull, v2, o);
    }
    __shared__ double warp_sum[kSpThreads / 32][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        warp_sum[warp][0] = v0;
        warp_sum[warp][1] = v1;
        warp_sum[warp][2] = v2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
#pragma unroll
        for (int wi = 0; wi < kSpThreads / 32; ++wi)
            t += warp_sum[wi][threadIdx.x];
        double *dst = a.partial + 4 * (size_t)blockIdx.x + threadIdx.x;
        *dst = a.first ? t : *dst + t;
    }
}

// ---------------------------------------------------------------------------
// Tensor-core variant.  The label contractions of a tile of 128 messages are
// one MMA each on the 5th-generation tensor cores: A = the 128 x L rows (u,
// or r in the adjoint), B = the L x L Toeplitz tables, D (128 x N, f32) in
// tensor memory with row m in TMEM lane m -- the lane of the thread that
// wrote A row m, so each thread reads back exactly its own message.  FP32
// accuracy comes from a 3xTF32 split, D = Ahi Bhi + Ahi Blo + Alo Bhi (the
// dropped Alo Blo term is 2^-22 relative).
//
// A CTA that holds TMEM gets an SM to itself (the occupancy calculator
// reports one CTA per SM for these kernels, whatever their shared memory), so
// a CTA runs G independent groups of 128 threads.  Each group has its own A
// buffers, TMEM columns and mbarrier and syncs on its own named barrier; the
// B tables are shared.  While one group waits on memory or its MMA, the
// others work.  CTAs are persistent; group g of CTA c takes tiles
// c G + g, c G + g + G gridDim, ...

constexpr int kTcRows = 128;

// Byte offset of (row, 16-byte K chunk) in a K-major canonical tile of
// `rows` rows: chunk-major, 8-row core matrices of 128 bytes.
__host__ __device__ constexpr uint32_t kmaj_off(int row, int chunk, int rows)
{
    return (uint32_t)chunk * (uint32_t)rows * 16u + (uint32_t)(row >> 3) * 128u + (uint32_t)(row & 7) * 16u;
}

constexpr uint32_t pow2_cols(uint32_t n)
{
    return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512;
}

// Per-(kernel, L) plan.  NB rows of B: L (forward: K) or 3L (adjoint:
// [Kl; K; Kt], so [Kl; K] and [K; Kt] are contiguous row ranges).  N columns
// per MMA.  kCorr: column offset of a group's correction accumulator.
template <int L, bool ADJ>
struct TcPlan {
    static constexpr int NB = ADJ ? 3 * L : L;
    static constexpr int N = ADJ ? 2 * L : L;
    static constexpr int G = ADJ ? 2 : (L <= 48 ? 4 : 3);
    static constexpr uint32_t kCorr = pow2_cols(N);
    static constexpr uint32_t kGroupCols = 2 * kCorr;
    static constexpr uint32_t kCols = pow2_cols(G * kGroupCols);
    static constexpr uint32_t kA = kTcRows * L * 4;          // one of A hi / lo
    static constexpr uint32_t kB = NB * L * 4;               // one of B hi / lo
    static constexpr uint32_t kBhi = 0, kBlo = kB;
    static constexpr uint32_t kAhi(int g) { return 2 * kB + 2 * kA * g; }
    static constexpr uint32_t kAlo(int g) { return 2 * kB + 2 * kA * g + kA; }
    static constexpr uint32_t kBar = 2 * kB + 2 * kA * G;    // G mbarriers, then the TMEM slot
    static constexpr uint32_t kBytes = kBar + 8 * G + 8 + 1024;
    static constexpr int kThreads = G * kTcRows;
    static_assert(G * kGroupCols <= 512, "TMEM columns");
    static_assert(kBytes <= 232448, "shared memory");
};

__device__ __forceinline__ uint8_t *align1k(uint8_t *p)
{
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ void group_sync(int g)
{
    asm volatile("bar.sync %0, 128;" ::"r"(g + 1) : "memory");
}

// Barrier over the group's 128 threads that also ORs `v` across them.
__device__ __forceinline__ bool group_any(int g, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(g + 1)
        : "memory");
    return r != 0;
}

// Row `row` of A, split into tf32 hi and lo parts.
template <int L>
__device__ __forceinline__ void store_row_split(uint8_t *sm, uint32_t off_hi, uint32_t off_lo, int row,
                                                const float (&x)[L])
{
#pragma unroll
    for (int c = 0; c < L / 4; ++c) {
        float hi[4], lo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            hi[i] = tc::to_tf32(x[4 * c + i]);
            lo[i] = x[4 * c + i] - hi[i];
        }
        const uint32_t o = kmaj_off(row, c, kTcRows);
        *reinterpret_cast<float4 *>(sm + off_hi + o) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<float4 *>(sm + off_lo + o) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// B tables, split hi / lo.
template <int L, int NB>
__device__ __forceinline__ void build_b(const SpArgs &a, uint8_t *sm, uint32_t off_hi, uint32_t off_lo)
{
    for (int i = threadIdx.x; i < NB * L; i += blockDim.x) {
        const int n = i / L, kk = i - (i / L) * L;
        const int blk = NB == L ? 1 : n / L;
        const int nn = NB == L ? n : n - blk * L;
        const int del = nn > kk ? nn - kk : kk - nn;
        const float v = blk == 0 ? a.kl[del] : (blk == 1 ? a.k[del] : a.kt[del]);
        const float hi = tc::to_tf32(v);
        const uint32_t o = kmaj_off(n, kk >> 2, NB) + (uint32_t)(kk & 3) * 4u;
        *reinterpret_cast<float *>(sm + off_hi + o) = hi;
        *reinterpret_cast<float *>(sm + off_lo + o) = v - hi;
    }
}

// D[:, 0:N) = A (128 x L) * B rows [b_row0, b_row0 + N) (3xTF32), one thread.
// The tensor cores truncate every accumulation step; keeping Ahi Bhi (d_main)
// apart from the two correction products (d_corr) and adding the two in
// registers halves that bias (measured on B300: mean relative error of a
// 48-term contraction 3.6e-7 instead of 6.9e-7; a plain FP32 FMA chain: up to 6e-7).
template <int L, int NB>
__device__ __forceinline__ void issue_mma_3x(const uint8_t *sm, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                             uint32_t b_lo, int b_row0, uint32_t d_main, uint32_t d_corr,
                                             uint32_t idesc)
{
    const uint32_t base = tc::smem_addr(sm);
#pragma unroll
    for (int s = 0; s < L / 8; ++s) {
        const uint32_t ao = kmaj_off(0, 2 * s, kTcRows), bo = kmaj_off(b_row0, 2 * s, NB);
        const uint64_t ahi = tc::smem_desc(base + a_hi + ao, kTcRows * 16, 128);
        const uint64_t alo = tc::smem_desc(base + a_lo + ao, kTcRows * 16, 128);
        const uint64_t bhi = tc::smem_desc(base + b_hi + bo, NB * 16, 128);
        const uint64_t blo = tc::smem_desc(base + b_lo + bo, NB * 16, 128);
        tc::mma_tf32(d_main, ahi, bhi, idesc, s > 0 ? 1u : 0u);
        tc::mma_tf32(d_corr, ahi, blo, idesc, s > 0 ? 1u : 0u);
        tc::mma_tf32(d_corr, alo, bhi, idesc, 1u);
    }
}

// 16 columns of this thread's row: main accumulator + correction accumulator.
__device__ __forceinline__ void tmem_ld16_sum(uint32_t taddr, uint32_t corr_off, float (&v)[16])
{
    float c[16];
    tc::tmem_ld16(taddr, v);
    tc::tmem_ld16(taddr + corr_off, c);
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] += c[i];
}

// Set-up shared by both kernels: B tables, one mbarrier per group, the wait
// for the previous kernel (programmatic dependent launch), then TMEM -- taken
// only once the previous kernel has finished and released its own.
template <int L, bool ADJ>
__device__ __forceinline__ uint32_t tc_setup(const SpArgs &a, uint8_t *sm)
{
    using P = TcPlan<L, ADJ>;
    build_b<L, P::NB>(a, sm, P::kBhi, P::kBlo);   // overlaps the previous kernel's tail
    tc::fence_proxy_async_smem();
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + P::kBar);
    if (threadIdx.x < P::G)
        tc::mbar_init(bars + threadIdx.x, 1);
    pdl_begin();
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + P::kBar + 8 * P::G);
    if ((threadIdx.x >> 5) == 0)
        tc::tmem_alloc(slot, P::kCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    return *slot;
}

// Tear-down: a group whose wait timed out gives its MMAs in flight a second
// bounded wait and records the failure; then TMEM is freed.
template <int L, bool ADJ>
__device__ __forceinline__ void tc_teardown(const SpArgs &a, uint8_t *sm, uint32_t tmem, int g, bool failed,
                                            uint32_t pending_parity)
{
    using P = TcPlan<L, ADJ>;
    if (failed && (threadIdx.x & (kTcRows - 1)) == 0) {
        if (!a.withhold_mma)   // nothing was issued under the test aid
            tc::mbar_wait(reinterpret_cast<uint64_t *>(sm + P::kBar) + g, pending_parity);
        atomicExch(a.err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, P::kCols);
    }
}

// Forward iteration on the tensor cores (pull form, as k_sp_fwd).
template <int L, bool BELIEF>
__global__ void __launch_bounds__(TcPlan<L, false>::kThreads, 1) k_sp_fwd_tc(const __grid_constant__ SpArgs a)
{
    using P = TcPlan<L, false>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align1k(smem_raw);
    const uint32_t tmem0 = tc_setup<L, false>(a, sm);
    const int g = threadIdx.x >> 7, tid = threadIdx.x & (kTcRows - 1);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + P::kBar) + g;
    const uint32_t tmem = tmem0 + g * P::kGroupCols;
    const uint32_t lanes = tmem + ((uint32_t)((tid >> 5) * 32) << 16);
    const uint32_t idesc = tc::idesc_tf32(kTcRows, P::N);

    const int ntiles = (a.npix + 31) / 32;
    uint32_t phase = 0;
    bool failed = false;
    for (int tile = blockIdx.x * P::G + g; tile < ntiles; tile += gridDim.x * P::G) {
        const int p = tile * 32 + (tid >> 2), k = tid & 3;
        const bool valid = p < a.npix;
        const int r = valid ? neighbour(p, k, a.w, a.h) : -1;
        float m[L];
        if (r >= 0) {
            gather_h<L, false>(a, r, k ^ 1, m);
            shift_to_min<L>(m);
#pragma unroll
            for (int d = 0; d < L; ++d)
                m[d] = exp2f(m[d] * a.nc);
        } else {
#pragma unroll
            for (int d = 0; d < L; ++d)
                m[d] = 0.f;
        }
        store_row_split<L>(sm, P::kAhi(g), P::kAlo(g), tid, m);
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        group_sync(g);
        if (tid == 0 && !a.withhold_mma) {
            tc::fence_after_sync();
            issue_mma_3x<L, P::NB>(sm, P::kAhi(g), P::kAlo(g), P::kBhi, P::kBlo, 0, tmem, tmem + P::kCorr, idesc);
            tc::mma_commit(bar);
        }
        const bool ok = tc::mbar_wait(bar, phase);
        phase ^= 1;
        if (group_any(g, !ok)) {
            failed = true;
            break;
        }
        tc::fence_after_sync();
#pragma unroll
        for (int j = 0; j < L / 16; ++j) {
            float v[16];
            tmem_ld16_sum(lanes + 16 * j, P::kCorr, v);
#pragma unroll
            for (int i = 0; i < 16; ++i)
                m[16 * j + i] = v[i];
        }
        if (r >= 0) {
            float lsum = 0.f;
#pragma unroll
            for (int d = 0; d < L; ++d) {
                m[d] = __log2f(m[d]);
                lsum += m[d];
            }
            const float mean = lsum * (1.0f / L);
#pragma unroll
            for (int d = 0; d < L; ++d)
                m[d] = a.tau_ln2 * (mean - m[d]);
        } else {
#pragma unroll
            for (int d = 0; d < L; ++d)
                m[d] = 0.f;
        }
        if constexpr (!BELIEF) {
            if (valid) {
                float *o = a.mout + (size_t)k * a.npix * L + (size_t)p * L;
#pragma unroll
                for (int c = 0; c < L / 4; ++c)
                    st4(o + 4 * c, m[4 * c], m[4 * c + 1], m[4 * c + 2], m[4 * c + 3]);
            }
        } else {
#pragma unroll
            for (int d = 0; d < L; ++d) {
                const float t = m[d] + __shfl_xor_sync(kFull, m[d], 1);
                m[d] = t + __shfl_xor_sync(kFull, t, 2);
            }
            if (valid) {
                const float *dp = a.cost + (size_t)p * L;
                float *o = a.beliefs + (size_t)p * L;
#pragma unroll
                for (int c = 0; c < L / 4; ++c)
                    if ((c & 3) == k) {
                        const float4 v = ld4(dp + 4 * c);
                        st4(o + 4 * c, v.x + m[4 * c], v.y + m[4 * c + 1], v.z + m[4 * c + 2],
                            v.w + m[4 * c + 3]);
                    }
            }
        }
        tc::fence_before_sync();
    }
    tc_teardown<L, false>(a, sm, tmem0, g, failed, phase ^ 1);
}

// Adjoint iteration on the tensor cores (sender form, as k_sp_adj).  Two MMAs
// per tile: [Kl u | K u] from A = u, then [K r | Kt r] from A = r.
template <int L>
__global__ void __launch_bounds__(TcPlan<L, true>::kThreads, 1) k_sp_adj_tc(const __grid_constant__ SpArgs a)
{
    using P = TcPlan<L, true>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align1k(smem_raw);
    const uint32_t tmem0 = tc_setup<L, true>(a, sm);
    const int g = threadIdx.x >> 7, tid = threadIdx.x & (kTcRows - 1);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + P::kBar) + g;
    const uint32_t tmem = tmem0 + g * P::kGroupCols;
    const uint32_t lanes = tmem + ((uint32_t)((tid >> 5) * 32) << 16);
    const uint32_t idesc = tc::idesc_tf32(kTcRows, P::N);

    const size_t plane = (size_t)a.npix * L;
    const int ntiles = (a.npix + 31) / 32;
    const float ln2 = 0.6931471805599453f;
    double acc_lam = 0.0, acc_T = 0.0, acc_tau = 0.0;
    uint32_t phase = 0;
    bool failed = false;
    for (int tile = blockIdx.x * P::G + g; tile < ntiles; tile += gridDim.x * P::G) {
        const int p = tile * 32 + (tid >> 2), q = tid & 3;
        const bool valid = p < a.npix;
        const int nb = valid ? neighbour(p, q, a.w, a.h) : -1;
        float u[L];
        if (nb >= 0) {
            gather_h<L, false>(a, p, q, u);
            shift_to_min<L>(u);
#pragma unroll
            for (int d = 0; d < L; ++d)
                u[d] = exp2f(u[d] * a.nc);
        } else {
#pragma unroll
            for (int d = 0; d < L; ++d)
                u[d] = 0.f;
        }
        store_row_split<L>(sm, P::kAhi(g), P::kAlo(g), tid, u);
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        group_sync(g);
        if (tid == 0 && !a.withhold_mma) {
            tc::fence_after_sync();
            issue_mma_3x<L, P::NB>(sm, P::kAhi(g), P::kAlo(g), P::kBhi, P::kBlo, 0, tmem, tmem + P::kCorr, idesc);
            tc::mma_commit(bar);
        }
        // while the tensor cores work: the gradient of the message p -> nb
        const float *gp = nullptr;
        float gmean = 0.f;
        if (nb >= 0) {
            gp = a.from_belief ? a.gin + (size_t)nb * L : a.gin + (size_t)(q ^ 1) * plane + (size_t)nb * L;
            float gsum = 0.f;
#pragma unroll
            for (int c = 0; c < L / 4; ++c) {
                const float4 v = ld4(gp + 4 * c);
                gsum += (v.x + v.y) + (v.z + v.w);
            }
            gmean = gsum * (1.0f / L);
        }
        bool ok = tc::mbar_wait(bar, phase);
        phase ^= 1;
        if (group_any(g, !ok)) {
            failed = true;
            break;
        }
        tc::fence_after_sync();
        // r = gt / S into A; glog = sum gt log2 S; s_lam = r . (Kl u)
        float glog = 0.f, s_lam = 0.f;
#pragma unroll
        for (int j = 0; j < L / 16; ++j) {
            float S[16], Klu[16], r[16];
            tmem_ld16_sum(lanes + L + 16 * j, P::kCorr, S);
            tmem_ld16_sum(lanes + 16 * j, P::kCorr, Klu);
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
                float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
                if (nb >= 0)
                    gv = ld4(gp + 16 * j + 4 * c4);
                const float gs[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int e = 4 * c4 + i;
                    if (nb >= 0) {
                        const float gt = gs[i] - gmean;
                        glog = fmaf(gt, __log2f(S[e]), glog);
                        r[e] = __fdividef(gt, S[e]);
                        s_lam = fmaf(r[e], Klu[e], s_lam);
                    } else {
                        r[e] = 0.f;
                    }
                }
            }
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
                const int c = 4 * j + c4;
                float hi[4], lo[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    hi[i] = tc::to_tf32(r[4 * c4 + i]);
                    lo[i] = r[4 * c4 + i] - hi[i];
                }
                const uint32_t o = kmaj_off(tid, c, kTcRows);
                *reinterpret_cast<float4 *>(sm + P::kAhi(g) + o) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<float4 *>(sm + P::kAlo(g) + o) = make_float4(lo[0], lo[1], lo[2], lo[3]);
            }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        group_sync(g);
        if (tid == 0 && !a.withhold_mma) {
            tc::fence_after_sync();
            issue_mma_3x<L, P::NB>(sm, P::kAhi(g), P::kAlo(g), P::kBhi, P::kBlo, L, tmem, tmem + P::kCorr, idesc);
            tc::mma_commit(bar);
        }
        ok = tc::mbar_wait(bar, phase);
        phase ^= 1;
        if (group_any(g, !ok)) {
            failed = true;
            break;
        }
        tc::fence_after_sync();
        // dL/dh = u (K r); s_T = u . (Kt r); s_lu = sum log2(u) dL/dh
        float s_T = 0.f, s_lu = 0.f;
#pragma unroll
        for (int j = 0; j < L / 16; ++j) {
            float V[16], Ktr[16];
            tmem_ld16_sum(lanes + 16 * j, P::kCorr, V);
            tmem_ld16_sum(lanes + L + 16 * j, P::kCorr, Ktr);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int d = 16 * j + i;
                const float hb = u[d] * V[i];
                s_T = fmaf(u[d], Ktr[i], s_T);
                s_lu = fmaf(__log2f(fmaxf(u[d], 1e-30f)), hb, s_lu);
                u[d] = hb;
            }
        }
        if (nb >= 0) {
            acc_lam += (double)s_lam;
            acc_T += (double)s_T;
            acc_tau += (double)(-ln2 * glog + ln2 * s_lu - (a.lambda * s_lam + a.trunc * s_T) / a.tau);
        }
        // combine the four senders of p
        float *go = (valid && a.gout != nullptr) ? a.gout + (size_t)q * plane + (size_t)p * L : nullptr;
        float *gc = a.gcost + (size_t)p * L;
        const float *gb = a.gbel + (size_t)p * L;
#pragma unroll
        for (int c = 0; c < L / 4; ++c) {
            float H[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float v = u[4 * c + i];
                const float t = v + __shfl_xor_sync(kFull, v, 1);
                H[i] = t + __shfl_xor_sync(kFull, t, 2);
            }
            if (go != nullptr)
                st4(go + 4 * c, H[0] - u[4 * c], H[1] - u[4 * c + 1], H[2] - u[4 * c + 2], H[3] - u[4 * c + 3]);
            if (valid && (c & 3) == q) {
                const float4 b = a.first ? ld4(gb + 4 * c) : *reinterpret_cast<const float4 *>(gc + 4 * c);
                st4(gc + 4 * c, b.x + H[0], b.y + H[1], b.z + H[2], b.w + H[3]);
            }
        }
        tc::fence_before_sync();
    }

    // per-CTA sums of the scalar parts, in double, in a fixed order
    double v0 = acc_lam, v1 = acc_T, v2 = acc_tau;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(kFull, v0, o);
        v1 += __shfl_xor_sync(kFull, v1, o);
        v2 += __shfl_xor_sync(kFull, v2, o);
    }
    __shared__ double warp_sum[P::kThreads / 32][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        warp_sum[warp][0] = v0;
        warp_sum[warp][1] = v1;
        warp_sum[warp][2] = v2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
#pragma unroll
        for (int wi = 0; wi < P::kThreads / 32; ++wi)
            t += warp_sum[wi][threadIdx.x];
        double *dst = a.partial + 4 * (size_t)blockIdx.x + threadIdx.x;
        *dst = a.first ? t : *dst + t;
    }
    tc_teardown<L, true>(a, sm, tmem0, g, failed, phase ^ 1);
}

// grad_params[i] = sum over CTAs of partial[cta][i], in double, fixed order.
__global__ void __launch_bounds__(256) k_sp_reduce(const double *partial, int nblocks, float *out)
{
    pdl_begin();
    __shared__ double sh[3][256];
    double t[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += 256)
        for (int i = 0; i < 3; ++i)
            t[i] += partial[4 * (size_t)b + i];
    for (int i = 0; i < 3; ++i)
        sh[i][threadIdx.x] = t[i];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int i = 0; i < 3; ++i)
                sh[i][threadIdx.x] += sh[i][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 3)
        out[threadIdx.x] = (float)sh[threadIdx.x][0];
}

// ---------------------------------------------------------------------------
// host side

struct SpLayout {
    size_t state_bytes, partial_bytes, total;
    int nck, nseg, nblocks;   // nblocks: 32-pixel tiles (an upper bound on the partial-sum slots)
};

bool sp_valid(int w, int h, const vs_sp_params *p)
{
    if (p == nullptr || w < 1 || h < 1 || (int64_t)w * h > (int64_t(1) << 22))
        return false;
    if (p->labels != 16 && p->labels != 32 && p->labels != 48 && p->labels != 64)
        return false;
    if (p->iters < 1 || p->iters > 64 || p->ckpt_every < 1 || p->ckpt_every > p->iters)
        return false;
    if (!std::isfinite(p->lambda) || !std::isfinite(p->trunc) || !std::isfinite(p->tau))
        return false;
    if (p->lambda < 0.f || p->trunc < 0.f || !(p->tau > 0.f))
        return false;
    return (double)p->trunc / (double)p->tau <= 50.0;
}

SpLayout sp_layout(int w, int h, const vs_sp_params *p)
{
    SpLayout lay;
    const size_t npix = (size_t)w * h;
    lay.state_bytes = align_up(16 * npix * (size_t)p->labels, 256);
    lay.nblocks = (int)((4 * npix + kSpThreads - 1) / kSpThreads);
    lay.partial_bytes = align_up((size_t)lay.nblocks * 4 * sizeof(double), 256);
    lay.nck = (p->iters - 1) / p->ckpt_every;
    lay.nseg = (p->ckpt_every < p->iters ? p->ckpt_every : p->iters) - 1;
    lay.total = (size_t)(lay.nck + lay.nseg + 2) * lay.state_bytes + lay.partial_bytes + 256;
    return lay;
}

struct SpStates {
    char *base;
    SpLayout lay;
    float *ckpt(int i) const { return reinterpret_cast<float *>(base + (size_t)i * lay.state_bytes); }
    float *seg(int i) const { return reinterpret_cast<float *>(base + (size_t)(lay.nck + i) * lay.state_bytes); }
    float *adj(int i) const
    {
        return reinterpret_cast<float *>(base + (size_t)(lay.nck + lay.nseg + i) * lay.state_bytes);
    }
    double *partial() const
    {
        return reinterpret_cast<double *>(base + (size_t)(lay.nck + lay.nseg + 2) * lay.state_bytes);
    }
    int *err() const
    {
        return reinterpret_cast<int *>(base + (size_t)(lay.nck + lay.nseg + 2) * lay.state_bytes +
                                       lay.partial_bytes);
    }
};

void fill_tables(SpArgs &a, const vs_sp_params *p)
{
    const double lam = p->lambda, T = p->trunc, tau = p->tau;
    for (int del = 0; del < kSpMaxLabels; ++del) {
        const double x = lam * del;
        const bool lin = x < T;
        const double k = std::exp(-(lin ? x : T) / tau);
        a.k[del] = (float)k;
        a.kl[del] = lin ? (float)(k * del) : 0.f;
        a.kt[del] = lin ? 0.f : (float)k;
    }
    const double kinf = std::exp(-T / tau);
    a.band = 0;
    while (a.band < kSpMaxLabels && lam * a.band < T)   // the same test as `lin` above
        ++a.band;
    a.kinf = (float)kinf;
    for (int del = 0; del < kSpMaxLabels; ++del)
        a.kd[del] = lam * del < T ? (float)(std::exp(-lam * del / tau) - kinf) : 0.f;
    a.nc = (float)(-1.0 / (tau * std::log(2.0)));
    a.tau_ln2 = (float)(tau * std::log(2.0));
    a.lambda = p->lambda;
    a.trunc = p->trunc;
    a.tau = p->tau;
}

// Kernel family: 1 = SIMT FP32 (default), 0 = tensor cores.  Measured on
// B300 at 338 x 190 x 48: SIMT 65 us per forward and 165 us per adjoint
// iteration, the tensor-core kernels 86-138 us and 163 us, with about twice
// the rounding error (the MMA truncates each accumulation).  The 48-label
// contraction is small next to the gathers, which leave the tensor-core
// kernels latency-bound with one CTA per SM.
int g_sp_kernels = 1;
std::atomic<int> g_withhold_mma{0};   // vs_sp_test_withhold_mma

// Persistent grid of a tensor-core kernel: resident CTAs per SM x SMs, at
// most one CTA per tile.  The kernel asks for the largest shared-memory
// carve-out, without which the driver may size it for one CTA per SM.
template <typename Kern>
int tc_grid(Kern kern, int threads, uint32_t smem, int groups, int ntiles)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
            cudaSuccess)
        return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
        return -1;
    const int g = sms * per_sm, need = (ntiles + groups - 1) / groups;
    return g < need ? g : need;
}

inline cudaLaunchConfig_t pdl_config(dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                      cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Band of the SIMT kernels for these parameters: the smallest compiled band
// (4, 6, 8) that holds the band of K, or 0 (the full product) for a wider
// band or 16 labels, where the full product is as cheap.
template <int L>
int sp_band(const SpArgs &a)
{
    if (L < 32 || a.band > kSpBand)
        return 0;
    return a.band <= 4 ? 4 : (a.band <= 6 ? 6 : 8);
}

// One forward iteration (pull form); with belief = true the last one, which
// writes the beliefs instead of a message state.
template <int L>
int launch_fwd(const SpArgs &a, bool belief, cudaStream_t st)
{
    const int slot = prof_begin(kProfSmoothFwd, st);
    const int ntiles = (a.npix + 31) / 32;
    cudaLaunchAttribute attr[1];
    cudaError_t err;
    if (g_sp_kernels == 0) {
        using P = TcPlan<L, false>;
        const int grid = belief ? tc_grid(k_sp_fwd_tc<L, true>, P::kThreads, P::kBytes, P::G, ntiles)
                                : tc_grid(k_sp_fwd_tc<L, false>, P::kThreads, P::kBytes, P::G, ntiles);
        if (grid < 1) {
            prof_end(slot, st);
            return VS_ECUDA;
        }
        cudaLaunchConfig_t cfg = pdl_config(dim3(grid), dim3(P::kThreads), P::kBytes, st, attr);
        err = belief ? cudaLaunchKernelEx(&cfg, k_sp_fwd_tc<L, true>, a)
                     : cudaLaunchKernelEx(&cfg, k_sp_fwd_tc<L, false>, a);
    } else {
        const int nblocks = (int)(((size_t)4 * a.npix + kSpThreads - 1) / kSpThreads);
        cudaLaunchConfig_t cfg = pdl_config(dim3(nblocks), dim3(kSpThreads), 0, st, attr);
        switch (sp_band<L>(a)) {
        case 4:
            err = belief ? cudaLaunchKernelEx(&cfg, k_sp_fwd<L, true, 4>, a)
                         : cudaLaunchKernelEx(&cfg, k_sp_fwd<L, false, 4>, a);
            break;
        case 6:
            err = belief ? cudaLaunchKernelEx(&cfg, k_sp_fwd<L, true, 6>, a)
                         : cudaLaunchKernelEx(&cfg, k_sp_fwd<L, false, 6>, a);
            break;
        case 8:
            err = belief ? cudaLaunchKernelEx(&cfg, k_sp_fwd<L, true, 8>, a)
                         : cudaLaunchKernelEx(&cfg, k_sp_fwd<L, false, 8>, a);
            break;
        default:
            err = belief ? cudaLaunchKernelEx(&cfg, k_sp_fwd<L, true, 0>, a)
                         : cudaLaunchKernelEx(&cfg, k_sp_fwd<L, false, 0>, a);
        }
    }
    prof_end(slot, st);
    note_launch();
    return err == cudaSuccess ? VS_OK : VS_ECUDA;
}

// Grid of the adjoint kernel (also the number of partial-sum slots it fills).
template <int L>
int adj_grid(int npix)
{
    const int ntiles = (npix + 31) / 32;   // = CTAs of the SIMT kernel (32 pixels x 4 lanes)
    if (g_sp_kernels != 0)
        return ntiles;
    using P = TcPlan<L, true>;
    return tc_grid(k_sp_adj_tc<L>, P::kThreads, P::kBytes, P::G, ntiles);
}

template <int L>
int launch_adj(const SpArgs &a, int grid, cudaStream_t st)
{
    const int slot = prof_begin(kProfSmoothAdj, st);
    cudaLaunchAttribute attr[1];
    cudaError_t err;
    if (g_sp_kernels == 0) {
        using P = TcPlan<L, true>;
        cudaLaunchConfig_t cfg = pdl_config(dim3(grid), dim3(P::kThreads), P::kBytes, st, attr);
        err = cudaLaunchKernelEx(&cfg, k_sp_adj_tc<L>, a);
    } else {
        cudaLaunchConfig_t cfg = pdl_config(dim3(grid), dim3(kSpThreads), 0, st, attr);
        switch (sp_band<L>(a)) {
        case 4: err = cudaLaunchKernelEx(&cfg, k_sp_adj<L, 4>, a); break;
        case 6: err = cudaLaunchKernelEx(&cfg, k_sp_adj<L, 6>, a); break;
        case 8: err = cudaLaunchKernelEx(&cfg, k_sp_adj<L, 8>, a); break;
        default: err = cudaLaunchKernelEx(&cfg, k_sp_adj<L, 0>, a);
        }
    }
    prof_end(slot, st);
    note_launch();
    return err == cudaSuccess ? VS_OK : VS_ECUDA;
}

int fwd_any(int L, const SpArgs &a, bool belief, cudaStream_t st)
{
    switch (L) {
    case 16: return launch_fwd<16>(a, belief, st);
    case 32: return launch_fwd<32>(a, belief, st);
    case 48: return launch_fwd<48>(a, belief, st);
    default: return launch_fwd<64>(a, belief, st);
    }
}

int adj_grid_any(int L, int npix)
{
    switch (L) {
    case 16: return adj_grid<16>(npix);
    case 32: return adj_grid<32>(npix);
    case 48: return adj_grid<48>(npix);
    default: return adj_grid<64>(npix);
    }
}

int adj_any(int L, const SpArgs &a, int grid, cudaStream_t st)
{
    switch (L) {
    case 16: return launch_adj<16>(a, grid, st);
    case 32: return launch_adj<32>(a, grid, st);
    case 48: return launch_adj<48>(a, grid, st);
    default: return launch_adj<64>(a, grid, st);
    }
}

int sp_check_ws(const void *ws, size_t ws_bytes, const SpLayout &lay)
{
    if (ws == nullptr || !aligned(ws, 256) || ws_bytes < lay.total)
        return VS_EWORKSPACE;
    return VS_OK;
}

}  // namespace
}  // namespace vs

using namespace vs;

extern "C" size_t vs_sp_workspace_size(int w, int h, const vs_sp_params *p)
{
    if (!sp_valid(w, h, p))
        return 0;
    return sp_layout(w, h, p).total;
}

extern "C" int vs_sp_select_kernels(int family)
{
    if (family != 0 && family != 1)
        return VS_EINVAL;
    g_sp_kernels = family;
    return VS_OK;
}

extern "C" int vs_sp_forward(const float *cost, int w, int h, const vs_sp_params *p, float *beliefs,
                             void *workspace, size_t ws_bytes, void *stream)
{
    vs::NvtxRange nvtx_range("vs_sp_forward");
    if (!sp_valid(w, h, p) || cost == nullptr || beliefs == nullptr)
        return VS_EINVAL;
    if (!aligned(cost, 16) || !aligned(beliefs, 16))
        return VS_EALIGN;
    const SpLayout lay = sp_layout(w, h, p);
    if (int rc = sp_check_ws(workspace, ws_bytes, lay))
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    SpStates S{static_cast<char *>(workspace), lay};
    if (cudaMemsetAsync(S.err(), 0, sizeof(int), st) != cudaSuccess)
        return VS_ECUDA;
    SpArgs a = {};
    fill_tables(a, p);
    a.cost = cost;
    a.err = S.err();
    a.withhold_mma = g_withhold_mma.load(std::memory_order_relaxed);
    a.w = w, a.h = h, a.npix = w * h;
    a.beliefs = beliefs;
    const int K = p->iters, c = p->ckpt_every;
    const float *prev = nullptr;
    for (int t = 1; t <= K; ++t) {
        a.min_ = prev;
        if (t == K) {
            a.mout = nullptr;
            if (int rc = fwd_any(p->labels, a, true, st))
                return rc;
        } else {
            float *out = (t % c == 0) ? S.ckpt(t / c - 1) : S.adj(t & 1);
            a.mout = out;
            if (int rc = fwd_any(p->labels, a, false, st))
                return rc;
            prev = out;
        }
    }
    return launch_status();
}

extern "C" int vs_sp_backward(const float *cost, int w, int h, const vs_sp_params *p, const float *grad_beliefs,
                              float *grad_cost, float *grad_params, void *workspace, size_t ws_bytes, void *stream)
{
    vs::NvtxRange nvtx_range("vs_sp_backward");
    if (!sp_valid(w, h, p) || cost == nullptr || grad_beliefs == nullptr || grad_cost == nullptr ||
        grad_params == nullptr)
        return VS_EINVAL;
    if (!aligned(cost, 16) || !aligned(grad_beliefs, 16) || !aligned(grad_cost, 16) || !aligned(grad_params, 4))
        return VS_EALIGN;
    const SpLayout lay = sp_layout(w, h, p);
    if (int rc = sp_check_ws(workspace, ws_bytes, lay))
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    SpStates S{static_cast<char *>(workspace), lay};
    SpArgs a = {};
    fill_tables(a, p);
    a.cost = cost;
    a.err = S.err();
    a.withhold_mma = g_withhold_mma.load(std::memory_order_relaxed);
    a.w = w, a.h = h, a.npix = w * h;
    a.gcost = grad_cost;
    a.gbel = grad_beliefs;
    a.partial = S.partial();
    const int K = p->iters, c = p->ckpt_every, L = p->labels;
    const int grid = adj_grid_any(L, a.npix);
    if (grid < 1)
        return VS_ECUDA;

    const float *gin = grad_beliefs;
    int from_belief = 1, first = 1, x = 0;
    for (int s0 = c * ((K - 1) / c); s0 >= 0; s0 -= c) {
        const int top = s0 + c < K ? s0 + c : K;
        const float *base = s0 == 0 ? nullptr : S.ckpt(s0 / c - 1);
        // recompute states s0 + 1 .. top - 1 of this segment from its checkpoint
        SpArgs f = a;
        const float *prev = base;
        for (int t = s0 + 1; t < top; ++t) {
            f.min_ = prev;
            f.mout = S.seg(t - s0 - 1);
            if (int rc = fwd_any(L, f, false, st))
                return rc;
            prev = f.mout;
        }
        for (int t = top; t > s0; --t) {
            a.min_ = (t - 1 == s0) ? base : S.seg(t - 1 - s0 - 1);
            a.gin = gin;
            a.gout = t > 1 ? S.adj(x) : nullptr;
            a.from_belief = from_belief;
            a.first = first;
            if (int rc = adj_any(L, a, grid, st))
                return rc;
            gin = a.gout;
            from_belief = 0;
            first = 0;
            x ^= 1;
        }
    }
    const cudaError_t err = launch_pdl(k_sp_reduce, dim3(1), dim3(256), st, (const double *)S.partial(), grid,
                                       grad_params);
    note_launch();
    if (err != cudaSuccess)
        return VS_ECUDA;
    return launch_status();
}

extern "C" int vs_sp_test_withhold_mma(int on)
{
    if (on != 0 && on != 1)
        return VS_EINVAL;
    vs::g_withhold_mma.store(on, std::memory_order_relaxed);
    return VS_OK;
}

extern "C" int vs_sp_status(const void *workspace, size_t ws_bytes, int w, int h, const vs_sp_params *p,
                            void *stream)
{
    if (!sp_valid(w, h, p))
        return VS_EINVAL;
    const SpLayout lay = sp_layout(w, h, p);
    if (int rc = sp_check_ws(workspace, ws_bytes, lay))
        return rc;
    SpStates S{static_cast<char *>(const_cast<void *>(workspace)), lay};
    int flag = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&flag, S.err(), sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return VS_ECUDA;
    return flag ? VS_ETIMEOUT : VS_OK;
}
