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
#include <cmath>
#include <cstdio>

#include "vs_common.cuh"

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
    int w, h, npix;
    int from_belief, first;
    float nc;              // -log2(e) / tau
    float tau_ln2;         // tau ln 2
    float lambda, trunc, tau;
    float k[kSpMaxLabels];
    float kl[kSpMaxLabels];
    float kt[kSpMaxLabels];
};

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
template <int L>
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
        for (int i = 0; i < 3; ++i) {
            const int j = (skip + 1 + i) & 3;
            const float *s = a.min_ + (size_t)j * plane + (size_t)q * L;
#pragma unroll
            for (int c = 0; c < L / 4; ++c) {
                const float4 v = ld4(s + 4 * c);
                h[4 * c] += v.x, h[4 * c + 1] += v.y, h[4 * c + 2] += v.z, h[4 * c + 3] += v.w;
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

// s(d) = sum_d' K(|d - d'|) u(d').
template <int L>
__device__ __forceinline__ void matvec_k(const SpArgs &a, const float (&u)[L], float (&s)[L])
{
#pragma unroll
    for (int d = 0; d < L; ++d)
        s[d] = 0.f;
#pragma unroll
    for (int dd = 0; dd < L; ++dd)
#pragma unroll
        for (int d = 0; d < L; ++d)
            s[d] = fmaf(a.k[d > dd ? d - dd : dd - d], u[dd], s[d]);
}

// ---------------------------------------------------------------------------
// Forward iteration, pull form: thread (p, k) computes the message that p
// receives in slot k, from r = p + off(k), out of state t - 1.  In the last
// iteration the four lanes of p add their messages to D_p and write the
// beliefs instead of a state.
template <int L, bool BELIEF>
__global__ void __launch_bounds__(kSpThreads, L <= 48 ? 4 : 3) k_sp_fwd(const __grid_constant__ SpArgs a)
{
    pdl_begin();
    const int gid = blockIdx.x * kSpThreads + threadIdx.x;
    const int p = gid >> 2, k = gid & 3;
    const bool valid = p < a.npix;
    const int r = valid ? neighbour(p, k, a.w, a.h) : -1;
    float m[L];
    if (r >= 0) {
        gather_h<L>(a, r, k ^ 1, m);   // r's slot k^1 holds what p sent it
        shift_to_min<L>(m);
#pragma unroll
        for (int d = 0; d < L; ++d)
            m[d] = exp2f(m[d] * a.nc);   // u
        float s[L];
        matvec_k<L>(a, m, s);
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
            float *o = a.mout + (size_t)k * a.npix * L + (size_t)p * L;
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
template <int L>
__global__ void __launch_bounds__(kSpThreads, L <= 48 ? 4 : 2) k_sp_adj(const __grid_constant__ SpArgs a)
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
        gather_h<L>(a, p, q, e);
        shift_to_min<L>(e);
#pragma unroll
        for (int d = 0; d < L; ++d)
            e[d] = exp2f(e[d] * a.nc);   // u
        float s[L];
        matvec_k<L>(a, e, s);             // S = K u
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
        // |d - d'| = delta of r(d) u(d')
#pragma unroll
        for (int del = 0; del < L; ++del) {
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
        // dL/dh(d') = u(d') (K r)(d'), and sum_d' log2 u(d') dL/dh(d'), where
        // h - a = -tau ln2 log2 u (u = 0 contributes nothing)
        float s_lu = 0.f;
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
    int nck, nseg, nblocks;
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
    lay.total = (size_t)(lay.nck + lay.nseg + 2) * lay.state_bytes + lay.partial_bytes;
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
    a.nc = (float)(-1.0 / (tau * std::log(2.0)));
    a.tau_ln2 = (float)(tau * std::log(2.0));
    a.lambda = p->lambda;
    a.trunc = p->trunc;
    a.tau = p->tau;
}

template <int L>
int launch_fwd(const SpArgs &a, bool belief, int nblocks, cudaStream_t st)
{
    const int slot = prof_begin(kProfSmoothFwd, st);
    cudaError_t err = belief ? launch_pdl(k_sp_fwd<L, true>, dim3(nblocks), dim3(kSpThreads), st, a)
                             : launch_pdl(k_sp_fwd<L, false>, dim3(nblocks), dim3(kSpThreads), st, a);
    prof_end(slot, st);
    note_launch();
    return err == cudaSuccess ? VS_OK : VS_ECUDA;
}

template <int L>
int launch_adj(const SpArgs &a, int nblocks, cudaStream_t st)
{
    const int slot = prof_begin(kProfSmoothAdj, st);
    const cudaError_t err = launch_pdl(k_sp_adj<L>, dim3(nblocks), dim3(kSpThreads), st, a);
    prof_end(slot, st);
    note_launch();
    return err == cudaSuccess ? VS_OK : VS_ECUDA;
}

int fwd_any(int L, const SpArgs &a, bool belief, int nblocks, cudaStream_t st)
{
    switch (L) {
    case 16: return launch_fwd<16>(a, belief, nblocks, st);
    case 32: return launch_fwd<32>(a, belief, nblocks, st);
    case 48: return launch_fwd<48>(a, belief, nblocks, st);
    default: return launch_fwd<64>(a, belief, nblocks, st);
    }
}

int adj_any(int L, const SpArgs &a, int nblocks, cudaStream_t st)
{
    switch (L) {
    case 16: return launch_adj<16>(a, nblocks, st);
    case 32: return launch_adj<32>(a, nblocks, st);
    case 48: return launch_adj<48>(a, nblocks, st);
    default: return launch_adj<64>(a, nblocks, st);
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

extern "C" int vs_sp_forward(const float *cost, int w, int h, const vs_sp_params *p, float *beliefs,
                             void *workspace, size_t ws_bytes, void *stream)
{
    if (!sp_valid(w, h, p) || cost == nullptr || beliefs == nullptr)
        return VS_EINVAL;
    if (!aligned(cost, 16) || !aligned(beliefs, 16))
        return VS_EALIGN;
    const SpLayout lay = sp_layout(w, h, p);
    if (int rc = sp_check_ws(workspace, ws_bytes, lay))
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    SpStates S{static_cast<char *>(workspace), lay};
    SpArgs a = {};
    fill_tables(a, p);
    a.cost = cost;
    a.w = w, a.h = h, a.npix = w * h;
    a.beliefs = beliefs;
    const int K = p->iters, c = p->ckpt_every;
    const float *prev = nullptr;
    for (int t = 1; t <= K; ++t) {
        a.min_ = prev;
        if (t == K) {
            a.mout = nullptr;
            if (int rc = fwd_any(p->labels, a, true, lay.nblocks, st))
                return rc;
        } else {
            float *out = (t % c == 0) ? S.ckpt(t / c - 1) : S.adj(t & 1);
            a.mout = out;
            if (int rc = fwd_any(p->labels, a, false, lay.nblocks, st))
                return rc;
            prev = out;
        }
    }
    return launch_status();
}

extern "C" int vs_sp_backward(const float *cost, int w, int h, const vs_sp_params *p, const float *grad_beliefs,
                              float *grad_cost, float *grad_params, void *workspace, size_t ws_bytes, void *stream)
{
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
    a.w = w, a.h = h, a.npix = w * h;
    a.gcost = grad_cost;
    a.gbel = grad_beliefs;
    a.partial = S.partial();
    const int K = p->iters, c = p->ckpt_every, L = p->labels;

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
            if (int rc = fwd_any(L, f, false, lay.nblocks, st))
                return rc;
            prev = f.mout;
        }
        for (int t = top; t > s0; --t) {
            a.min_ = (t - 1 == s0) ? base : S.seg(t - 1 - s0 - 1);
            a.gin = gin;
            a.gout = t > 1 ? S.adj(x) : nullptr;
            a.from_belief = from_belief;
            a.first = first;
            if (int rc = adj_any(L, a, lay.nblocks, st))
                return rc;
            gin = a.gout;
            from_belief = 0;
            first = 0;
            x ^= 1;
        }
    }
    const cudaError_t err = launch_pdl(k_sp_reduce, dim3(1), dim3(256), st, (const double *)S.partial(),
                                       lay.nblocks, grad_params);
    note_launch();
    if (err != cudaSuccess)
        return VS_ECUDA;
    return launch_status();
}
