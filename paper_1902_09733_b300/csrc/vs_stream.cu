// Streaming drivers: many pairs (or a flight's frame sequence) from host
// memory, with host->device copies, compute and device->host copies of
// consecutive pairs overlapped on three CUDA streams.
//
// All device memory comes from the caller's workspace; the pipeline itself
// only creates streams and events (host objects).
//
// Pair mode: every submit carries both frames of an independent pair.
// Flight mode: every submit carries one new frame; frame f is remapped once
// into a ring of k + 1 rectified frames, and once f >= k the pair
// (left = frame f - k, right = frame f) is matched, upsampled and
// reprojected in the left frame's camera (the camera moves along +x, so the
// later frame is the right view; Section 3.2 forms pairs from frames a fixed
// number apart).
#include "vs_common.cuh"

#include <algorithm>
#include <new>
#include <vector>

namespace vs {
namespace {

constexpr int kModePairs = 0;
constexpr int kModeFlight = 1;

struct Slot {
    uint8_t *dev_in = nullptr;    // one or two frames of host input
    float *dev_xyz = nullptr;     // this slot's point cloud
    cudaEvent_t in_done = nullptr, comp_done = nullptr, t_start = nullptr, t_end = nullptr;
    bool busy = false;
    bool has_output = false;
};

struct RingFrame {
    uint8_t *rect = nullptr;      // rectified full-res RGB
    uint8_t *low_rgb = nullptr;   // downsampled RGB
    uint8_t *low_gray = nullptr;  // downsampled grey
};

struct Geometry {
    int W, H, w, h;
    size_t frame, low;
    size_t slot_in, slot_xyz, ring_frame, labels, bp;
};

bool geometry(const vs_pair_config *cfg, int mode, int depth, int k, Geometry *g)
{
    if (!cfg || cfg->W <= 0 || cfg->H <= 0 || depth < 1 || depth > 16)
        return false;
    if (mode != kModePairs && mode != kModeFlight)
        return false;
    if (mode == kModeFlight && (k < 1 || k > 64))
        return false;
    const int s = cfg->jbu.scale;
    if (s < 1 || s > 16)
        return false;
    g->W = cfg->W;
    g->H = cfg->H;
    g->w = (cfg->W + s - 1) / s;
    g->h = (cfg->H + s - 1) / s;
    g->frame = (size_t)cfg->W * cfg->H * 3;
    g->low = (size_t)g->w * g->h;
    g->slot_in = align_up((mode == kModePairs ? 2 : 1) * g->frame, 256);
    g->slot_xyz = align_up((size_t)cfg->W * cfg->H * 3 * sizeof(float), 256);
    g->ring_frame = align_up(g->frame, 256) + align_up(3 * g->low, 256) + align_up(g->low, 256);
    g->labels = align_up(g->low, 256);
    g->bp = vs_bp_workspace_size(g->w, g->h, &cfg->bp);
    return g->bp != 0;
}

size_t total_bytes(const vs_pair_config *cfg, int mode, int depth, int k, const Geometry &g)
{
    size_t t = (size_t)depth * (g.slot_in + g.slot_xyz);
    if (mode == kModePairs)
        t += align_up(vs_pair_workspace_size(cfg), 256);
    else
        t += (size_t)(k + 1) * g.ring_frame + g.labels + align_up(g.bp, 256);
    return t;
}

}  // namespace
}  // namespace vs

struct vs_pipeline {
    vs_pair_config cfg;
    int mode = 0, depth = 0, k = 0;
    vs::Geometry g;
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    std::vector<vs::Slot> slots;
    std::vector<vs::RingFrame> ring;
    uint8_t *pair_ws = nullptr;   // pair mode: vs_pair_run workspace
    size_t pair_ws_bytes = 0;
    uint8_t *labels = nullptr, *bp_ws = nullptr;   // flight mode
    size_t bp_bytes = 0;
    long long submitted = 0;      // pairs (pair mode) or frames (flight mode)
    long long next_slot = 0;
    std::vector<float> latency_ms;
    int error = VS_OK;
};

namespace vs {
namespace {

void destroy_objects(vs_pipeline *p)
{
    for (auto &s : p->slots) {
        for (cudaEvent_t e : {s.in_done, s.comp_done, s.t_start, s.t_end})
            if (e)
                cudaEventDestroy(e);
    }
    for (cudaStream_t s : {p->s_in, p->s_comp, p->s_out})
        if (s)
            cudaStreamDestroy(s);
}

// Waits for the slot's previous pair (if any) and records its latency.
int retire(vs_pipeline *p, Slot &s)
{
    if (!s.busy)
        return VS_OK;
    if (cudaEventSynchronize(s.t_end) != cudaSuccess)
        return VS_ECUDA;
    if (s.has_output) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, s.t_start, s.t_end) == cudaSuccess)
            p->latency_ms.push_back(ms);
    }
    s.busy = false;
    s.has_output = false;
    return VS_OK;
}

// Enqueue the device->host copy of a slot's cloud after its compute.
int finish_slot(vs_pipeline *p, Slot &s, float *xyz_host)
{
    if (cudaEventRecord(s.comp_done, p->s_comp) != cudaSuccess ||
        cudaStreamWaitEvent(p->s_out, s.comp_done, 0) != cudaSuccess)
        return VS_ECUDA;
    if (xyz_host && cudaMemcpyAsync(xyz_host, s.dev_xyz, (size_t)p->g.W * p->g.H * 3 * sizeof(float),
                                    cudaMemcpyDeviceToHost, p->s_out) != cudaSuccess)
        return VS_ECUDA;
    if (cudaEventRecord(s.t_end, p->s_out) != cudaSuccess)
        return VS_ECUDA;
    s.busy = true;
    return VS_OK;
}

}  // namespace
}  // namespace vs

extern "C" size_t vs_pipeline_workspace_size(const vs_pair_config *cfg, int mode, int depth, int k)
{
    vs::Geometry g;
    if (!vs::geometry(cfg, mode, depth, k, &g))
        return 0;
    return vs::total_bytes(cfg, mode, depth, k, g);
}

extern "C" int vs_pipeline_create(const vs_pair_config *cfg, int mode, int depth, int k, void *workspace,
                                  size_t ws_bytes, vs_pipeline **out)
{
    using namespace vs;
    if (!out)
        return VS_EINVAL;
    *out = nullptr;
    Geometry g;
    if (!geometry(cfg, mode, depth, k, &g))
        return VS_EINVAL;
    if (!workspace || !aligned(workspace, 256) || ws_bytes < total_bytes(cfg, mode, depth, k, g))
        return VS_EWORKSPACE;
    vs_pipeline *p = new (std::nothrow) vs_pipeline;
    if (!p)
        return VS_EINVAL;
    p->cfg = *cfg;
    p->mode = mode;
    p->depth = depth;
    p->k = k;
    p->g = g;
    uint8_t *ws = reinterpret_cast<uint8_t *>(workspace);
    size_t off = 0;
    p->slots.resize(depth);
    for (auto &s : p->slots) {
        s.dev_in = ws + off;
        off += g.slot_in;
        s.dev_xyz = reinterpret_cast<float *>(ws + off);
        off += g.slot_xyz;
    }
    if (mode == kModePairs) {
        p->pair_ws = ws + off;
        p->pair_ws_bytes = vs_pair_workspace_size(cfg);
    } else {
        p->ring.resize(k + 1);
        for (auto &r : p->ring) {
            r.rect = ws + off;
            r.low_rgb = ws + off + align_up(g.frame, 256);
            r.low_gray = r.low_rgb + align_up(3 * g.low, 256);
            off += g.ring_frame;
        }
        p->labels = ws + off;
        off += g.labels;
        p->bp_ws = ws + off;
        p->bp_bytes = g.bp;
    }
    bool ok = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking) == cudaSuccess;
    for (auto &s : p->slots) {
        ok = ok && cudaEventCreateWithFlags(&s.in_done, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&s.comp_done, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreate(&s.t_start) == cudaSuccess && cudaEventCreate(&s.t_end) == cudaSuccess;
    }
    if (!ok) {
        destroy_objects(p);
        delete p;
        return VS_ECUDA;
    }
    *out = p;
    return VS_OK;
}

extern "C" int vs_pipeline_submit_pair(vs_pipeline *p, const uint8_t *left_host, const uint8_t *right_host,
                                       float *xyz_host)
{
    using namespace vs;
    if (!p || p->mode != kModePairs || !left_host || !right_host)
        return VS_EINVAL;
    if (p->error != VS_OK)
        return p->error;
    Slot &s = p->slots[p->next_slot % p->depth];
    int rc = retire(p, s);
    if (rc != VS_OK)
        return p->error = rc;
    const size_t frame = p->g.frame;
    if (cudaEventRecord(s.t_start, p->s_in) != cudaSuccess ||
        cudaMemcpyAsync(s.dev_in, left_host, frame, cudaMemcpyHostToDevice, p->s_in) != cudaSuccess ||
        cudaMemcpyAsync(s.dev_in + frame, right_host, frame, cudaMemcpyHostToDevice, p->s_in) != cudaSuccess ||
        cudaEventRecord(s.in_done, p->s_in) != cudaSuccess ||
        cudaStreamWaitEvent(p->s_comp, s.in_done, 0) != cudaSuccess)
        return p->error = VS_ECUDA;
    rc = vs_pair_run(&p->cfg, s.dev_in, s.dev_in + frame, nullptr, s.dev_xyz, p->pair_ws, p->pair_ws_bytes,
                     p->s_comp);
    if (rc != VS_OK)
        return p->error = rc;
    s.has_output = true;
    rc = finish_slot(p, s, xyz_host);
    if (rc != VS_OK)
        return p->error = rc;
    ++p->next_slot;
    ++p->submitted;
    return VS_OK;
}

extern "C" int vs_pipeline_submit_frame(vs_pipeline *p, const uint8_t *frame_host, float *xyz_host)
{
    using namespace vs;
    if (!p || p->mode != kModeFlight || !frame_host)
        return VS_EINVAL;
    if (p->error != VS_OK)
        return p->error;
    Slot &s = p->slots[p->next_slot % p->depth];
    int rc = retire(p, s);
    if (rc != VS_OK)
        return p->error = rc;
    const long long f = p->submitted;
    const RingFrame &cur = p->ring[f % (p->k + 1)];
    const Geometry &g = p->g;
    if (cudaEventRecord(s.t_start, p->s_in) != cudaSuccess ||
        cudaMemcpyAsync(s.dev_in, frame_host, g.frame, cudaMemcpyHostToDevice, p->s_in) != cudaSuccess ||
        cudaEventRecord(s.in_done, p->s_in) != cudaSuccess ||
        cudaStreamWaitEvent(p->s_comp, s.in_done, 0) != cudaSuccess)
        return p->error = VS_ECUDA;
    const int s_scale = p->cfg.jbu.scale;
    rc = vs_rectify_remap(s.dev_in, g.W, g.H, 3 * g.W, &p->cfg.cam, nullptr, cur.rect, 3 * g.W, s_scale, cur.low_rgb,
                          3 * g.w, cur.low_gray, g.w, p->s_comp);
    if (rc != VS_OK)
        return p->error = rc;
    if (f >= p->k) {
        const RingFrame &left = p->ring[(f - p->k) % (p->k + 1)];
        rc = vs_bp_stereo(left.low_gray, cur.low_gray, g.w, g.h, g.w, &p->cfg.bp, p->labels, g.w, p->bp_ws,
                          p->bp_bytes, p->s_comp);
        if (rc == VS_OK)
            rc = vs_guided_upsample_reproject(p->labels, g.w, g.h, g.w, left.low_rgb, 3 * g.w, left.rect, g.W, g.H,
                                              3 * g.W, &p->cfg.jbu, &p->cfg.cam, p->cfg.baseline, nullptr,
                                              s.dev_xyz, p->s_comp);
        if (rc != VS_OK)
            return p->error = rc;
        s.has_output = true;
    }
    rc = finish_slot(p, s, s.has_output ? xyz_host : nullptr);
    if (rc != VS_OK)
        return p->error = rc;
    ++p->next_slot;
    ++p->submitted;
    return VS_OK;
}

extern "C" int vs_pipeline_flush(vs_pipeline *p)
{
    using namespace vs;
    if (!p)
        return VS_EINVAL;
    for (long long i = 0; i < p->depth; ++i) {
        Slot &s = p->slots[(p->next_slot + i) % p->depth];
        const int rc = retire(p, s);
        if (rc != VS_OK)
            return p->error = rc;
    }
    return p->error;
}

extern "C" int vs_pipeline_latencies(vs_pipeline *p, float *ms, int max)
{
    if (!p || (max > 0 && !ms))
        return VS_EINVAL;
    const int n = (int)std::min<size_t>(p->latency_ms.size(), (size_t)std::max(max, 0));
    for (int i = 0; i < n; ++i)
        ms[i] = p->latency_ms[i];
    p->latency_ms.erase(p->latency_ms.begin(), p->latency_ms.begin() + n);
    return n;
}

extern "C" void vs_pipeline_destroy(vs_pipeline *p)
{
    if (!p)
        return;
    vs_pipeline_flush(p);
    vs::destroy_objects(p);
    delete p;
}
