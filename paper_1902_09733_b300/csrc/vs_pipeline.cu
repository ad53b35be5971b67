// Whole-pair drivers (Section 2.1 -> Eq. 1 -> Eq. 2 -> Eq. 3), status names
// and launch bookkeeping.
#include "vs_common.cuh"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

namespace vs {
namespace {

std::atomic<uint64_t> g_launches{0};

// event ring for vs_profile_*: slots are handed out in order; a slot stays
// pending until vs_profile_collect reads it
struct ProfState {
    std::mutex mu;
    std::vector<cudaEvent_t> start, stop;
    std::vector<int> tag;
    std::vector<int> pending;
    int next = 0;
    bool on = false;
} g_prof;

struct PairLayout {
    int w, h;
    size_t rect_l, rect_r, low_rgb, gray_l, gray_r, labels, bp;
    size_t bp_bytes, total;
};

bool pair_layout(const vs_pair_config *cfg, PairLayout *out)
{
    if (!cfg || cfg->W <= 0 || cfg->H <= 0)
        return false;
    const int s = cfg->jbu.scale;
    if (s < 1 || s > 16)
        return false;
    PairLayout lay;
    lay.w = (cfg->W + s - 1) / s;
    lay.h = (cfg->H + s - 1) / s;
    const size_t full = (size_t)cfg->W * cfg->H * 3;
    const size_t low = (size_t)lay.w * lay.h;
    size_t off = 0;
    lay.rect_l = off;
    off = align_up(off + full, 256);
    lay.rect_r = off;
    off = align_up(off + full, 256);
    lay.low_rgb = off;
    off = align_up(off + 3 * low, 256);
    lay.gray_l = off;
    off = align_up(off + low, 256);
    lay.gray_r = off;
    off = align_up(off + low, 256);
    lay.labels = off;
    off = align_up(off + low, 256);
    lay.bp = off;
    lay.bp_bytes = vs_bp_workspace_size(lay.w, lay.h, &cfg->bp);
    if (lay.bp_bytes == 0)
        return false;
    off = align_up(off + lay.bp_bytes, 256);
    lay.total = off;
    *out = lay;
    return true;
}

}  // namespace

void note_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

cudaStream_t *library_streams()
{
    static std::mutex mu;
    static std::vector<std::vector<cudaStream_t>> per_dev;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)per_dev.size() <= dev)
        per_dev.resize(dev + 1);
    std::vector<cudaStream_t> &v = per_dev[dev];
    while ((int)v.size() < kLibStreams) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return nullptr;
        v.push_back(s);
    }
    return v.data();
}

}  // namespace

int fork_join(cudaStream_t st, int n, const std::function<int(int, cudaStream_t)> &body)
{
    cudaStream_t *side = library_streams();
    if (!side || n < 1 || n > kLibStreams)
        return VS_ECUDA;
    cudaEvent_t fork;
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess)
        return VS_ECUDA;
    int rc = cudaEventRecord(fork, st) == cudaSuccess ? VS_OK : VS_ECUDA;
    for (int k = 0; k < n && rc == VS_OK; ++k) {
        if (cudaStreamWaitEvent(side[k], fork, 0) != cudaSuccess) {
            rc = VS_ECUDA;
            break;
        }
        rc = body(k, side[k]);
        // join even after a failed body, so that `st` (or its capture) stays whole
        cudaEvent_t join;
        if (cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
            rc = VS_ECUDA;
            break;
        }
        if (cudaEventRecord(join, side[k]) != cudaSuccess || cudaStreamWaitEvent(st, join, 0) != cudaSuccess)
            rc = VS_ECUDA;
        cudaEventDestroy(join);
    }
    cudaEventDestroy(fork);
    return rc;
}

int launch_status()
{
    return cudaGetLastError() == cudaSuccess ? VS_OK : VS_ECUDA;
}

// Inside stream capture a plain cudaEventRecord only orders the capture; the
// external flag makes it an event-record node of the graph, so the pair
// times every replay of the captured kernel.
static void prof_record(cudaEvent_t ev, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, st);
}

int prof_begin(int tag, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (!g_prof.on || g_prof.start.empty())
        return -1;
    const int slot = g_prof.next;
    g_prof.next = (g_prof.next + 1) % (int)g_prof.start.size();
    g_prof.tag[slot] = tag;
    g_prof.pending.push_back(slot);
    prof_record(g_prof.start[slot], st);
    return slot;
}

void prof_end(int slot, cudaStream_t st)
{
    if (slot < 0)
        return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    prof_record(g_prof.stop[slot], st);
}

}  // namespace vs

extern "C" int vs_profile_enable(int capacity)
{
    using namespace vs;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (size_t i = 0; i < g_prof.start.size(); ++i) {
        cudaEventDestroy(g_prof.start[i]);
        cudaEventDestroy(g_prof.stop[i]);
    }
    g_prof.start.clear();
    g_prof.stop.clear();
    g_prof.tag.clear();
    g_prof.pending.clear();
    g_prof.next = 0;
    g_prof.on = false;
    if (capacity < 0 || capacity > (1 << 20))
        return VS_EINVAL;
    for (int i = 0; i < capacity; ++i) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess)
            return VS_ECUDA;
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return VS_ECUDA;
        }
        g_prof.start.push_back(a);
        g_prof.stop.push_back(b);
        g_prof.tag.push_back(-1);
    }
    g_prof.on = capacity > 0;
    return VS_OK;
}

extern "C" int vs_profile_collect(int *tags, float *ms, int max)
{
    using namespace vs;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    int n = 0;
    for (int slot : g_prof.pending) {
        if (n >= max)
            break;
        // a pair recorded only during stream capture has no time until its
        // graph has run; such pairs are skipped
        float t = 0.0f;
        if (cudaEventSynchronize(g_prof.stop[slot]) != cudaSuccess ||
            cudaEventElapsedTime(&t, g_prof.start[slot], g_prof.stop[slot]) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        tags[n] = g_prof.tag[slot];
        ms[n] = t;
        ++n;
    }
    g_prof.pending.clear();
    return n;
}

extern "C" const char *vs_status_string(int status)
{
    switch (status) {
    case VS_OK: return "ok";
    case VS_EINVAL: return "invalid argument (size, count or parameter out of range)";
    case VS_EALIGN: return "pointer or pitch breaks an alignment rule";
    case VS_EWORKSPACE: return "workspace missing, misaligned or too small";
    case VS_ECUDA: return "CUDA runtime error";
    case VS_ETIMEOUT: return "bounded wait inside a kernel timed out";
    default: return "unknown status";
    }
}

extern "C" uint64_t vs_kernel_launches(void) { return vs::g_launches.load(std::memory_order_relaxed); }

extern "C" size_t vs_pair_workspace_size(const vs_pair_config *cfg)
{
    vs::PairLayout lay;
    return vs::pair_layout(cfg, &lay) ? lay.total : 0;
}

extern "C" int vs_pair_run(const vs_pair_config *cfg, const uint8_t *left_src, const uint8_t *right_src,
                           float *disp, float *xyz, void *workspace, size_t ws_bytes, void *stream)
{
    vs::NvtxRange nvtx_range("vs_pair_run");
    using namespace vs;
    PairLayout lay;
    if (!pair_layout(cfg, &lay) || !left_src || !right_src || !xyz)
        return VS_EINVAL;
    if (!workspace || !aligned(workspace, 256) || ws_bytes < lay.total)
        return VS_EWORKSPACE;
    uint8_t *ws = reinterpret_cast<uint8_t *>(workspace);
    const int W = cfg->W, H = cfg->H, s = cfg->jbu.scale;
    // the right frame only feeds the matcher: its full-res copy is not needed,
    // and with the block kernel it is sampled in the left frame's launch
    int rc = remap_pair(left_src, right_src, W, H, 3 * W, &cfg->cam, s, ws + lay.rect_l, 3 * W, ws + lay.low_rgb,
                        3 * lay.w, ws + lay.gray_l, ws + lay.gray_r, lay.w, (cudaStream_t)stream);
    if (rc != VS_OK && rc != VS_EINVAL)
        return rc;
    if (rc == VS_EINVAL) {   // not for the block kernel: one frame at a time
        rc = vs_rectify_remap(left_src, W, H, 3 * W, &cfg->cam, nullptr, ws + lay.rect_l, 3 * W, s, ws + lay.low_rgb,
                              3 * lay.w, ws + lay.gray_l, lay.w, stream);
        if (rc != VS_OK)
            return rc;
        rc = vs_rectify_remap(right_src, W, H, 3 * W, &cfg->cam, nullptr, nullptr, 0, s, nullptr, 0,
                              ws + lay.gray_r, lay.w, stream);
        if (rc != VS_OK)
            return rc;
    }
    rc = vs_bp_stereo(ws + lay.gray_l, ws + lay.gray_r, lay.w, lay.h, lay.w, &cfg->bp, ws + lay.labels, lay.w,
                      ws + lay.bp, lay.bp_bytes, stream);
    if (rc != VS_OK)
        return rc;
    return vs_guided_upsample_reproject(ws + lay.labels, lay.w, lay.h, lay.w, ws + lay.low_rgb, 3 * lay.w,
                                        ws + lay.rect_l, W, H, 3 * W, &cfg->jbu, &cfg->cam, cfg->baseline, disp,
                                        xyz, stream);
}

namespace vs {
namespace {

bool pair_batch_layouts(const vs_pair_job *jobs, int n, std::vector<PairLayout> &lays, std::vector<size_t> &offs,
                        size_t &total)
{
    if (!jobs || n < 1 || n > 4096)
        return false;
    lays.resize(n);
    offs.resize(n);
    total = 0;
    for (int i = 0; i < n; ++i) {
        if (!pair_layout(&jobs[i].cfg, &lays[i]))
            return false;
        offs[i] = total;
        total = align_up(total + lays[i].total, 256);
    }
    return true;
}

// Relative cost of a pair for balancing the streams: the BP sweeps (low-res
// pixels x padded labels x iterations x 4/3 for the coarser levels) plus the
// full-resolution remap and upsampling, weighted as measured on B300 (the
// 2.7K pair at s = 4: about 240 us of BP, 60 us of remap and JBU).
double pair_work(const vs_pair_job &j, const PairLayout &lay)
{
    const vs_bp_params &p = j.cfg.bp;
    const int Lp = p.labels <= 64 ? (p.labels + 15) / 16 * 16 : (p.labels <= 96 ? 96 : 128);
    return (double)lay.w * lay.h * Lp * p.iters * (4.0 / 3.0) + 13.0 * (double)j.cfg.W * j.cfg.H;
}

}  // namespace
}  // namespace vs

extern "C" size_t vs_pair_batch_workspace_size(const vs_pair_job *jobs, int n)
{
    std::vector<vs::PairLayout> lays;
    std::vector<size_t> offs;
    size_t total = 0;
    return vs::pair_batch_layouts(jobs, n, lays, offs, total) ? total : 0;
}

extern "C" int vs_pair_run_batch(const vs_pair_job *jobs, int n, void *workspace, size_t ws_bytes, void *stream)
{
    vs::NvtxRange nvtx_range("vs_pair_run_batch");
    using namespace vs;
    std::vector<PairLayout> lays;
    std::vector<size_t> offs;
    size_t total = 0;
    if (!pair_batch_layouts(jobs, n, lays, offs, total))
        return VS_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!jobs[i].left || !jobs[i].right || !jobs[i].xyz)
            return VS_EINVAL;
    if (!workspace || !aligned(workspace, 256) || ws_bytes < total)
        return VS_EWORKSPACE;
    // largest first, each to the least loaded library stream
    const int S = std::min(n, kLibStreams);
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i)
        order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return pair_work(jobs[a], lays[a]) > pair_work(jobs[b], lays[b]); });
    std::vector<std::vector<int>> queue(S);
    std::vector<double> load(S, 0.0);
    for (int i : order) {
        int k = 0;
        for (int j = 1; j < S; ++j)
            if (load[j] < load[k])
                k = j;
        queue[k].push_back(i);
        load[k] += pair_work(jobs[i], lays[i]);
    }
    uint8_t *base = reinterpret_cast<uint8_t *>(workspace);
    return fork_join((cudaStream_t)stream, S, [&](int k, cudaStream_t side) {
        for (int i : queue[k]) {
            const vs_pair_job &j = jobs[i];
            const int rc = vs_pair_run(&j.cfg, j.left, j.right, j.disp, j.xyz, base + offs[i], lays[i].total, side);
            if (rc != VS_OK)
                return rc;
        }
        return VS_OK;
    });
}

extern "C" int vs_pair_run_host(const vs_pair_config *cfg, const uint8_t *left_host, const uint8_t *right_host,
                                float *disp_host, float *xyz_host, uint8_t *dev_in, float *dev_disp,
                                float *dev_xyz, void *workspace, size_t ws_bytes, void *stream)
{
    vs::NvtxRange nvtx_range("vs_pair_run_host");
    using namespace vs;
    PairLayout lay;
    if (!pair_layout(cfg, &lay) || !left_host || !right_host || !xyz_host || !dev_in || !dev_xyz)
        return VS_EINVAL;
    if (disp_host && !dev_disp)
        return VS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t frame = (size_t)cfg->W * cfg->H * 3;
    const size_t npx = (size_t)cfg->W * cfg->H;
    if (cudaMemcpyAsync(dev_in, left_host, frame, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dev_in + frame, right_host, frame, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return VS_ECUDA;
    int rc = vs_pair_run(cfg, dev_in, dev_in + frame, disp_host ? dev_disp : nullptr, dev_xyz, workspace,
                         ws_bytes, stream);
    if (rc != VS_OK)
        return rc;
    if (cudaMemcpyAsync(xyz_host, dev_xyz, npx * 3 * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return VS_ECUDA;
    if (disp_host &&
        cudaMemcpyAsync(disp_host, dev_disp, npx * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return VS_ECUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? VS_OK : VS_ECUDA;
}
