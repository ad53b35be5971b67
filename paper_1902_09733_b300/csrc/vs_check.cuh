// Bounds checking of the checked build (compiled with -DVS_CHECKED into
// libvstereo_checked.so, for tests only; the product library is built
// without it and these checks compile to nothing there).
//
// Before its kernels, an entry point registers the address ranges of its
// call's buffers (images, labels, workspace, outputs) in a small table in
// device memory, ordered on the call's stream.  Every instrumented global
// access of the min-sum kernels tests its address against that table; the
// first access outside every range records its site and address in a device
// word and is skipped (a load returns zeros, a store does nothing), and the
// kernel carries on -- no trap, no device assert, no access outside the
// caller's buffers.  Each translation unit that includes this header has its
// own table (static device variables), set by its own entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <initializer_list>
#include <utility>
#include <vector>

namespace vs {

#ifdef VS_CHECKED

constexpr int kCheckRanges = 64;

struct CheckRange {
    unsigned long long lo, hi;
};

struct CheckTable {
    int n;
    CheckRange r[kCheckRanges];
};

static __device__ CheckTable g_check_table;
static __device__ unsigned long long g_check_first[2];   // site + 1 and address of the first violation

// True if [p, p + n) lies inside a registered range; otherwise records the
// first violation and returns false (the caller skips the access).
__device__ __forceinline__ bool chk(const void *p, unsigned n, int site)
{
    const unsigned long long a = reinterpret_cast<unsigned long long>(p);
    const int cnt = g_check_table.n;
    for (int i = 0; i < cnt; ++i)
        if (a >= g_check_table.r[i].lo && a + n <= g_check_table.r[i].hi)
            return true;
    if (atomicCAS(&g_check_first[0], 0ull, (unsigned long long)(site + 1)) == 0ull)
        g_check_first[1] = a;
    return false;
}

// Host: this translation unit's ranges for the kernels enqueued next on
// `st` (more than kCheckRanges buffers: their hull).  Test aid: `shrink`
// bytes are taken off the end of the last range.
inline void check_ranges(cudaStream_t st, std::initializer_list<std::pair<const void *, size_t>> bufs,
                         size_t shrink = 0)
{
    static thread_local CheckTable t;   // the copy's source must outlive the enqueue
    t.n = 0;
    unsigned long long lo = ~0ull, hi = 0;
    for (const auto &b : bufs) {
        if (!b.first || b.second == 0)
            continue;
        const unsigned long long a = reinterpret_cast<unsigned long long>(b.first);
        lo = a < lo ? a : lo;
        hi = a + b.second > hi ? a + b.second : hi;
        if (t.n < kCheckRanges)
            t.r[t.n++] = CheckRange{a, a + b.second};
    }
    if ((int)bufs.size() > kCheckRanges) {
        t.n = 1;
        t.r[0] = CheckRange{lo, hi};
    }
    if (t.n > 0 && shrink > 0 && t.r[t.n - 1].hi - t.r[t.n - 1].lo > shrink)
        t.r[t.n - 1].hi -= shrink;
    cudaMemcpyToSymbolAsync(g_check_table, &t, sizeof(t), 0, cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);   // `t` is reused by the next call
}

// The same for a list built at run time.
inline void check_ranges_list(cudaStream_t st, const std::vector<std::pair<const void *, size_t>> &bufs)
{
    static thread_local CheckTable t;
    t.n = 0;
    unsigned long long lo = ~0ull, hi = 0;
    for (const auto &b : bufs) {
        if (!b.first || b.second == 0)
            continue;
        const unsigned long long a = reinterpret_cast<unsigned long long>(b.first);
        lo = a < lo ? a : lo;
        hi = a + b.second > hi ? a + b.second : hi;
        if (t.n < kCheckRanges)
            t.r[t.n++] = CheckRange{a, a + b.second};
    }
    if ((int)bufs.size() > kCheckRanges) {
        t.n = 1;
        t.r[0] = CheckRange{lo, hi};
    }
    cudaMemcpyToSymbolAsync(g_check_table, &t, sizeof(t), 0, cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
}

// Host: the first violation recorded in this translation unit since the
// last read (site + 1, 0 if none) and its address; clears it.
inline unsigned long long check_take(unsigned long long *addr)
{
    unsigned long long v[2] = {0, 0};
    cudaMemcpyFromSymbol(v, g_check_first, sizeof(v));
    const unsigned long long z[2] = {0, 0};
    cudaMemcpyToSymbol(g_check_first, z, sizeof(z));
    if (addr)
        *addr = v[1];
    return v[0];
}

#else

__device__ __forceinline__ constexpr bool chk(const void *, unsigned, int) { return true; }

inline void check_ranges(cudaStream_t, std::initializer_list<std::pair<const void *, size_t>>, size_t = 0) {}

#endif

// Sites of the instrumented accesses (reported as site + 1).
enum CheckSite {
    kSitePieceLoad = 0,
    kSitePieceStore = 1,
    kSiteImage = 2,
    kSiteCostWord = 3,
    kSiteLabel = 4,
    kSiteBulkCopy = 5,
    kSiteAsyncCopy = 6,
    kSiteStatus = 7,
    kSiteExport = 8,
    kSiteWideLoad = 9,
    kSiteWideStore = 10,
};

}  // namespace vs
