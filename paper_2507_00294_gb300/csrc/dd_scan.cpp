// Host runtime: scan construction (visit order and times), validation, error state
// and the per-device cache of the visit list.
//
// Scan strategies follow Sec. 1 of Javadi Rad et al. (raster, alternating,
// interleaved, random, subsampled); the visit order feeds the cumulative sum of
// Eq. 5, each visit starting when the previous dwell ends (Sec. 2).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "dd_internal.h"

namespace dd {

static thread_local std::string g_last_error;

dd_status fail(dd_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

dd_status fail_cuda(cudaError_t err, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")";
    return DD_ECUDA;
}

void clear_error() { g_last_error.clear(); }

bool fault_injected(const char *site) {
    const char *v = std::getenv("DD_FAULT");
    return v && std::strcmp(v, site) == 0;
}

static std::mutex g_scans_mu;
static std::unordered_set<dd_scan *> g_scans;

// Destroyed scans kept for their host storage (a few, of bounded size): the next scan of
// at most that many visits is built in vectors that keep their capacity, instead of pages
// the allocator handed back to the system and must fault in and zero again (about half the
// host time of building a 4,096-visit scan).
static std::mutex g_spare_mu;
static std::vector<dd_scan *> g_spare;
constexpr size_t kSpareScans = 4, kSpareBytes = size_t(16) << 20;

static size_t scan_bytes(const dd_scan *s) {
    return s->visit.capacity() * sizeof(int32_t) +
           (s->t_start.capacity() + s->tau.capacity() + s->X.capacity() + s->Y.capacity() + s->T.capacity() +
            s->TAU.capacity()) * sizeof(double);
}

dd_scan *reuse_scan() {
    std::lock_guard<std::mutex> lock(g_spare_mu);
    if (g_spare.empty()) return nullptr;
    dd_scan *s = g_spare.back();
    g_spare.pop_back();
    return s;
}

void recycle_scan(dd_scan *s) {
    if (scan_bytes(s) <= kSpareBytes) {
        std::lock_guard<std::mutex> lock(g_spare_mu);
        if (g_spare.size() < kSpareScans) {
            g_spare.push_back(s);
            return;
        }
    }
    delete s;
}

void register_scan(dd_scan *s) {
    std::lock_guard<std::mutex> lock(g_scans_mu);
    g_scans.insert(s);
}

bool unregister_scan(dd_scan *s) {
    std::lock_guard<std::mutex> lock(g_scans_mu);
    return g_scans.erase(s) == 1;
}

bool is_device_pointer(const void *p) {
    return memory_kind(p) == MemKind::Device;
}

MemKind memory_kind(const void *p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();   // unregistered host memory on old runtimes
        return MemKind::Pageable;
    }
    if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) return MemKind::Device;
    return attr.type == cudaMemoryTypeHost ? MemKind::Pinned : MemKind::Pageable;
}

bool host_sync_needed(cudaStream_t stream, std::initializer_list<MemKind> kinds) {
    bool any_host = false, all_pinned = true;
    for (MemKind k : kinds) {
        if (k == MemKind::Device) continue;
        any_host = true;
        all_pinned = all_pinned && k == MemKind::Pinned;
    }
    return any_host && (stream == nullptr || !all_pinned);
}

static cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t stream) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int device = 0;
    cudaError_t err = cudaGetDevice(&device);
    if (err != cudaSuccess) return err;
    if (device < 0 || device >= 64) return cudaMallocAsync(p, bytes, stream);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!pools[device]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = device;
            err = cudaMemPoolCreate(&pools[device], &props);
            if (err != cudaSuccess) { pools[device] = nullptr; return err; }
            uint64_t keep = uint64_t(4) << 30;
            err = cudaMemPoolSetAttribute(pools[device], cudaMemPoolAttrReleaseThreshold, &keep);
            if (err != cudaSuccess) return err;
        }
        pool = pools[device];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, stream);
}

// Released workspaces, kept per device with the stream that last used them and an event
// recorded there after that use: a block is taken again on the same stream at once (stream
// order) and on another stream once its event has completed.  Two calls in flight on two
// streams each keep their own block, where the stream-ordered pool's allocation measured up
// to 75 us of host time per call.  Sizes are rounded to 2^k or 3 * 2^(k-1) bytes (>= 1 MiB);
// at most 8 GiB per device is kept, the rest goes back to the pool.
struct WsFree {
    void *p;
    size_t cap;
    cudaStream_t last;
    cudaEvent_t ev;
};
static std::mutex g_ws_mu;
static std::vector<WsFree> g_ws_free[64];
static std::vector<cudaEvent_t> g_ws_events[64];
static std::unordered_map<void *, std::pair<int, size_t>> g_ws_live;     // block -> (device, bytes)
static size_t g_ws_kept[64];
constexpr size_t kWsKeep = size_t(8) << 30;

static size_t ws_class(size_t bytes) {
    size_t c = size_t(1) << 20;
    for (;;) {
        if (c >= bytes) return c;
        if (c + c / 2 >= bytes) return c + c / 2;
        c <<= 1;
    }
}

cudaError_t workspace_alloc(void **p, size_t bytes, cudaStream_t stream) {
    int device = 0;
    cudaError_t err = cudaGetDevice(&device);
    if (err != cudaSuccess) return err;
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    const size_t cap = ws_class(bytes);
    {
        std::lock_guard<std::mutex> lock(g_ws_mu);
        auto &fl = g_ws_free[device];
        for (size_t i = 0; i < fl.size(); ++i) {
            if (fl[i].cap != cap) continue;
            // another stream, or the per-thread default stream (one handle for a different
            // stream on each host thread): only once the block's last use has completed
            if (fl[i].last != stream || stream == cudaStreamPerThread) {
                const cudaError_t q = cudaEventQuery(fl[i].ev);
                if (q != cudaSuccess) {
                    cudaGetLastError();             // unfinished work is not an error
                    continue;
                }
            }
            *p = fl[i].p;
            g_ws_events[device].push_back(fl[i].ev);
            g_ws_kept[device] -= cap;
            fl.erase(fl.begin() + (std::ptrdiff_t)i);
            g_ws_live[*p] = {device, cap};
            return cudaSuccess;
        }
    }
    err = pool_alloc(p, cap, stream);
    if (err != cudaSuccess) return err;
    std::lock_guard<std::mutex> lock(g_ws_mu);
    g_ws_live[*p] = {device, cap};
    return cudaSuccess;
}

cudaError_t workspace_release(void *p, cudaStream_t stream) {
    if (!p) return cudaSuccess;
    int device = 0;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_ws_mu);
        auto it = g_ws_live.find(p);
        if (it != g_ws_live.end()) {
            device = it->second.first;
            cap = it->second.second;
            g_ws_live.erase(it);
            if (g_ws_kept[device] + cap > kWsKeep) {
                cap = 0;                                  // over the cap: back to the pool
            } else {
                g_ws_kept[device] += cap;
                if (!g_ws_events[device].empty()) {
                    ev = g_ws_events[device].back();
                    g_ws_events[device].pop_back();
                }
            }
        }
    }
    if (cap == 0) return cudaFreeAsync(p, stream);
    cudaError_t err = ev ? cudaSuccess : cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventRecord(ev, stream);
    std::lock_guard<std::mutex> lock(g_ws_mu);
    if (err != cudaSuccess) {
        cudaGetLastError();
        if (ev) g_ws_events[device].push_back(ev);
        g_ws_kept[device] -= cap;
        return cudaFreeAsync(p, stream);
    }
    g_ws_free[device].push_back({p, cap, stream, ev});
    return cudaSuccess;
}

static std::mutex g_pinned_mu;
static std::vector<void *> g_pinned_free[48];    // by size class: 2^k bytes

PinnedBlock pinned_take(size_t bytes) {
    int k = 12;                                    // at least 4 KiB
    while (k < 47 && (size_t(1) << k) < bytes) ++k;
    {
        std::lock_guard<std::mutex> lock(g_pinned_mu);
        if (!g_pinned_free[k].empty()) {
            void *p = g_pinned_free[k].back();
            g_pinned_free[k].pop_back();
            return {p, size_t(1) << k};
        }
    }
    void *p = nullptr;
    if (cudaHostAlloc(&p, size_t(1) << k, cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return {};
    }
    return {p, size_t(1) << k};
}

void pinned_give(PinnedBlock b) {
    if (!b.p) return;
    int k = 12;
    while (k < 47 && (size_t(1) << k) < b.cap) ++k;
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    g_pinned_free[k].push_back(b.p);
}

struct Deferred {
    cudaEvent_t ev;
    int device;
    void *obj;
    void (*del)(void *);
};
static std::mutex g_deferred_mu;
static std::deque<Deferred> g_deferred;
static std::vector<cudaEvent_t> g_free_events[64];   // events are per device

cudaError_t defer_release(cudaStream_t stream, void *obj, void (*del)(void *)) {
    std::vector<Deferred> done;
    int device = 0;
    cudaError_t err = cudaGetDevice(&device);
    if (err == cudaSuccess && (device < 0 || device >= 64)) err = cudaErrorInvalidDevice;
    if (err == cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_deferred_mu);
        // release what has completed (in order: the list is in enqueue order per stream)
        for (auto it = g_deferred.begin(); it != g_deferred.end();) {
            if (cudaEventQuery(it->ev) == cudaSuccess) {
                done.push_back(*it);
                it = g_deferred.erase(it);
            } else {
                ++it;
            }
        }
        cudaGetLastError();                         // a query of unfinished work is not an error
        if (g_deferred.size() > 256) {
            Deferred d = g_deferred.front();
            g_deferred.pop_front();
            cudaEventSynchronize(d.ev);
            done.push_back(d);
        }
        cudaEvent_t ev = nullptr;
        if (!g_free_events[device].empty()) {
            ev = g_free_events[device].back();
            g_free_events[device].pop_back();
        } else {
            err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        }
        if (err == cudaSuccess) err = cudaEventRecord(ev, stream);
        if (err == cudaSuccess) {
            g_deferred.push_back({ev, device, obj, del});
        } else {
            cudaGetLastError();
            if (ev) g_free_events[device].push_back(ev);
        }
        for (auto &d : done) g_free_events[d.device].push_back(d.ev);
    }
    for (auto &d : done) d.del(d.obj);
    if (err != cudaSuccess) {
        cudaDeviceSynchronize();
        del(obj);
    }
    return err;
}

// Device blocks of visit caches: a destroyed scan's block (once the work that read it is
// done) is kept per device and power-of-two size class for the next scan, up to 1 GiB per
// device, since a stream-ordered pool allocation of a fresh block took about 66 us of host
// time per scan.
static std::mutex g_vcache_mu;
static std::vector<void *> g_vcache_free[64][48];
static size_t g_vcache_kept[64];
constexpr size_t kVCacheKeep = size_t(1) << 30;

static int vcache_class(size_t bytes) {
    int k = 12;
    while (k < 47 && (size_t(1) << k) < bytes) ++k;
    return k;
}

static cudaError_t vcache_take(int device, size_t bytes, void **p, size_t *cap) {
    const int k = vcache_class(bytes);
    *cap = size_t(1) << k;
    {
        std::lock_guard<std::mutex> lock(g_vcache_mu);
        if (!g_vcache_free[device][k].empty()) {
            *p = g_vcache_free[device][k].back();
            g_vcache_free[device][k].pop_back();
            g_vcache_kept[device] -= *cap;
            return cudaSuccess;
        }
    }
    return cudaMalloc(p, *cap);
}

// the caller has waited for every use of the block (or for the whole device)
static void vcache_give(int device, void *p, size_t cap) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lock(g_vcache_mu);
        if (g_vcache_kept[device] + cap <= kVCacheKeep) {
            g_vcache_free[device][vcache_class(cap)].push_back(p);
            g_vcache_kept[device] += cap;
            return;
        }
    }
    cudaFree(p);
}

const double *device_sources(const dd_scan *scan, cudaStream_t stream, dd_status *st) {
    int device = 0;
    cudaError_t err = cudaGetDevice(&device);
    if (err != cudaSuccess) { *st = fail_cuda(err, "cudaGetDevice"); return nullptr; }
    std::lock_guard<std::mutex> lock(scan->mu);
    for (auto &c : scan->dev)
        if (c.device == device) {
            if (stream != c.home) {
                err = cudaStreamWaitEvent(stream, c.ready, 0);
                if (err != cudaSuccess) { *st = fail_cuda(err, "cudaStreamWaitEvent(scan visit cache)"); return nullptr; }
            }
            return c.src;
        }
    const size_t n = (size_t)scan->n;
    // 4n doubles, then n float4 of float-float coordinates (16-byte aligned: 32n bytes in),
    // written straight into a pinned staging block (a pageable vector when none is free)
    const size_t bytes = 6 * n * sizeof(double);
    void *d = nullptr;
    size_t cap = 0;
    err = device < 64 ? vcache_take(device, bytes, &d, &cap) : cudaErrorInvalidDevice;
    if (err != cudaSuccess) { *st = fail_cuda(err, "scan visit cache allocation"); cudaGetLastError(); return nullptr; }
    cudaEvent_t ready = nullptr;
    err = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    if (err != cudaSuccess) { vcache_give(device, d, cap); *st = fail_cuda(err, "cudaEventCreate"); return nullptr; }
    auto *stage = new CallStaging();
    std::vector<double> pageable;
    double *host = static_cast<double *>(stage->stage(bytes));
    if (!host) {
        pageable.resize(6 * n);
        host = pageable.data();
    }
    std::memcpy(host, scan->X.data(), n * sizeof(double));
    std::memcpy(host + n, scan->Y.data(), n * sizeof(double));
    std::memcpy(host + 2 * n, scan->T.data(), n * sizeof(double));
    std::memcpy(host + 3 * n, scan->TAU.data(), n * sizeof(double));
    float *ff = reinterpret_cast<float *>(host + 4 * n);
    for (size_t i = 0; i < n; ++i) {
        const float xh = (float)scan->X[i], yh = (float)scan->Y[i];
        ff[4 * i] = xh;
        ff[4 * i + 1] = (float)(scan->X[i] - (double)xh);
        ff[4 * i + 2] = yh;
        ff[4 * i + 3] = (float)(scan->Y[i] - (double)yh);
    }
    err = cudaMemcpyAsync(d, host, bytes, cudaMemcpyHostToDevice, stream);
    if (err == cudaSuccess && !pageable.empty()) err = cudaStreamSynchronize(stream);  // pageable source
    if (err == cudaSuccess) err = cudaEventRecord(ready, stream);
    if (err != cudaSuccess) {
        cudaStreamSynchronize(stream);
        delete stage;
        vcache_give(device, d, cap);
        cudaEventDestroy(ready);
        *st = fail_cuda(err, "scan visit cache upload");
        return nullptr;
    }
    defer_release(stream, stage, [](void *p) { delete static_cast<CallStaging *>(p); });
    scan->dev.push_back({device, static_cast<double *>(d), cap, stream, ready});
    return static_cast<double *>(d);
}

constexpr size_t kMaxUseStreams = 8;

void note_scan_use(const dd_scan *scan, cudaStream_t stream) {
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) { cudaGetLastError(); return; }
    std::lock_guard<std::mutex> lock(scan->mu);
    for (auto &c : scan->dev) {
        if (c.device != device) continue;
        if (c.any_stream) return;
        if (stream == cudaStreamPerThread) {
            // one handle for a different stream on each host thread: the release waits for
            // the whole device instead
            c.any_stream = true;
            return;
        }
        for (auto &u : c.uses)
            if (u.stream == stream) {
                if (cudaEventRecord(u.done, stream) != cudaSuccess) { cudaGetLastError(); c.any_stream = true; }
                return;
            }
        cudaEvent_t ev = nullptr;
        if (c.uses.size() >= kMaxUseStreams || cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(ev, stream) != cudaSuccess) {
            cudaGetLastError();
            if (ev) cudaEventDestroy(ev);
            c.any_stream = true;                 // released after a device synchronisation
            return;
        }
        c.uses.push_back({stream, ev});
        return;
    }
}

void scan_shared(const dd_scan *scan) {
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) { cudaGetLastError(); return; }
    std::lock_guard<std::mutex> lock(scan->mu);
    for (auto &c : scan->dev)
        if (c.device == device) c.any_stream = true;
}

const float4 *device_sources_ff(const dd_scan *scan, cudaStream_t stream, dd_status *st) {
    const double *d = device_sources(scan, stream, st);
    return d ? reinterpret_cast<const float4 *>(d + 4 * scan->n) : nullptr;
}

}  // namespace dd

namespace {

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): add the golden-gamma increment,
// then two xor-shift-multiply rounds and a final xor-shift.
struct SplitMix64 {
    uint64_t state;
    explicit SplitMix64(uint64_t seed) : state(seed) {}
    uint64_t next() {
        state += 0x9E3779B97F4A7C15ull;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};

// Fisher-Yates from the top; the swap partner of slot i is floor(u (i+1) / 2^64).
std::vector<int32_t> seeded_permutation(int64_t n, uint64_t seed) {
    std::vector<int32_t> p((size_t)n);
    for (int64_t i = 0; i < n; ++i) p[(size_t)i] = (int32_t)i;
    SplitMix64 rng(seed);
    for (int64_t i = n - 1; i > 0; --i) {
        unsigned __int128 prod = (unsigned __int128)rng.next() * (unsigned __int128)(uint64_t)(i + 1);
        int64_t j = (int64_t)(uint64_t)(prod >> 64);
        std::swap(p[(size_t)i], p[(size_t)j]);
    }
    return p;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

}  // namespace

extern "C" {

const char *dd_last_error(void) { return dd::g_last_error.c_str(); }

const char *dd_version(void) { return "dd-gb300 0.1 (sm_103a)"; }

dd_status dd_create_scan(const dd_scan_desc *d, dd_scan **out) {
    dd::clear_error();
    if (!d || !out) return dd::fail(DD_EINVAL, "dd_create_scan: NULL argument");
    if (d->nx < 1 || d->ny < 1 || (int64_t)d->nx * d->ny > (int64_t(1) << 26))
        return dd::fail(DD_EINVAL, "dd_create_scan: grid must be >= 1x1 and at most 2^26 positions");
    if (!finite_pos(d->pitch_m) || !finite_pos(d->sigma_m) || !finite_pos(d->D_m2s) ||
        !finite_pos(d->dwell_s) || !std::isfinite(d->Q0))
        return dd::fail(DD_EINVAL, "dd_create_scan: pitch, sigma, D, dwell must be finite and > 0; Q0 finite");
    if (!std::isfinite(d->flyback_s) || d->flyback_s < 0.0)
        return dd::fail(DD_EINVAL, "dd_create_scan: flyback must be finite and >= 0");
    if (!std::isfinite(d->blank_s) || d->blank_s < 0.0 || !std::isfinite(d->blank_s_per_m) ||
        d->blank_s_per_m < 0.0)
        return dd::fail(DD_EINVAL, "dd_create_scan: blanker travel times must be finite and >= 0");
    if (d->order < DD_RASTER || d->order > DD_CUSTOM)
        return dd::fail(DD_EINVAL, "dd_create_scan: unknown order");
    if (d->flyback_s != 0.0 && d->order != DD_RASTER && d->order != DD_SERPENTINE)
        return dd::fail(DD_EINVAL, "dd_create_scan: flyback applies to raster and serpentine scans only");
    if (d->order == DD_INTERLEAVED && d->interleave_stride < 1)
        return dd::fail(DD_EINVAL, "dd_create_scan: interleave stride must be >= 1");
    if (!(d->keep_fraction > 0.0 && d->keep_fraction <= 1.0))
        return dd::fail(DD_EINVAL, "dd_create_scan: keep_fraction must be in (0, 1]");
    if (d->mask && (d->keep_fraction < 1.0 || d->order == DD_CUSTOM))
        return dd::fail(DD_EINVAL, "dd_create_scan: a mask cannot be combined with keep_fraction < 1 or a custom order");
    if (d->order == DD_CUSTOM && (!d->custom_visit || d->n_custom < 1))
        return dd::fail(DD_EINVAL, "dd_create_scan: custom order needs custom_visit and n_custom >= 1");
    if (d->order == DD_CUSTOM && d->keep_fraction < 1.0)
        return dd::fail(DD_EINVAL, "dd_create_scan: keep_fraction < 1 cannot be combined with a custom order");

    const int64_t nx = d->nx, ny = d->ny, ngrid = nx * ny;
    dd_scan *s = dd::reuse_scan();
    if (!s) s = new (std::nothrow) dd_scan();
    if (!s) return dd::fail(DD_ENOMEM, "dd_create_scan: out of host memory");
    try {
        std::vector<int32_t> &seq = s->visit;            // built in place
        seq.clear();
        switch (d->order) {
        case DD_RASTER:
            seq.resize((size_t)ngrid);
            for (int64_t g = 0; g < ngrid; ++g) seq[(size_t)g] = (int32_t)g;
            break;
        case DD_SERPENTINE:
            seq.reserve((size_t)ngrid);
            for (int64_t iy = 0; iy < ny; ++iy)
                for (int64_t k = 0; k < nx; ++k)
                    seq.push_back((int32_t)(iy * nx + ((iy & 1) ? nx - 1 - k : k)));
            break;
        case DD_INTERLEAVED: {
            const int64_t S = d->interleave_stride;
            seq.reserve((size_t)ngrid);
            for (int64_t py = 0; py < S; ++py)
                for (int64_t px = 0; px < S; ++px)
                    for (int64_t iy = py; iy < ny; iy += S)
                        for (int64_t ix = px; ix < nx; ix += S)
                            seq.push_back((int32_t)(iy * nx + ix));
            break;
        }
        case DD_RANDOM:
            seq = seeded_permutation(ngrid, d->seed);
            break;
        case DD_CUSTOM:
            seq.assign(d->custom_visit, d->custom_visit + d->n_custom);
            for (int32_t g : seq)
                if (g < 0 || g >= ngrid) {
                    delete s;
                    return dd::fail(DD_EINVAL, "dd_create_scan: custom_visit index outside the grid");
                }
            break;
        }
        if (d->mask) {
            std::vector<int32_t> kept;
            kept.reserve(seq.size());
            for (int32_t g : seq)
                if (d->mask[g]) kept.push_back(g);
            seq.swap(kept);
        }
        if (d->keep_fraction < 1.0) {
            int64_t k = (int64_t)std::floor(d->keep_fraction * (double)ngrid + 0.5);
            if (k < 1) k = 1;
            std::vector<int32_t> perm = seeded_permutation(ngrid, d->seed);
            if (d->order == DD_RANDOM) {
                seq.assign(perm.begin(), perm.begin() + k);
            } else {
                std::vector<uint8_t> keep((size_t)ngrid, 0);
                for (int64_t i = 0; i < k; ++i) keep[(size_t)perm[(size_t)i]] = 1;
                std::vector<int32_t> kept;
                kept.reserve((size_t)k);
                for (int32_t g : seq)
                    if (keep[(size_t)g]) kept.push_back(g);
                seq.swap(kept);
            }
        }
        if (seq.empty()) {
            delete s;
            return dd::fail(DD_EINVAL, "dd_create_scan: the scan visits no position");
        }
        const int64_t n = (int64_t)seq.size();
        s->nx = d->nx; s->ny = d->ny; s->pitch = d->pitch_m; s->sigma = d->sigma_m;
        s->D = d->D_m2s; s->Q0 = d->Q0; s->dwell = d->dwell_s; s->flyback = d->flyback_s;
        s->order = d->order; s->stride = d->interleave_stride; s->seed = d->seed;
        s->keep_fraction = d->keep_fraction;
        s->blank = d->blank_s; s->blank_per_m = d->blank_s_per_m;
        s->n = n;
        const std::vector<int32_t> &vis = s->visit;
        s->t_start.resize((size_t)n);
        s->tau.resize((size_t)n);
        if (d->dwell_per_visit) {
            for (int64_t k = 0; k < n; ++k) {
                double tk = d->dwell_per_visit[k];
                if (!finite_pos(tk)) {
                    delete s;
                    return dd::fail(DD_EINVAL, "dd_create_scan: dwell_per_visit entries must be finite and > 0");
                }
                s->tau[(size_t)k] = tk;
            }
        } else {
            for (int64_t k = 0; k < n; ++k) s->tau[(size_t)k] = d->dwell_s;
        }
        const bool travel = d->blank_s != 0.0 || d->blank_s_per_m != 0.0;
        s->uniform = !d->dwell_per_visit && d->flyback_s == 0.0 && !travel;
        if (s->uniform) {
            for (int64_t k = 0; k < n; ++k) s->t_start[(size_t)k] = (double)k * d->dwell_s;
        } else {
            double t = 0.0;
            for (int64_t k = 0; k < n; ++k) {
                s->t_start[(size_t)k] = t;
                t = t + s->tau[(size_t)k];
                if (k + 1 == n) break;
                const int64_t g0 = vis[(size_t)k], g1 = vis[(size_t)k + 1];
                const int64_t r0 = g0 / nx, r1 = g1 / nx;
                if (d->flyback_s != 0.0 && r0 != r1) t = t + d->flyback_s;
                if (travel) {
                    // blanker travel over a jump longer than one pitch
                    const int64_t dx = g1 - r1 * nx - (g0 - r0 * nx), dy = r1 - r0;
                    const int64_t d2 = dx * dx + dy * dy;
                    if (d2 > 1) t = t + (d->blank_s + d->blank_s_per_m * (d->pitch_m * std::sqrt((double)d2)));
                }
            }
        }
        // dimensionless form
        const double p = d->pitch_m, tref = d->dwell_s;
        s->s = (d->sigma_m / p) * (d->sigma_m / p);
        s->kappa = d->D_m2s * tref / (p * p);
        s->pref = d->Q0 / (4.0 * 3.14159265358979323846 * d->D_m2s);
        s->X.resize((size_t)n); s->Y.resize((size_t)n); s->T.resize((size_t)n); s->TAU.resize((size_t)n);
        // grid row and column of each visit: g / nx from a double reciprocal, corrected to
        // the exact quotient (g < 2^26, so the product is off by less than one), instead of
        // an integer division per visit
        const double inv_nx = 1.0 / (double)nx;
        int64_t c_lo = nx, c_hi = -1, r_lo = ny, r_hi = -1;     // column and row ranges
        for (int64_t k = 0; k < n; ++k) {
            const int64_t g = vis[(size_t)k];
            int64_t q = (int64_t)((double)g * inv_nx), r = g - q * nx;
            if (r < 0) { --q; r += nx; } else if (r >= nx) { ++q; r -= nx; }
            s->X[(size_t)k] = (double)r;
            s->Y[(size_t)k] = (double)q;
            c_lo = std::min(c_lo, r); c_hi = std::max(c_hi, r);
            r_lo = std::min(r_lo, q); r_hi = std::max(r_hi, q);
        }
        s->x_lo = (double)c_lo; s->x_hi = (double)c_hi;
        s->y_lo = (double)r_lo; s->y_hi = (double)r_hi;
        if (s->uniform) {
            for (int64_t k = 0; k < n; ++k) s->T[(size_t)k] = (double)k;
            std::fill(s->TAU.begin(), s->TAU.end(), 1.0);
            s->tau_min = s->tau_max = 1.0;
        } else {
            double t_lo = s->tau[0] / tref, t_hi = t_lo;
            for (int64_t k = 0; k < n; ++k) {
                s->T[(size_t)k] = s->t_start[(size_t)k] / tref;
                const double tk = s->tau[(size_t)k] / tref;
                s->TAU[(size_t)k] = tk;
                t_lo = std::min(t_lo, tk); t_hi = std::max(t_hi, tk);
            }
            s->tau_min = t_lo; s->tau_max = t_hi;
        }
    } catch (const std::bad_alloc &) {
        delete s;
        return dd::fail(DD_ENOMEM, "dd_create_scan: out of host memory");
    }
    dd::register_scan(s);
    *out = s;
    return DD_OK;
}

dd_status dd_scan_size(const dd_scan *scan, int64_t *n_visits) {
    dd::clear_error();
    if (!scan || !n_visits) return dd::fail(DD_EINVAL, "dd_scan_size: NULL argument");
    *n_visits = scan->n;
    return DD_OK;
}

dd_status dd_scan_visits(const dd_scan *scan, int32_t *grid_index, double *t_start_s, double *dwell_s) {
    dd::clear_error();
    if (!scan) return dd::fail(DD_EINVAL, "dd_scan_visits: NULL scan");
    const size_t n = (size_t)scan->n;
    if (grid_index) std::memcpy(grid_index, scan->visit.data(), n * sizeof(int32_t));
    if (t_start_s) std::memcpy(t_start_s, scan->t_start.data(), n * sizeof(double));
    if (dwell_s) std::memcpy(dwell_s, scan->tau.data(), n * sizeof(double));
    return DD_OK;
}

void dd_destroy(dd_scan *scan) {
    if (!scan || !dd::unregister_scan(scan)) return;     // NULL or already destroyed
    int prev = -1;
    cudaGetDevice(&prev);
    for (auto &c : scan->dev) {
        if (cudaSetDevice(c.device) == cudaSuccess) {
            // wait for the work that may read the block: the upload and each stream's
            // latest use, or the whole device when the block may be read from any stream
            bool waited = !c.any_stream && cudaEventSynchronize(c.ready) == cudaSuccess;
            for (auto &u : c.uses) {
                waited = waited && cudaEventSynchronize(u.done) == cudaSuccess;
                cudaEventDestroy(u.done);
            }
            if (!waited) {
                cudaGetLastError();
                cudaDeviceSynchronize();
            }
            dd::vcache_give(c.device, c.src, c.cap);
            cudaEventDestroy(c.ready);
        }
    }
    if (!scan->dev.empty() && prev >= 0) cudaSetDevice(prev);
    cudaGetLastError();
    scan->dev.clear();
    dd::recycle_scan(scan);
}

}  // extern "C"
