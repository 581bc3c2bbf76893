// Internal declarations shared by the library's translation units (not installed).
#pragma once
#include <initializer_list>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "dd.h"

// A scan after dd_create_scan: visit list and times (SI) plus the dimensionless
// form used on the device.  Lengths are in units of the pitch p, times in units of
// the reference dwell tau_ref = desc.dwell_s.  With w(dt) = 2Ds + 4D dt (Eq. 1/2):
//   w / p^2 = 2 s + 4 kappa (dt / tau_ref),  s = Ds / p^2,  kappa = D tau_ref / p^2,
// and the arguments rho^2 / w are unchanged by the scaling.
struct dd_scan {
    int32_t nx = 0, ny = 0;
    double pitch = 0, sigma = 0, D = 0, Q0 = 0, dwell = 0, flyback = 0, blank = 0, blank_per_m = 0;
    int32_t order = 0, stride = 1;
    uint64_t seed = 0;
    double keep_fraction = 1.0;

    int64_t n = 0;                       // visits
    std::vector<int32_t> visit;          // grid index per visit
    std::vector<double> t_start, tau;    // SI seconds
    bool uniform = false;                // t_k = k * dwell and tau_k = dwell for all k (no dead time)

    double s = 0, kappa = 0, pref = 0;   // dimensionless Ds, D, and Q0/(4 pi D) [u/m^2]
    std::vector<double> X, Y, T, TAU;    // dimensionless, visit order
    double x_lo = 0, x_hi = 0, y_lo = 0, y_hi = 0, tau_min = 0, tau_max = 0;   // their ranges

    // per device: 4n doubles X | Y | T | TAU, then n float4 (x_hi, x_lo, y_hi, y_lo),
    // uploaded stream-ordered on `home`; `ready` marks the end of the upload for calls on
    // other streams
    struct DevCache {
        int device;
        double *src;
        size_t cap;                      // bytes of the block (a size class of the block cache)
        cudaStream_t home;
        cudaEvent_t ready;
        // streams whose enqueued work reads the block, each with an event recorded after
        // its latest such work; any_stream: the block was handed to work that may run on
        // any stream (a batch plan), so its release waits for the whole device
        struct Use {
            cudaStream_t stream;
            cudaEvent_t done;
        };
        std::vector<Use> uses = {};
        bool any_stream = false;
    };
    mutable std::mutex mu;
    mutable std::vector<DevCache> dev;
};

namespace ddk {
struct TcScan;
struct TcItem;
struct RecF32;
}  // namespace ddk

namespace dd {

// Record `msg` as this thread's last error and return `st`.
dd_status fail(dd_status st, const std::string &msg);
dd_status fail_cuda(cudaError_t err, const char *what);
void clear_error();

// Device copy of the scan's dimensionless visit arrays on the current device, usable by
// work enqueued on `stream` after this call: created on first use in a block that a
// destroyed scan gave back (else a new one) and uploaded on `stream` (no host
// synchronisation); a call on another stream waits for the upload's event.  Returns NULL
// on failure after recording the error in *st.
const double *device_sources(const dd_scan *scan, cudaStream_t stream, dd_status *st);
// The same visits' X, Y as float-float pairs (hi = fl32(v), lo = fl32(v - hi)), so FP32
// kernels form coordinate differences without FP64 arithmetic: n float4 stored after the
// FP64 arrays of the same cache (call after device_sources on the same stream).
const float4 *device_sources_ff(const dd_scan *scan, cudaStream_t stream, dd_status *st);

// Tensor-core contraction of grids (dd_field.cu, dd_field_tc.cuh), for batches of scans:
// the prefixes of one snapshot (visits [0, K2) on the degree-2 series and [K2, K) on the
// degree-4 series at every point of the W x H grid; both 0 when the grid takes none), the
// kernels' one-time attributes, the CTAs resident at once, and a launch over work items
// whose grids, visits and partial rows come from the scan table.
void tc_prefixes(const dd_scan *scan, double x0, double y0, double dx, double dy, int64_t W, int64_t H, double tdim,
                 int nact, int *K2, int *K);
cudaError_t prepare_field_tc();
int64_t field_tc_resident(int deg);
cudaError_t launch_field_tc(int deg, const ddk::TcScan *scans, const ddk::RecF32 *rec, const ddk::TcItem *items,
                            int n_items, int n_ctas, cudaStream_t stream);

// The work enqueued so far on `stream` may read the scan's device block on the current
// device: dd_destroy waits for it before the block is released.  scan_shared: the block
// was handed to work that may run on any stream (dd_destroy synchronises the device).
void note_scan_use(const dd_scan *scan, cudaStream_t stream);
void scan_shared(const dd_scan *scan);
// Notes the calling function's use of the scan on `stream` when it goes out of scope,
// on every return path after the device block was obtained.
struct ScanUse {
    const dd_scan *scan;
    cudaStream_t stream;
    ~ScanUse() { note_scan_use(scan, stream); }
};

// True if `p` is device-accessible memory of the current device.
bool is_device_pointer(const void *p);
// Where a user buffer lives: device (or managed) memory, page-locked host memory, or
// pageable host memory.
enum class MemKind { Device, Pinned, Pageable };
MemKind memory_kind(const void *p);
// Whether a call with these buffers must synchronise its stream before returning: it has
// a host buffer, and either runs on the legacy default stream (NULL) or one of its host
// buffers is pageable.  With a stream given and only page-locked host buffers the call
// leaves its copies enqueued (the caller synchronises before reading).
bool host_sync_needed(cudaStream_t stream, std::initializer_list<MemKind> kinds);

// Stream-ordered workspace of a call on the current device: a released block of the same
// size class that is free for `stream` (last used on it, or its work done), else a new
// block from the library's memory pool (which keeps up to 4 GiB of freed memory mapped:
// the default pool returns it to the driver at every synchronisation).  Returns the CUDA
// error.
cudaError_t workspace_alloc(void **p, size_t bytes, cudaStream_t stream);
// Hands a workspace back after the work enqueued on `stream` that uses it (an event
// recorded there marks when another stream may take it).
cudaError_t workspace_release(void *p, cudaStream_t stream);

// Pinned host staging for the small tables a call uploads (work lists, snapshot
// tables).  A copy from pageable memory is staged by the driver and can hold the host
// until the stream drains, which serialises the host's preparation of the next call
// with the GPU; from pinned memory it is a plain asynchronous DMA.  Blocks are recycled:
// a call takes blocks, and the host function it enqueues after its copies gives them
// back once the copies have completed.  pinned_take returns
// {nullptr, 0} if pinned memory cannot be had; the caller then copies from pageable
// memory.
struct PinnedBlock {
    void *p = nullptr;
    size_t cap = 0;
};
PinnedBlock pinned_take(size_t bytes);
void pinned_give(PinnedBlock b);

// The pinned blocks one call staged its uploads through; given back when this is deleted
// (after the stream has consumed the copies: see defer_release).
struct CallStaging {
    std::vector<PinnedBlock> blocks;
    CallStaging() = default;
    CallStaging(const CallStaging &) = delete;
    CallStaging &operator=(const CallStaging &) = delete;
    ~CallStaging() {
        for (auto &b : blocks) pinned_give(b);
    }
    // n bytes at host src to device dst on `stream`, through a pinned block when one can be
    // had (src must then stay valid only for this call), else straight from src (which
    // must stay valid until the stream has consumed the copy).
    cudaError_t upload(void *dst, const void *src, size_t n, cudaStream_t stream) {
        if (n == 0) return cudaSuccess;
        PinnedBlock b = pinned_take(n);
        if (!b.p) return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, stream);
        std::memcpy(b.p, src, n);
        blocks.push_back(b);
        return cudaMemcpyAsync(dst, b.p, n, cudaMemcpyHostToDevice, stream);
    }
    // A pinned block of n bytes, kept with the others, for the caller to fill in place and
    // copy from (one pass over the data instead of two); nullptr when none can be had.
    void *stage(size_t n) {
        PinnedBlock b = pinned_take(n);
        if (!b.p) return nullptr;
        blocks.push_back(b);
        return b.p;
    }
};

// Keeps a call's host tables (and the pinned blocks their uploads came from) alive until
// the work enqueued so far on `stream` has completed, without putting a host function in
// the stream (a host function stalls the stream until the driver's callback thread has
// run it).  An event recorded now marks the point; later calls release every entry whose
// event has completed, and wait for the oldest once more than 256 are pending.  `obj` is
// deleted by `del`.  Returns the CUDA error of the event record (then `obj` is deleted
// only after a device synchronisation).
cudaError_t defer_release(cudaStream_t stream, void *obj, void (*del)(void *));

// Host-side fault injection for tests: true when the environment variable DD_FAULT
// names `site` (e.g. DD_FAULT=alloc makes the next workspace allocations fail as if
// the device were out of memory).  No device fault is ever produced.
bool fault_injected(const char *site);

// Registry of live scan handles (guards dd_destroy against double frees).
void register_scan(dd_scan *s);
bool unregister_scan(dd_scan *s);
// A destroyed scan kept for its host storage (NULL if none), and the hand-back of a
// destroyed scan (kept if small enough and the spares are not full, else deleted).
dd_scan *reuse_scan();
void recycle_scan(dd_scan *s);

// Kernel timing scope (dd_profile.cpp): records an event pair around the launch
// made inside the scope when profiling is enabled, nothing otherwise.
class ProfScope {
  public:
    ProfScope(const char *name, cudaStream_t stream);
    ~ProfScope();
    ProfScope(const ProfScope &) = delete;
    ProfScope &operator=(const ProfScope &) = delete;

  private:
    const char *name_;
    cudaStream_t stream_;
    cudaEvent_t a_{}, b_{};
    bool active_ = false;
};

}  // namespace dd

// Launch `launch` (a kernel<<<...>>> expression) under a ProfScope named `name`.
#define DD_PROFILED(name, stream, launch) \
    do {                                   \
        dd::ProfScope dd_ps_(name, stream); \
        launch;                            \
    } while (0)

#define DD_CUDA_TRY(expr)                                              \
    do {                                                               \
        cudaError_t dd_err_ = (expr);                                  \
        if (dd_err_ != cudaSuccess) return dd::fail_cuda(dd_err_, #expr); \
    } while (0)
