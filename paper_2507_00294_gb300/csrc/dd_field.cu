// dd_field.cu -- cumulative damage field psi(r, t) of Eq. 5 on the GPU.
//
//   psi(r,t) = Q0/(4 pi D) sum_{i : t_i < t} [E1(rho_i^2 / w1) - E1(rho_i^2 / w0)]
//   w1 = 2s + 4 kappa (t - t_i),  w0 = 2s (beam on, Eq. 1) or 2s + 4 kappa (t - t_i - tau_i)
//   (beam off, Eq. 2), in units of the pitch and the reference dwell (dd_internal.h).
//
// Pipeline of one dd_field_at_times call (all on the caller's stream):
//   1. points SI -> pitch units (prep_points_kernel; with the lag table of step 2 in one
//      launch, prep_points_lag_kernel, when the snapshots lie on the dwell lattice);
//   2. per (snapshot, visit) FP64 coefficients: q1 = 1/w1, dq = 1/w0 - 1/w1 and the
//      moment coefficients c_0..c_M of dd_e1.cuh (coef_kernel);
//   3. work items (point tile, snapshot chunk, visit block), sorted by cost, one CTA
//      each (field_kernel): the block's visits are staged in shared memory in visit
//      order, every thread keeps PPT points x TCH snapshots in registers, and each
//      snapshot only sums the visits that have started (causal prefix n_active(t));
//   4. deterministic reduce of the per-block partial sums in block order, times
//      Q0/(4 pi D), into out[snapshot][point] (reduce_kernel).
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <limits>
#include <numeric>
#include <vector>

#include "dd_coef.cuh"
#include "dd_e1.cuh"
#include "dd_field_grid.cuh"
#include "dd_field_impl.cuh"
#include "dd_field_tc.cuh"
#include "dd_internal.h"

namespace ddk {

// A rectilinear grid of evaluation points: point k = r W + c at (x0 + c dx, y0 + r dy)
// (SI); W = 0 for an explicit point list.
struct GridDesc {
    double x0 = 0, y0 = 0, dx = 0, dy = 0;
    int64_t W = 0, H = 0;
};

// Points in pitch units: FP64 X, Y, and float-float (x_hi, x_lo, y_hi, y_lo) for the FP32
// tile, so that the FP32 kernels form coordinate differences without FP64 arithmetic.
// A grid point is formed in SI as x0 + c dx (one product, one sum, no fused multiply-add:
// the values a caller's point list of the same grid holds).
__device__ __forceinline__ void prep_point(int64_t k, const double *__restrict__ xy, const GridDesc &g, int64_t n,
                                           double inv_p, double *__restrict__ X, double *__restrict__ Y,
                                           float4 *__restrict__ F) {
    if (k >= n) return;
    double xs, ys;
    if (g.W > 0) {
        const int64_t r = k / g.W, c = k - r * g.W;
        xs = __dadd_rn(__dmul_rn((double)c, g.dx), g.x0);
        ys = __dadd_rn(__dmul_rn((double)r, g.dy), g.y0);
    } else {
        xs = xy[2 * k];
        ys = xy[2 * k + 1];
    }
    const double x = xs * inv_p, y = ys * inv_p;
    X[k] = x;
    Y[k] = y;
    const float xh = (float)x, yh = (float)y;
    F[k] = make_float4(xh, (float)(x - (double)xh), yh, (float)(y - (double)yh));
}
__global__ void prep_points_kernel(const double *__restrict__ xy, GridDesc g, int64_t n, double inv_p,
                                   double *__restrict__ X, double *__restrict__ Y, float4 *__restrict__ F) {
    prep_point((int64_t)blockIdx.x * blockDim.x + threadIdx.x, xy, g, n, inv_p, X, Y, F);
}

// The reversed lag table (blocks [0, nb_lag), one record per thread: a long serial chain,
// so these blocks go first) and the points in pitch units (the blocks after) in one
// launch: the field's two preparation steps cost one launch instead of two.
template <typename Rec>
__global__ void prep_points_lag_kernel(int nb_lag, int64_t M, double s, double kappa, Rec *__restrict__ rev,
                                       const double *__restrict__ xy, GridDesc g, int64_t n, double inv_p,
                                       double *__restrict__ X, double *__restrict__ Y, float4 *__restrict__ F) {
    if ((int)blockIdx.x < nb_lag)
        rev_lag_record<Rec>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, M, s, kappa, rev);
    else
        prep_point((int64_t)(blockIdx.x - nb_lag) * blockDim.x + threadIdx.x, xy, g, n, inv_p, X, Y, F);
}

// out[row[j]][p] = pref * (sum_{q < nq[j]} tpart[(trow0[j] + q) * pstride + p]
//                          + sum_{kb0[j] <= k < nblk[j]} partial[(k * n_tg + j) * pstride + p]):
// the tensor-core chunks of snapshot j (the older visits), then its visit blocks, in that
// order (deterministic); four points per thread, so that each load moves 16 bytes or more.
// kb0 and nq NULL: every block from 0, no tensor-core rows.
template <typename Part>
__global__ void reduce_kernel(const Part *__restrict__ partial, const int *__restrict__ nblk_of_snap,
                              const int *__restrict__ kb0_of_snap, const Part *__restrict__ tpart,
                              const int *__restrict__ nq_of_snap, const int *__restrict__ trow0,
                              const int *__restrict__ row, int n_tg, int64_t n_pts, int64_t pstride, double pref,
                              double *__restrict__ out) {
    const int j = blockIdx.y;
    const int64_t p0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (p0 >= n_pts) return;
    const int nb = nblk_of_snap[j];
    const int kb0 = kb0_of_snap ? kb0_of_snap[j] : 0;
    const int nq = nq_of_snap ? nq_of_snap[j] : 0;
    BlockSum<Part> acc[4];
    for (int k = 0; k < nq; ++k) {
        Part v[4];
        load4_cg(tpart + ((int64_t)trow0[j] + k) * pstride + p0, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q].add(v[q]);
    }
#pragma unroll 4
    for (int k = kb0; k < nb; ++k) {
        Part v[4];
        load4_cg(partial + ((int64_t)k * n_tg + j) * pstride + p0, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q].add(v[q]);
    }
    double *o = out + (int64_t)row[j] * n_pts + p0;
    if (p0 + 3 < n_pts && (reinterpret_cast<uintptr_t>(o) & 15) == 0) {
        // 32 contiguous bytes per thread: whole lines per warp
        reinterpret_cast<double2 *>(o)[0] = make_double2(pref * acc[0].result(), pref * acc[1].result());
        reinterpret_cast<double2 *>(o)[1] = make_double2(pref * acc[2].result(), pref * acc[3].result());
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (p0 + q < n_pts) o[q] = pref * acc[q].result();
    }
}

}  // namespace ddk

// ============================================================== host dispatcher
namespace {

using ddk::RecF32;
using ddk::RecF64;

struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(void *b) : base((char *)b) {}
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = (T *)(base + off);
        off += count * sizeof(T);
        return p;
    }
};

// Host-side tables, uploaded through pinned staging blocks; freed (and the blocks given
// back) once an event recorded after the uploads has completed.
struct HostTables {
    std::vector<std::vector<int2>> items;
    std::vector<std::vector<int>> ints;
    std::vector<std::vector<double>> reals;
    std::vector<std::vector<int64_t>> offs;
    std::vector<std::vector<char>> images; // per group: the tables as laid out on the device
    dd::CallStaging staging;               // pinned copies the uploads were made from
    static void release(void *p) { delete static_cast<HostTables *>(p); }
};

// Sizes of the workspace a call needs (the same function drives the carve).
template <typename Cfg>
size_t workspace_bytes(int64_t n_pts, int64_t n_src, int group, int sb, bool out_host, bool pts_host,
                       int n_t, int64_t n_rec, int64_t trows, int64_t n_titems) {
    using Rec = typename Cfg::Rec;
    const int nblk_max = (int)((n_src + sb - 1) / sb);
    const int n_chunks = (group + Cfg::kTCH - 1) / Cfg::kTCH;
    size_t b = 0;
    auto add = [&](size_t bytes) { b = ((b + 255) & ~size_t(255)) + bytes; };
    if (pts_host) add(2 * (size_t)n_pts * sizeof(double));
    if (out_host) add((size_t)n_t * n_pts * sizeof(double));
    add(2 * (size_t)n_pts * sizeof(double));                  // X, Y in pitch units
    add((size_t)n_pts * sizeof(float4));                      // the same as float-float
    add((size_t)group * sizeof(double));                      // snapshot times
    add((size_t)group * sizeof(int) * 7);                     // nact, row, nblk, kst, kb0, nq, trow0 per snapshot
    add((size_t)group * sizeof(int64_t));                     // record row offset per snapshot
    add((size_t)n_chunks * nblk_max * sizeof(int2));          // (chunk, block) descriptors
    add((size_t)n_titems * sizeof(ddk::TcItem));              // tensor-core work items
    add((size_t)n_rec * sizeof(Rec));                         // coefficient records
    add((size_t)nblk_max * group * ((n_pts + 3) / 4 * 4) * sizeof(typename Cfg::Real));   // partial sums
    add((size_t)trows * ((n_pts + 3) / 4 * 4) * sizeof(float));                           // tensor-core partials
    return b + 256;
}

// Shared-memory carveout of the tile kernels (Cfg::kCarveout, percent of the L1/shared
// array), set once per device: the FP32-mixed tile's 8 CTAs of 13 KB fit in 132 KB and
// the rest stays L1 for the minority classes' record reads (about 1 % faster than the
// whole array as shared memory); the FP64 tile takes the whole array.
// The grid tile (dd_field_grid.cuh): 128 columns x GridCfg::kPPT = 4 rows (a tile of 8 rows
// per thread, 80 registers and 6 CTAs per SM, measured 8 % slower).  Its row tables sit
// beside the general tile's 12 KB: 8 CTAs of 17.3 KB (with the per-CTA reserve) need a 66 %
// carveout.
using GridCfg = ddk::CfgMixed;
constexpr int kGridCarveout = 66;

template <typename Cfg, bool kGrid>
struct TileKernel {
    static constexpr auto fn() { return ddk::field_kernel<Cfg>; }
    static constexpr int carveout = Cfg::kCarveout;
};
template <>
struct TileKernel<ddk::CfgMixed, true> {
    static constexpr auto fn() { return ddk::field_grid_kernel<GridCfg>; }
    static constexpr int carveout = kGridCarveout;
};

template <typename Cfg, bool kGrid = false>
cudaError_t prefer_shared() {
    static std::atomic<uint64_t> done{0};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess || dev >= 64) return err;
    if (done.load() & (uint64_t(1) << dev)) return cudaSuccess;
    err = cudaFuncSetAttribute(TileKernel<Cfg, kGrid>::fn(), cudaFuncAttributePreferredSharedMemoryCarveout,
                               TileKernel<Cfg, kGrid>::carveout);
    if (err == cudaSuccess) done.fetch_or(uint64_t(1) << dev);
    return err;
}

// CTAs of the tile kernel resident on the whole device at once (0 if unknown).
template <typename Cfg, bool kGrid = false>
int64_t resident_ctas() {
    static std::atomic<int64_t> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return 0;
    int64_t v = cached[dev].load();
    if (v > 0) return v;
    if (prefer_shared<Cfg, kGrid>() != cudaSuccess) cudaGetLastError();   // occupancy at the carveout used
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, TileKernel<Cfg, kGrid>::fn(), Cfg::kThreads, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    v = (int64_t)per_sm * sms;
    cached[dev].store(v);
    return v;
}

// ---- the tensor-core part of the grid field (dd_field_tc.cuh)
//
// A visit is handed to the contraction for snapshot j when its pair term is on the degree-2
// (or degree-4) series at every point of the grid: h = rho^2 dq <= kL2H (kL4H) for rho^2 up
// to R2, the largest squared distance between the grid's box and the box of the visits.
// With c = 4 kappa tau_max, dq = 1/w0 - 1/w1 <= c / ((w1 - c) w1) for every visit of the
// scan (dq grows with the dwell at a fixed w1 = 2s + 4 kappa (t - T_i)), so every visit
// with w1 at or above the root w1* of (w1 - c) w1 = c R2 / h_limit (and its dwell over)
// qualifies: the prefix of the visits that started by t_j - dT*, dT* = (w1* - 2s) /
// (4 kappa), found by bisection of the start times.  The degree-2 prefix [0, K2) and the
// degree-4 band [K2, K) go to the contraction (the degree-4 band only while its records'
// g_4x = log2(e) l_4 dq^4 stay in the FP32 normal range, dq >= kMinDqX), the rest [K, nact)
// to the CUDA-core tile.
struct TcPlan {
    bool on = false;
    int64_t n_tile_cols = 0, n_tiles = 0;
    std::vector<int> K2;         // per snapshot (time order): the degree-2 visits [0, K2)
    std::vector<int> K;          // and the degree-4 band [K2, K); the CUDA-core tile from K
};

// Age (in dwells) from which every visit of the scan is on the series of the given h limit
// at every point within R2, or a negative value if none is.
double tc_min_age(const dd_scan *scan, double R2, double h_limit, double *w1s_out) {
    const double dq_max = h_limit * (1.0 - 1e-4) / R2;
    const double c = 4.0 * scan->kappa * scan->tau_max;
    if (!(c > 0.0) || !(dq_max > 0.0) || !std::isfinite(dq_max)) return -1.0;
    double w1s = 0.5 * (c + std::sqrt(c * c + 4.0 * c / dq_max));
    w1s = std::max(w1s, (2.0 * scan->s + c) * (1.0 + 1e-9));        // the dwell is over
    if (w1s_out) *w1s_out = w1s;
    return (w1s - 2.0 * scan->s) / (4.0 * scan->kappa) * (1.0 + 1e-9);
}

TcPlan plan_tc(const dd_scan *scan, const ddk::GridDesc &grid, const std::vector<double> &tdim,
               const std::vector<int> &nact) {
    TcPlan tp;
    const int n_t = (int)tdim.size();
    tp.K2.assign(n_t, 0);
    tp.K.assign(n_t, 0);
    // tiles of 128 x 128 points: only grids that fill them reasonably
    if (grid.W < ddk::kTcTile / 2 || grid.H < ddk::kTcTile / 2 || scan->n == 0) return tp;
    const double ip = 1.0 / scan->pitch;
    const double xa = grid.x0 * ip, xb = (grid.x0 + (double)(grid.W - 1) * grid.dx) * ip;
    const double ya = grid.y0 * ip, yb = (grid.y0 + (double)(grid.H - 1) * grid.dy) * ip;
    const double ex = std::max(std::max(xa, xb) - scan->x_lo, scan->x_hi - std::min(xa, xb));
    const double ey = std::max(std::max(ya, yb) - scan->y_lo, scan->y_hi - std::min(ya, yb));
    // margins for the points' own rounding and the records' rounding to FP32
    const double R2 = (ex * ex + ey * ey) * (1.0 + 1e-6) + 1e-6;
    double w1s2 = 0.0;
    const double age2 = tc_min_age(scan, R2, (double)ddk::kL2H, &w1s2);
    if (age2 < 0.0) return tp;
    double age4 = tc_min_age(scan, R2, (double)ddk::kL4H, nullptr);
    // the degree-4 band's smallest dq: its oldest visit (w1 up to w1s2) with the shortest dwell
    const double cmin = 4.0 * scan->kappa * scan->tau_min;
    if (age4 < 0.0 || !(w1s2 > cmin) || cmin / ((w1s2 - cmin) * w1s2) < 2.0 * (double)ddk::kMinDqX) age4 = age2;
    int64_t any = 0;
    for (int k = 0; k < n_t; ++k) {
        const int64_t k2 = std::upper_bound(scan->T.begin(), scan->T.end(), tdim[k] - age2) - scan->T.begin();
        const int64_t k4 = std::upper_bound(scan->T.begin(), scan->T.end(), tdim[k] - std::min(age4, age2)) - scan->T.begin();
        tp.K2[k] = (int)std::min<int64_t>(k2, nact[k]);
        tp.K[k] = (int)std::max<int64_t>(tp.K2[k], std::min<int64_t>(k4, nact[k]));
        any += tp.K[k];
    }
    if (any == 0) return tp;
    tp.n_tile_cols = (grid.W + ddk::kTcTile - 1) / ddk::kTcTile;
    tp.n_tiles = tp.n_tile_cols * ((grid.H + ddk::kTcTile - 1) / ddk::kTcTile);
    tp.on = true;
    return tp;
}

// dynamic shared memory above 48 KB and the whole L1/shared array as shared memory, set
// once per device
template <int kDeg>
cudaError_t prepare_tc_kernel() {
    static std::atomic<uint64_t> done{0};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess || dev >= 64) return err;
    if (done.load() & (uint64_t(1) << dev)) return cudaSuccess;
    err = cudaFuncSetAttribute(ddk::field_grid_tc_kernel<kDeg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               ddk::TcConst<kDeg>::kSmemBytes);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(ddk::field_grid_tc_kernel<kDeg>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared);
    if (err == cudaSuccess) done.fetch_or(uint64_t(1) << dev);
    return err;
}

// Tensor-core CTAs of the degree-kDeg kernel resident on the whole device at once (their
// shared memory and tensor memory bound it per SM; 0 if unknown).
template <int kDeg>
int64_t tc_resident_ctas() {
    static std::atomic<int64_t> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return 0;
    int64_t v = cached[dev].load();
    if (v > 0) return v;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    v = (int64_t)ddk::TcShape<kDeg>::kCtasPerSm * sms;
    cached[dev].store(v);
    return v;
}

// The tensor-core contraction runs on a side stream of the calling thread, forked from the
// caller's stream after the coefficients and joined back before the reduce, so that its CTAs
// fill the SMs the CUDA-core tile kernel leaves idle.  One stream and two events per
// (thread, device), created on first use (reusing an event is safe: a wait takes the state
// of the event's latest record when it is issued).
constexpr bool kTcBeforeCore = false;        // submission order of the two grid kernels
constexpr bool kTcHighPriority = false;      // the side stream's priority (else the lowest)
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
cudaError_t side_stream(SideStream **out) {
    thread_local SideStream per_dev[64];
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev >= 64) return cudaErrorInvalidDevice;
    SideStream &ss = per_dev[dev];
    if (!ss.s) {
        int lo = 0, hi = 0;
        if ((err = cudaDeviceGetStreamPriorityRange(&lo, &hi)) != cudaSuccess) return err;
        if ((err = cudaStreamCreateWithPriority(&ss.s, cudaStreamNonBlocking, kTcHighPriority ? hi : lo)) != cudaSuccess)
            return err;
        if ((err = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming)) != cudaSuccess) return err;
        if ((err = cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming)) != cudaSuccess) return err;
    }
    *out = &ss;
    return cudaSuccess;
}

// Pieces of each snapshot's visit range [lo[j], hi[j]) for one launch over snapshots
// [g0, g0 + ng): about one work item per resident CTA (every item the same number of 16-visit
// stages, give or take the rounding), so that the launch is one wave and each CTA writes one
// partial row per item; and no piece longer than kTcMaxItemStages stages (the accumulation's
// error budget).
std::vector<int> tc_pieces(const std::vector<int> &lo, const std::vector<int> &hi, int64_t n_tiles, int g0, int ng,
                           int64_t slots) {
    std::vector<int> pieces(ng, 0);
    auto stages = [&](int j) { return (int64_t)((hi[g0 + j] - lo[g0 + j] + ddk::kTcStage - 1) / ddk::kTcStage); };
    int64_t total = 0;
    for (int j = 0; j < ng; ++j) total += stages(j) * n_tiles;
    if (total == 0) return pieces;
    const int64_t per = std::max<int64_t>(1, (total + std::max<int64_t>(slots, 1) - 1) / std::max<int64_t>(slots, 1));
    for (int j = 0; j < ng; ++j) {
        const int64_t S = stages(j);
        if (S > 0) pieces[j] = (int)std::max<int64_t>(1, (S * n_tiles + per / 2) / per / std::max<int64_t>(n_tiles, 1));
        if (S > 0) pieces[j] = (int)std::min<int64_t>(std::max<int64_t>({(int64_t)pieces[j], 1,
                                                                        (S + ddk::kTcMaxItemStages - 1) / ddk::kTcMaxItemStages}), S);
    }
    return pieces;
}

// Snapshots in time order: order[k] = index into times of the k-th earliest, tdim[k] its time
// in dwells and nact[k] = #{i : T_i < t} (the visits started by then).  Returns true for
// snapshots on the dwell lattice of a uniform scan (t = integer number of dwells, to within
// 2 ulp of the quotient -- the rounding t/dwell itself already carries; tdim is then rounded
// to those integers and M is the last): the record of (snapshot, visit) then depends on the
// lag only, so one reversed lag table of M + 1 records serves every snapshot.
bool snapshot_dims(const dd_scan *scan, const std::vector<double> &times, std::vector<int> &order,
                   std::vector<double> &tdim, std::vector<int> &nact, int64_t &M) {
    const int n_t = (int)times.size();
    const int64_t n_src = scan->n;
    order.resize(n_t);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return times[a] < times[b]; });
    tdim.resize(n_t);
    nact.resize(n_t);
    for (int k = 0; k < n_t; ++k) tdim[k] = times[order[k]] / scan->dwell;
    bool lattice = scan->uniform;
    M = 0;
    for (int k = 0; k < n_t && lattice; ++k) {
        const double r = std::nearbyint(tdim[k]);
        if (std::fabs(tdim[k] - r) > 2.0 * std::numeric_limits<double>::epsilon() * std::fabs(r)) lattice = false;
        else if (r > (double)M) M = (int64_t)r;
    }
    if (M < 1 || M > 4 * n_src + 64) lattice = false;
    if (lattice)
        for (int k = 0; k < n_t; ++k) tdim[k] = std::nearbyint(tdim[k]);
    for (int k = 0; k < n_t; ++k)
        nact[k] = (int)(std::lower_bound(scan->T.begin(), scan->T.end(), tdim[k]) - scan->T.begin());
    return lattice;
}

// pts_xy_m == NULL: the points are the grid `grid` (row-major, n_pts = W H), formed on
// the device; the FP32-mixed path then runs the grid tile kernel.
template <typename Cfg>
dd_status run_field(const dd_scan *scan, const double *pts_xy_m, int64_t n_pts, const ddk::GridDesc &grid,
                    const std::vector<double> &times, double *out, cudaStream_t stream) {
    using Rec = typename Cfg::Rec;
    constexpr bool kMixed = std::is_same<typename Cfg::Real, float>::value;
    const bool on_grid = grid.W > 0;
    const bool grid_tiles = kMixed && on_grid;
    const int64_t n_src = scan->n;
    const int n_t = (int)times.size();
    const dd::MemKind pts_kind = on_grid ? dd::MemKind::Device : dd::memory_kind(pts_xy_m);
    const dd::MemKind out_kind = dd::memory_kind(out);
    const bool pts_host = pts_kind != dd::MemKind::Device;
    const bool out_host = out_kind != dd::MemKind::Device;
    // host buffers go through a workspace copy (a pinned output written in place by the
    // reduce measured slower than the copy engine's transfer)
    const bool pts_copy = pts_host, out_copy = out_host;

    std::vector<int> order, nact;
    std::vector<double> tdim;
    int64_t M = 0;
    const bool lattice = snapshot_dims(scan, times, order, tdim, nact, M);
    // the degree-2 prefixes that the tensor-core contraction takes (grid tiles only)
    TcPlan tp;
    tp.K2.assign(n_t, 0);
    tp.K.assign(n_t, 0);
    if (grid_tiles) tp = plan_tc(scan, grid, tdim, nact);
    const std::vector<int> zeros(n_t, 0);

    // visit block size and snapshot groups bound the partial and record buffers
    const int tile = Cfg::kThreads * Cfg::kPPT;
    // grid tiles: 128 columns x 4 rows (kThreads x kPPT); otherwise 512 consecutive points
    const int64_t n_tc = grid_tiles ? (grid.W + Cfg::kThreads - 1) / Cfg::kThreads : 0;
    const int64_t n_tiles = grid_tiles ? n_tc * ((grid.H + GridCfg::kPPT - 1) / GridCfg::kPPT)
                                       : (n_pts + tile - 1) / tile;
    int sb = Cfg::kSB;
    int group = n_t;
    const size_t budget = size_t(1) << 30;
    while (group > Cfg::kTCH &&
           (size_t)(lattice ? 0 : group * n_src) * sizeof(Rec) + (size_t)((n_src + sb - 1) / sb) * group * ((n_pts + 3) / 4 * 4) * sizeof(typename Cfg::Real) > budget)
        group = std::max(Cfg::kTCH, group / 2);
    // larger blocks only while the FP32 stage sums stay short (<= 32 stages)
    while ((size_t)((n_src + sb - 1) / sb) * group * ((n_pts + 3) / 4 * 4) * sizeof(typename Cfg::Real) > budget && sb < 32 * Cfg::kSTILE) sb *= 2;
    // smaller blocks (down to 128 visits, 64 for grid tiles) while one launch has fewer than
    // 4 waves of resident CTAs, so that the last wave's stragglers cost little (on a grid the
    // tile kernel takes only the visits the tensor-core contraction leaves, and 64-visit
    // blocks measured 3 % faster there)
    {
        constexpr int kWaves = 4;
        const int64_t waves4 = kWaves * (grid_tiles ? resident_ctas<Cfg, true>() : resident_ctas<Cfg>());
        const int n_groups = (n_t + group - 1) / group;
        auto items_per_launch = [&](int b) {
            int64_t blocks = 0;
            for (int j0 = 0; j0 < n_t; j0 += Cfg::kTCH) {
                int cmax = 0, kmin = INT_MAX;
                for (int j = j0; j < std::min(n_t, j0 + Cfg::kTCH); ++j) {
                    cmax = std::max(cmax, nact[j]);
                    kmin = std::min(kmin, tp.K[j] / b);
                }
                blocks += std::max(0, (cmax + b - 1) / b - kmin);
            }
            return blocks * n_tiles / std::max(1, n_groups);
        };
        const int sb_min = grid_tiles ? 64 : 128;
        while (sb > sb_min && waves4 > 0 && items_per_launch(sb) < waves4 &&
               (size_t)((n_src + sb / 2 - 1) / (sb / 2)) * group * ((n_pts + 3) / 4 * 4) * sizeof(typename Cfg::Real) <= budget)
            sb /= 2;
    }
    const int nblk_max = (int)((n_src + sb - 1) / sb);
    const int n_chunks_max = (group + Cfg::kTCH - 1) / Cfg::kTCH;
    // tensor-core chunks: rows of partial sums per snapshot and work items per group, within
    // the partial-sum budget (else the CUDA-core tile takes every visit)
    int64_t trows_max = 0, n_titems_max = 0;
    const int64_t tc_slots2 = tp.on ? std::max<int64_t>(1, tc_resident_ctas<2>()) : 1;
    const int64_t tc_slots4 = tp.on ? std::max<int64_t>(1, tc_resident_ctas<4>()) : 1;
    if (tp.on) {
        for (int g0 = 0; g0 < n_t; g0 += group) {
            const int ng = std::min(group, n_t - g0);
            const std::vector<int> p2 = tc_pieces(zeros, tp.K2, tp.n_tiles, g0, ng, tc_slots2);
            const std::vector<int> p4 = tc_pieces(tp.K2, tp.K, tp.n_tiles, g0, ng, tc_slots4);
            int64_t rows = 0;
            for (int j = 0; j < ng; ++j) rows += p2[j] + p4[j];
            trows_max = std::max(trows_max, rows);
            n_titems_max = std::max(n_titems_max, rows * tp.n_tiles);
        }
        if ((size_t)trows_max * ((n_pts + 3) / 4 * 4) * sizeof(float) > budget || n_titems_max > (int64_t(1) << 24)) {
            tp.on = false;
            std::fill(tp.K2.begin(), tp.K2.end(), 0);
            std::fill(tp.K.begin(), tp.K.end(), 0);
            trows_max = 0;
            n_titems_max = 0;
        }
    }

    const int64_t n_rec = lattice ? M + 1 : (int64_t)group * n_src;
    const size_t ws_bytes = workspace_bytes<Cfg>(n_pts, n_src, group, sb, out_copy, pts_copy, n_t, n_rec, trows_max,
                                                 n_titems_max);
    dd_status st = DD_OK;
    const double *src = dd::device_sources(scan, stream, &st);
    if (!src) return st;
    const dd::ScanUse use{scan, stream};
    const float4 *srcF = dd::device_sources_ff(scan, stream, &st);
    void *ws = nullptr;
    cudaError_t err = dd::fault_injected("alloc") ? cudaErrorMemoryAllocation
                                                  : dd::workspace_alloc(&ws, ws_bytes, stream);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return dd::fail(err == cudaErrorMemoryAllocation ? DD_ENOMEM : DD_ECUDA,
                        std::string("field workspace allocation: ") + cudaGetErrorString(err));
    }
    Carve cv(ws);
    const double *pts_dev = pts_xy_m;
    if (pts_copy) {
        double *p = cv.take<double>(2 * (size_t)n_pts);
        DD_CUDA_TRY(cudaMemcpyAsync(p, pts_xy_m, 2 * (size_t)n_pts * sizeof(double), cudaMemcpyHostToDevice, stream));
        pts_dev = p;
    }
    double *out_dev = out_copy ? cv.take<double>((size_t)n_t * n_pts) : out;
    double *X = cv.take<double>(2 * (size_t)n_pts);
    double *Y = X + n_pts;
    float4 *PF = cv.take<float4>((size_t)n_pts);
    double *d_t = cv.take<double>(group);
    int *d_nact = cv.take<int>(7 * (size_t)group);
    int *d_row = d_nact + group;
    int *d_nblk = d_row + group;
    int *d_kst = d_nblk + group;
    int *d_kb0 = d_kst + group;
    int *d_nq = d_kb0 + group;
    int *d_trow0 = d_nq + group;
    int64_t *d_roff = cv.take<int64_t>(group);
    int2 *d_desc = cv.take<int2>((size_t)n_chunks_max * nblk_max);
    ddk::TcItem *d_titems = cv.take<ddk::TcItem>((size_t)n_titems_max);
    Rec *d_rec = cv.take<Rec>((size_t)n_rec);
    using Part = typename Cfg::Real;
    const int64_t pstride = (n_pts + 3) / 4 * 4;            // 16-byte aligned partial rows
    Part *d_part = cv.take<Part>((size_t)nblk_max * group * pstride);
    float *d_tpart = cv.take<float>((size_t)trows_max * pstride);

    if (!lattice) {
        DD_PROFILED("prep_points", stream,
                    (ddk::prep_points_kernel<<<(unsigned)((n_pts + 255) / 256), 256, 0, stream>>>(pts_dev, grid, n_pts, 1.0 / scan->pitch, X, Y, PF)));
        DD_CUDA_TRY(cudaGetLastError());
    }

    const double *srcX = src, *srcY = src + n_src, *srcT = src + 2 * n_src, *srcTAU = src + 3 * n_src;
    // host staging for the per-group tables, released by a host callback once the
    // stream has consumed them (the copies below may read pageable memory late)
    HostTables *keep = new HostTables();
    if (lattice) {
        // the lag table and the points in one launch of 32-thread blocks
        const int nb_lag = (int)((M + 1 + 31) / 32);
        const int64_t nb_pts = (n_pts + 31) / 32;
        DD_PROFILED(Cfg::kCoefName, stream,
                    (ddk::prep_points_lag_kernel<Rec><<<(unsigned)(nb_lag + nb_pts), 32, 0, stream>>>(
                        nb_lag, M, scan->s, scan->kappa, d_rec, pts_dev, grid, n_pts, 1.0 / scan->pitch, X, Y, PF)));
        DD_CUDA_TRY(cudaGetLastError());
    }
    for (int g0 = 0; g0 < n_t; g0 += group) {
        const int ng = std::min(group, n_t - g0);
        const int n_chunks = (ng + Cfg::kTCH - 1) / Cfg::kTCH;
        std::vector<int> tabs(7 * (size_t)ng);
        // tensor-core pieces: of the degree-2 prefix [0, K2) and of the degree-4 band [K2, K)
        const std::vector<int> tp2 = tp.on ? tc_pieces(zeros, tp.K2, tp.n_tiles, g0, ng, tc_slots2) : std::vector<int>(ng, 0);
        const std::vector<int> tp4 = tp.on ? tc_pieces(tp.K2, tp.K, tp.n_tiles, g0, ng, tc_slots4) : std::vector<int>(ng, 0);
        std::vector<double> tg(ng);
        std::vector<int64_t> roff(ng);
        int max_nact = 0;
        for (int j = 0; j < ng; ++j) {
            tg[j] = tdim[g0 + j];
            tabs[j] = nact[g0 + j];
            tabs[ng + j] = order[g0 + j];
            tabs[3 * ng + j] = tp.K[g0 + j];                               // kst
            tabs[4 * ng + j] = tp.K[g0 + j] / sb;                          // kb0
            tabs[5 * ng + j] = tp2[j] + tp4[j];                            // nq
            tabs[6 * ng + j] = j > 0 ? tabs[6 * ng + j - 1] + tabs[5 * ng + j - 1] : 0;   // trow0
            max_nact = std::max(max_nact, nact[g0 + j]);
            // lattice: snapshot t reads lag t - i at rev[M - t + i]; otherwise row j of the
            // per-(snapshot, visit) records
            roff[j] = lattice ? (tdim[g0 + j] > 0 ? M - (int64_t)tdim[g0 + j] : M) : (int64_t)j * n_src;
        }
        // work items: (tile, chunk, block) for every block below the chunk's largest
        // n_active (from the first block that holds a visit past some snapshot's
        // tensor-core prefix), longest first.  Every tile of a (chunk, block) costs the
        // same, so the (chunk, block) descriptors are sorted (stable: ties keep chunk, block
        // order) and the kernel expands each into its tiles in tile order.
        std::vector<std::pair<int64_t, int2>> blocks;
        for (int c = 0; c < n_chunks; ++c) {
            const int j0 = c * Cfg::kTCH, j1 = std::min(ng, j0 + Cfg::kTCH);
            int cmax = 0, kbmin = INT_MAX;
            for (int j = j0; j < j1; ++j) {
                cmax = std::max(cmax, nact[g0 + j]);
                kbmin = std::min(kbmin, tp.K[g0 + j] / sb);
            }
            const int nb = (cmax + sb - 1) / sb;
            for (int j = j0; j < j1; ++j) tabs[2 * ng + j] = nb;
            for (int k = kbmin; k < nb; ++k) {
                int64_t cost = 0;
                for (int j = j0; j < j1; ++j)
                    cost += std::max(0, std::min(nact[g0 + j], (k + 1) * sb) - std::max(k * sb, tp.K[g0 + j]));
                blocks.push_back({cost, make_int2(c, k)});
            }
        }
        // tensor-core items: piece p of a snapshot's range [lo, hi) (stages [p S / P,
        // (p + 1) S / P) of its S 16-visit stages) on each tile; degree-2 items (partial rows
        // trow0[j] + p) then degree-4 items (rows trow0[j] + P2 + p), each list longest first
        std::vector<ddk::TcItem> titems;
        size_t n_t2 = 0;
        if (tp.on) {
            auto add_items = [&](const std::vector<int> &lo, const std::vector<int> &hi, const std::vector<int> &pc,
                                 bool deg4) {
                const size_t first = titems.size();
                for (int j = 0; j < ng; ++j) {
                    const int v0 = lo[g0 + j], P = pc[j];
                    const int64_t S = (hi[g0 + j] - v0 + ddk::kTcStage - 1) / ddk::kTcStage;
                    for (int p = 0; p < P; ++p) {
                        const int vb = v0 + (int)(S * p / P) * ddk::kTcStage;
                        const int ve = std::min(hi[g0 + j], v0 + (int)(S * (p + 1) / P) * ddk::kTcStage);
                        const int row = tabs[6 * ng + j] + (deg4 ? tp2[j] : 0) + p;
                        for (int64_t t = 0; t < tp.n_tiles; ++t) titems.push_back({vb, ve, (int)t, row, roff[j], 0, 0});
                    }
                }
                std::stable_sort(titems.begin() + first, titems.end(), [](const ddk::TcItem &a, const ddk::TcItem &b) {
                    return a.v_end - a.v_begin > b.v_end - b.v_begin;
                });
            };
            add_items(zeros, tp.K2, tp2, false);
            n_t2 = titems.size();
            add_items(tp.K2, tp.K, tp4, true);
        }
        std::stable_sort(blocks.begin(), blocks.end(),
                         [](const std::pair<int64_t, int2> &a, const std::pair<int64_t, int2> &b) { return a.first > b.first; });
        std::vector<int2> it(blocks.size());
        for (size_t q = 0; q < blocks.size(); ++q) it[q] = blocks[q].second;

        // the group's tables in one copy: a host image of the device span d_t .. the end of
        // the descriptors (of the tensor-core items, if any)
        {
            char *const d0 = reinterpret_cast<char *>(d_t);
            const size_t span = titems.empty() ? reinterpret_cast<char *>(d_desc + it.size()) - d0
                                               : reinterpret_cast<char *>(d_titems + titems.size()) - d0;
            std::vector<char> img(span);
            std::memcpy(img.data(), tg.data(), ng * sizeof(double));
            std::memcpy(img.data() + (reinterpret_cast<char *>(d_nact) - d0), tabs.data(), 7 * (size_t)ng * sizeof(int));
            std::memcpy(img.data() + (reinterpret_cast<char *>(d_roff) - d0), roff.data(), ng * sizeof(int64_t));
            std::memcpy(img.data() + (reinterpret_cast<char *>(d_desc) - d0), it.data(), it.size() * sizeof(int2));
            if (!titems.empty())
                std::memcpy(img.data() + (reinterpret_cast<char *>(d_titems) - d0), titems.data(),
                            titems.size() * sizeof(ddk::TcItem));
            DD_CUDA_TRY(keep->staging.upload(d0, img.data(), span, stream));
            keep->images.push_back(std::move(img));
        }
        if (max_nact > 0 && !lattice) {
            dim3 cg((unsigned)((max_nact + 127) / 128), (unsigned)ng);
            DD_PROFILED(Cfg::kCoefName, stream,
                        (ddk::coef_kernel<Rec><<<cg, 128, 0, stream>>>(srcT, srcTAU, d_t, d_nact, scan->s, scan->kappa, d_rec, n_src)));
            DD_CUDA_TRY(cudaGetLastError());
        }
        // the tensor-core contraction's fork point: after the coefficients
        SideStream *side = nullptr;
        if (kMixed && !titems.empty()) {
            DD_CUDA_TRY(side_stream(&side));
            DD_CUDA_TRY(cudaEventRecord(side->fork, stream));
        }
        // the contraction on the side stream (after the CUDA-core tile kernel is submitted,
        // so that the latter's CTAs are placed first and the contraction's fill what they leave)
        auto launch_tc = [&]() -> cudaError_t {
            if constexpr (kMixed) {
                if (side) {
                    cudaError_t e = cudaStreamWaitEvent(side->s, side->fork, 0);
                    if (e != cudaSuccess) return e;
                    // DD_FAULT=field_tc_wait (tests): no MMA is issued, so the completion waits
                    // run out and the kernel reports it (dd_field_check)
                    const int withhold = dd::fault_injected("field_tc_wait") ? 1 : 0;
                    // persistent CTAs: as many as are resident at once, at most one per item
                    auto launch = [&](auto deg, const ddk::TcItem *items, size_t n_items, int64_t resident,
                                      const char *name) -> cudaError_t {
                        constexpr int kDeg = decltype(deg)::value;
                        if (n_items == 0) return cudaSuccess;
                        cudaError_t e2 = prepare_tc_kernel<kDeg>();
                        if (e2 != cudaSuccess) return e2;
                        const unsigned n_cta = (unsigned)std::min<int64_t>((int64_t)n_items, resident);
                        DD_PROFILED(name, side->s,
                                    (ddk::field_grid_tc_kernel<kDeg><<<n_cta, ddk::kTcThreads, ddk::TcConst<kDeg>::kSmemBytes, side->s>>>(
                                        ddk::TcScan{grid.W, grid.H, tp.n_tile_cols, srcF, PF, d_tpart, pstride}, nullptr,
                                        d_rec, items, (int)n_items, withhold)));
                        return cudaGetLastError();
                    };
                    if ((e = launch(std::integral_constant<int, 2>(), d_titems, n_t2, tc_slots2, "field_grid_tc")) != cudaSuccess)
                        return e;
                    if ((e = launch(std::integral_constant<int, 4>(), d_titems + n_t2, titems.size() - n_t2, tc_slots4,
                                    "field_grid_tc4")) != cudaSuccess)
                        return e;
                    if ((e = cudaEventRecord(side->join, side->s)) != cudaSuccess) return e;
                }
            }
            return cudaSuccess;
        };
        if (kTcBeforeCore) DD_CUDA_TRY(launch_tc());
        if (!it.empty()) {
            if (grid_tiles) DD_CUDA_TRY((prefer_shared<Cfg, true>()));
            else DD_CUDA_TRY(prefer_shared<Cfg>());
            // one CTA per item, in launches of at most 2^31 - 1 CTAs (the grid's x limit)
            const int64_t n_items = (int64_t)it.size() * n_tiles, kMaxGrid = (int64_t(1) << 31) - 1;
            for (int64_t item0 = 0; item0 < n_items; item0 += kMaxGrid) {
                const unsigned nctas = (unsigned)std::min(kMaxGrid, n_items - item0);
                if constexpr (kMixed) {
                    if (grid_tiles) {
                        DD_PROFILED("field_grid_mixed", stream,
                                    (ddk::field_grid_kernel<GridCfg><<<nctas, Cfg::kThreads, 0, stream>>>(
                                        grid.W, grid.H, n_tc, d_rec, d_roff, d_nact, tp.on ? d_kst : nullptr, d_desc,
                                        n_tiles, item0, ng, sb, d_part, pstride, srcF, PF)));
                        DD_CUDA_TRY(cudaGetLastError());
                        continue;
                    }
                }
                DD_PROFILED(Cfg::kFieldName, stream,
                            (ddk::field_kernel<Cfg><<<nctas, Cfg::kThreads, 0, stream>>>(
                                srcX, srcY, X, Y, n_pts, d_rec, d_roff, d_nact, d_desc, n_tiles, item0, ng, sb, d_part,
                                pstride, srcF, PF)));
                DD_CUDA_TRY(cudaGetLastError());
            }
        }
        if (!kTcBeforeCore) DD_CUDA_TRY(launch_tc());
        if (side) DD_CUDA_TRY(cudaStreamWaitEvent(stream, side->join, 0));
        dim3 rg((unsigned)((n_pts + 1023) / 1024), (unsigned)ng);
        DD_PROFILED("field_reduce", stream,
                    (ddk::reduce_kernel<Part><<<rg, 256, 0, stream>>>(
                        d_part, d_nblk, tp.on ? d_kb0 : nullptr, reinterpret_cast<const Part *>(d_tpart),
                        tp.on ? d_nq : nullptr, d_trow0, d_row, ng, n_pts, pstride, scan->pref, out_dev)));
        DD_CUDA_TRY(cudaGetLastError());
        keep->items.push_back(std::move(it));
        keep->ints.push_back(std::move(tabs));
        keep->reals.push_back(std::move(tg));
        keep->offs.push_back(std::move(roff));
    }
    if (out_copy)
        DD_CUDA_TRY(cudaMemcpyAsync(out, out_dev, (size_t)n_t * n_pts * sizeof(double), cudaMemcpyDeviceToHost, stream));
    DD_CUDA_TRY(dd::workspace_release(ws, stream));
    DD_CUDA_TRY(dd::defer_release(stream, keep, HostTables::release));
    if (dd::host_sync_needed(stream, {pts_kind, out_kind})) DD_CUDA_TRY(cudaStreamSynchronize(stream));
    return DD_OK;
}

}  // namespace

extern "C" dd_status dd_field_at_times(const dd_scan *scan, const double *pts_xy_m, int64_t n_pts,
                                       const double *times_s, int64_t n_t, dd_precision prec,
                                       double *out, void *cuda_stream) {
    dd::clear_error();
    if (!scan) return dd::fail(DD_EINVAL, "dd_field_at_times: NULL scan");
    if (n_pts < 0 || n_t < 0) return dd::fail(DD_EINVAL, "dd_field_at_times: negative size");
    if (prec != DD_FP64 && prec != DD_MIXED) return dd::fail(DD_EINVAL, "dd_field_at_times: unknown precision");
    if (n_pts == 0 || n_t == 0) return DD_OK;
    if (!pts_xy_m || !times_s || !out) return dd::fail(DD_EINVAL, "dd_field_at_times: NULL buffer");
    if (n_t > (int64_t(1) << 24) || n_pts > (int64_t(1) << 31))
        return dd::fail(DD_EINVAL, "dd_field_at_times: too many points or snapshots");
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    std::vector<double> times((size_t)n_t);
    if (dd::is_device_pointer(times_s)) {
        DD_CUDA_TRY(cudaMemcpyAsync(times.data(), times_s, n_t * sizeof(double), cudaMemcpyDeviceToHost, stream));
        DD_CUDA_TRY(cudaStreamSynchronize(stream));
    } else {
        std::memcpy(times.data(), times_s, n_t * sizeof(double));
    }
    for (double t : times)
        if (!std::isfinite(t)) return dd::fail(DD_EINVAL, "dd_field_at_times: non-finite time");
    const ddk::GridDesc list;                                     // an explicit point list
    if (prec == DD_MIXED) return run_field<ddk::CfgMixed>(scan, pts_xy_m, n_pts, list, times, out, stream);
    return run_field<ddk::CfgF64>(scan, pts_xy_m, n_pts, list, times, out, stream);
}

extern "C" dd_status dd_field_on_grid(const dd_scan *scan, double x0_m, double y0_m, double dx_m, double dy_m,
                                      int64_t n_cols, int64_t n_rows, const double *times_s, int64_t n_t,
                                      dd_precision prec, double *out, void *cuda_stream) {
    dd::clear_error();
    if (!scan) return dd::fail(DD_EINVAL, "dd_field_on_grid: NULL scan");
    if (n_cols < 0 || n_rows < 0 || n_t < 0) return dd::fail(DD_EINVAL, "dd_field_on_grid: negative size");
    if (prec != DD_FP64 && prec != DD_MIXED) return dd::fail(DD_EINVAL, "dd_field_on_grid: unknown precision");
    if (!std::isfinite(x0_m) || !std::isfinite(y0_m) || !std::isfinite(dx_m) || !std::isfinite(dy_m))
        return dd::fail(DD_EINVAL, "dd_field_on_grid: grid origin and spacing must be finite");
    if (n_cols == 0 || n_rows == 0 || n_t == 0) return DD_OK;
    if (!times_s || !out) return dd::fail(DD_EINVAL, "dd_field_on_grid: NULL buffer");
    if (n_t > (int64_t(1) << 24) || n_cols > (int64_t(1) << 31) || n_rows > (int64_t(1) << 31) ||
        n_cols * n_rows > (int64_t(1) << 31))
        return dd::fail(DD_EINVAL, "dd_field_on_grid: too many points or snapshots");
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    std::vector<double> times((size_t)n_t);
    if (dd::is_device_pointer(times_s)) {
        DD_CUDA_TRY(cudaMemcpyAsync(times.data(), times_s, n_t * sizeof(double), cudaMemcpyDeviceToHost, stream));
        DD_CUDA_TRY(cudaStreamSynchronize(stream));
    } else {
        std::memcpy(times.data(), times_s, n_t * sizeof(double));
    }
    for (double t : times)
        if (!std::isfinite(t)) return dd::fail(DD_EINVAL, "dd_field_on_grid: non-finite time");
    ddk::GridDesc g;
    g.x0 = x0_m; g.y0 = y0_m; g.dx = dx_m; g.dy = dy_m; g.W = n_cols; g.H = n_rows;
    const int64_t n_pts = n_cols * n_rows;
    if (prec == DD_MIXED) return run_field<ddk::CfgMixed>(scan, nullptr, n_pts, g, times, out, stream);
    return run_field<ddk::CfgF64>(scan, nullptr, n_pts, g, times, out, stream);
}

extern "C" dd_status dd_field_check(void) {
    dd::clear_error();
    DD_CUDA_TRY(cudaDeviceSynchronize());
    int flag = 0;
    DD_CUDA_TRY(cudaMemcpyFromSymbol(&flag, ddk::g_field_tc_timeout, sizeof(int)));
    if (!flag) return DD_OK;
    const int zero = 0;
    DD_CUDA_TRY(cudaMemcpyToSymbol(ddk::g_field_tc_timeout, &zero, sizeof(int)));
    return dd::fail(DD_ETIMEOUT, "dd_field_check: a tensor-core contraction of the grid field gave up waiting for its MMAs");
}

namespace dd {

void tc_prefixes(const dd_scan *scan, double x0, double y0, double dx, double dy, int64_t W, int64_t H, double tdim,
                 int nact, int *K2, int *K) {
    *K2 = *K = 0;
    if (W <= 0 || H <= 0 || nact <= 0) return;
    ddk::GridDesc g;
    g.x0 = x0; g.y0 = y0; g.dx = dx; g.dy = dy; g.W = W; g.H = H;
    const TcPlan tp = plan_tc(scan, g, std::vector<double>{tdim}, std::vector<int>{nact});
    if (!tp.on) return;
    *K2 = tp.K2[0];
    *K = tp.K[0];
}

cudaError_t prepare_field_tc() {
    cudaError_t err = prepare_tc_kernel<2>();
    return err == cudaSuccess ? prepare_tc_kernel<4>() : err;
}

int64_t field_tc_resident(int deg) { return deg == 2 ? tc_resident_ctas<2>() : tc_resident_ctas<4>(); }

cudaError_t launch_field_tc(int deg, const ddk::TcScan *scans, const ddk::RecF32 *rec, const ddk::TcItem *items,
                            int n_items, int n_ctas, cudaStream_t stream) {
    if (n_items <= 0) return cudaSuccess;
    // (no profiling scope: batch plans capture this launch into a CUDA graph)
    const ddk::TcScan none{};
    if (deg == 2)
        ddk::field_grid_tc_kernel<2><<<(unsigned)n_ctas, ddk::kTcThreads, ddk::TcConst<2>::kSmemBytes, stream>>>(
            none, scans, rec, items, n_items, 0);
    else
        ddk::field_grid_tc_kernel<4><<<(unsigned)n_ctas, ddk::kTcThreads, ddk::TcConst<4>::kSmemBytes, stream>>>(
            none, scans, rec, items, n_items, 0);
    return cudaGetLastError();
}

}  // namespace dd

extern "C" dd_status dd_field_grid_split(const dd_scan *scan, double x0_m, double y0_m, double dx_m, double dy_m,
                                         int64_t n_cols, int64_t n_rows, const double *times_s, int64_t n_t,
                                         int64_t *prefix, int64_t *prefix_deg2) {
    dd::clear_error();
    if (!scan) return dd::fail(DD_EINVAL, "dd_field_grid_split: NULL scan");
    if (n_cols < 0 || n_rows < 0 || n_t < 0) return dd::fail(DD_EINVAL, "dd_field_grid_split: negative size");
    if (!std::isfinite(x0_m) || !std::isfinite(y0_m) || !std::isfinite(dx_m) || !std::isfinite(dy_m))
        return dd::fail(DD_EINVAL, "dd_field_grid_split: grid origin and spacing must be finite");
    if (n_t == 0) return DD_OK;
    if (!times_s || !prefix) return dd::fail(DD_EINVAL, "dd_field_grid_split: NULL buffer");
    if (dd::is_device_pointer(times_s) || dd::is_device_pointer(prefix) || (prefix_deg2 && dd::is_device_pointer(prefix_deg2)))
        return dd::fail(DD_EINVAL, "dd_field_grid_split: times and prefix are host arrays");
    std::vector<double> times(times_s, times_s + n_t);
    for (double t : times)
        if (!std::isfinite(t)) return dd::fail(DD_EINVAL, "dd_field_grid_split: non-finite time");
    std::vector<int> order, nact;
    std::vector<double> tdim;
    int64_t M = 0;
    snapshot_dims(scan, times, order, tdim, nact, M);
    ddk::GridDesc g;
    g.x0 = x0_m; g.y0 = y0_m; g.dx = dx_m; g.dy = dy_m; g.W = n_cols; g.H = n_rows;
    const TcPlan tp = n_cols > 0 && n_rows > 0 ? plan_tc(scan, g, tdim, nact) : TcPlan();
    for (int k = 0; k < (int)n_t; ++k) {
        prefix[order[k]] = tp.on ? tp.K[k] : 0;
        if (prefix_deg2) prefix_deg2[order[k]] = tp.on ? tp.K2[k] : 0;
    }
    return DD_OK;
}
