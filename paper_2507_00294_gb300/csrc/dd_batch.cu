// dd_batch.cu -- many independent scans in one persistent, graph-captured launch.
//
// The paper balances its CPU tasks over subsets of the probe positions (Sec. 3); on the
// GPU the same idea spans scans: every (scan, point tile, visit block) is one work item,
// the items of all scans are sorted by cost (longest first) and a persistent grid of
// CTAs claims them with an atomic counter, so scans of very different size share the
// machine without a tail.  Each scan is evaluated at one snapshot time.  The launch
// sequence (counter reset, point scaling, coefficients, persistent field kernel,
// fixed-order reduce) is captured once into a CUDA graph and replayed.
//
// A tile-shape autotuner picks, per (GPU, precision, batch size), the fastest of
// several kernel variants that share the same work list (same tile size, different
// threads x points-per-thread) by timing each once; choices are cached in-process and,
// when DD_TUNE_CACHE names a file, in that JSON file.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <type_traits>
#include <vector>

#include "dd_batch_grid.cuh"
#include "dd_coef.cuh"
#include "dd_e1.cuh"
#include "dd_field_impl.cuh"
#include "dd_field_tc.cuh"
#include "dd_internal.h"

namespace ddk {

struct BScan {
    const double *src;          // X | Y | T | TAU of the scan, n each (dimensionless)
    const float4 *srcF;         // X, Y of the scan's visits as float-float pairs
    int64_t n;                  // visits
    int64_t pt_off, n_pts;      // points of the scan in the global arrays
    int64_t rec_off;            // first record of the scan
    int64_t part_off;           // first partial of the scan (nblk * n_pts of them)
    double s, kappa, pref, tdim, inv_pitch;
    int nact, nblk;
    // a grid of points (dd_batch_create_grid): point r W + c at (x0 + c dx, y0 + r dy) [m];
    // W = 0 for an explicit point list
    double gx0, gy0, gdx, gdy;
    int64_t gW, gH, n_tc;
    // grid plans in FP32-mixed: visits [0, k_tc) are summed by the tensor-core contraction
    // into nq_tc FP32 rows of t_stride points at t_off (dd_field_tc.cuh); the CUDA-core tile
    // kernel takes visits [k_tc, nact), in the blocks [blk0, nblk)
    int k_tc, nq_tc, blk0;
    int64_t t_off, t_stride;
};

__device__ __forceinline__ int find_segment(const int64_t *__restrict__ offs, int n, int64_t g) {
    int lo = 0, hi = n - 1;                     // largest k with offs[k] <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Points in pitch units: FP64 X, Y and float-float F (x_hi, x_lo, y_hi, y_lo).
__global__ void batch_prep_kernel(const BScan *__restrict__ sc, const int64_t *__restrict__ pt_offs, int n_scans,
                                  const double *__restrict__ xy, int64_t total, double *__restrict__ X,
                                  double *__restrict__ Y, float4 *__restrict__ F) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const BScan &S = sc[find_segment(pt_offs, n_scans, g)];
    const double ip = S.inv_pitch;
    double xs, ys;
    if (S.gW > 0) {                     // grid point: one product and one sum, no fused multiply-add
        const int64_t p = g - S.pt_off, r = p / S.gW, c = p - r * S.gW;
        xs = __dadd_rn(__dmul_rn((double)c, S.gdx), S.gx0);
        ys = __dadd_rn(__dmul_rn((double)r, S.gdy), S.gy0);
    } else {
        xs = xy[2 * g];
        ys = xy[2 * g + 1];
    }
    const double x = xs * ip, y = ys * ip;
    X[g] = x;
    Y[g] = y;
    const float xh = (float)x, yh = (float)y;
    F[g] = make_float4(xh, (float)(x - (double)xh), yh, (float)(y - (double)yh));
}

template <typename Rec>
__global__ void batch_coef_kernel(const BScan *__restrict__ sc, const int64_t *__restrict__ rec_offs, int n_scans,
                                  int64_t total, Rec *__restrict__ rec) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const BScan &S = sc[find_segment(rec_offs, n_scans, g)];
    const int64_t i = g - S.rec_off;
    if (i >= S.nact) return;
    double q1, dq, r, ell;
    pair_geometry<RecTraits<Rec>::kFP64Ell>(S.tdim - S.src[2 * S.n + i], S.src[3 * S.n + i], S.s, S.kappa, q1, dq, r, ell);
    Rec out;
    RecTraits<Rec>::fill(out, q1, dq, r, ell);
    rec[g] = out;
}

// Resident CTAs per SM each variant is compiled for (register cap 65536 / (threads x
// blocks)); 0 leaves the register count to the compiler.
template <typename Cfg>
struct BatchMinBlocks { static constexpr int value = 0; };
struct CfgMixed64x12;
template <> struct BatchMinBlocks<CfgMixed64x12> { static constexpr int value = 12; };
template <> struct BatchMinBlocks<CfgMixed> { static constexpr int value = 9; };

// Persistent CTAs: claim item indices from *counter until the list is exhausted.
template <typename Cfg>
__global__ void __launch_bounds__(Cfg::kThreads, BatchMinBlocks<Cfg>::value)
batch_field_kernel(const BScan *__restrict__ sc, const int4 *__restrict__ items, int n_items,
                   unsigned *__restrict__ counter, const double *__restrict__ X, const double *__restrict__ Y,
                   const float4 *__restrict__ F, const typename Cfg::Rec *__restrict__ rec, int sb,
                   double *__restrict__ partial) {
    constexpr bool kMixed = std::is_same<typename Cfg::Real, float>::value;
    using Smem = typename std::conditional<kMixed, TileSmemMixed<Cfg, 1>, TileSmem<Cfg, 1>>::type;
    __shared__ Smem sm;
    __shared__ int s_item;
    constexpr int TILE = Cfg::kThreads * Cfg::kPPT;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const int4 item = items[it];
        const BScan &S = sc[item.x];
        const int na[1] = {S.nact};
        const typename Cfg::Rec *rows[1] = {rec + S.rec_off};
        const int s_begin = item.z * sb;
        const int s_end = min(s_begin + sb, S.nact);
        if constexpr (kMixed)
            field_tile_mixed<Cfg, 1>(sm, S.srcF, F + S.pt_off, S.n_pts,
                                     (int64_t)item.y * TILE, rows, na, 1, s_begin, s_end,
                                     partial + S.part_off + (int64_t)item.z * S.n_pts, S.n_pts);
        else
            field_tile<Cfg, 1>(sm, S.src, S.src + S.n, X + S.pt_off, Y + S.pt_off, S.n_pts, (int64_t)item.y * TILE,
                               rows, na, 1, s_begin, s_end, partial + S.part_off + (int64_t)item.z * S.n_pts,
                               S.n_pts);
    }
}

// Persistent CTAs over grid tiles of 32 x 32 points (FP32-mixed): item (scan, tile, block).
__global__ void __launch_bounds__(kBgThreads, 8)
batch_grid_kernel(const BScan *__restrict__ sc, const int4 *__restrict__ items, int n_items,
                  unsigned *__restrict__ counter, const float4 *__restrict__ F, const RecF32 *__restrict__ rec,
                  int sb, double *__restrict__ partial) {
    __shared__ BGridSmem sm;
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const int4 item = items[it];
        const BScan &S = sc[item.x];
        const int s_begin = max(item.z * sb, S.k_tc);
        const int s_end = min(item.z * sb + sb, S.nact);
        field_tile_bgrid(sm, S.srcF, F + S.pt_off, S.gW, S.gH, item.y % S.n_tc, item.y / S.n_tc,
                         rec + S.rec_off, s_begin, s_end, partial + S.part_off + (int64_t)item.z * S.n_pts);
    }
}

__global__ void batch_reduce_kernel(const BScan *__restrict__ sc, const int64_t *__restrict__ pt_offs, int n_scans,
                                    int64_t total, const double *__restrict__ partial, const float *__restrict__ tpart,
                                    bool mixed_grid, double *__restrict__ out) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const BScan &S = sc[find_segment(pt_offs, n_scans, g)];
    const int64_t p = g - S.pt_off;
    // the tensor-core rows first, then the CUDA-core blocks from the first one past k_tc.
    // Grid plans in FP32-mixed hold FP32 sums (the block sums exactly, in FP64 storage):
    // a compensated FP32 sum (FP64 arithmetic is 64 times slower on this part); the others
    // sum in FP64.
    if (S.nq_tc > 0 || mixed_grid) {
        BlockSum<float> acc;
        for (int q = 0; q < S.nq_tc; ++q) acc.add(tpart[S.t_off + (int64_t)q * S.t_stride + p]);
        for (int b = S.blk0; b < S.nblk; ++b) acc.add((float)partial[S.part_off + (int64_t)b * S.n_pts + p]);
        out[g] = S.pref * acc.value();
    } else {
        double acc = 0.0;
        for (int b = 0; b < S.nblk; ++b) acc += partial[S.part_off + (int64_t)b * S.n_pts + p];
        out[g] = S.pref * acc;
    }
}

// Kernel variants with the same 512-point tile (so they share one work list).
struct CfgMixed256 : CfgMixed {
    static constexpr int kThreads = 256, kPPT = 2, kSTILE = 64;
};
struct CfgMixed64 : CfgMixed {
    static constexpr int kThreads = 64, kPPT = 8, kSTILE = 64;
};
// the same, held to 80 registers (12 CTAs per SM, a few spilled values) instead of 96
struct CfgMixed64x12 : CfgMixed64 {};
struct CfgF64x256 : CfgF64 {
    static constexpr int kThreads = 256, kPPT = 1;
};

}  // namespace ddk

// =================================================================== plan object
struct dd_batch {
    int device = 0;
    dd_precision prec = DD_MIXED;
    int n_scans = 0;
    int64_t total_pts = 0, total_rec = 0, total_part = 0, pairs = 0;
    int n_items = 0, sb = 512;
    int variant = 0;
    std::vector<int> grid;              // persistent grid size per variant
    void *ws = nullptr;                 // device tables and buffers (cudaMalloc)
    ddk::BScan *d_sc = nullptr;
    int64_t *d_pt_offs = nullptr, *d_rec_offs = nullptr;
    int4 *d_items = nullptr;
    unsigned *d_counter = nullptr;
    double *d_X = nullptr, *d_Y = nullptr, *d_part = nullptr;
    float4 *d_F = nullptr;
    void *d_rec = nullptr;
    // tensor-core contraction of grid plans: scan table, work items (degree 2, then
    // degree 4), their CTA counts and FP32 partial rows
    ddk::TcScan *d_tcs = nullptr;
    ddk::TcItem *d_titems = nullptr;
    int n_t2 = 0, n_t4 = 0, cta_t2 = 0, cta_t4 = 0;
    float *d_tpart = nullptr;
    double *d_pts = nullptr, *d_out = nullptr;   // staging for host buffers
    cudaStream_t cap = nullptr;
    cudaStream_t side = nullptr;        // the graph's second branch (coefficients, contraction)
    cudaEvent_t ev_fork = nullptr, ev_coef = nullptr, ev_join = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool on_grid = false;               // points formed from per-scan grids (no point buffer)
    bool grid_tiles = false;            // ... and evaluated by the grid tile kernel (FP32-mixed)
    const double *g_pts = nullptr;
    double *g_out = nullptr;
    int g_variant = -1;
    std::string tune_key;
};

namespace {

constexpr int kTile = 512;
constexpr int kVariants = 4;

const char *variant_name(dd_precision prec, int v) {
    static const char *mixed[kVariants] = {"batch_field_mixed_128x4", "batch_field_mixed_256x2", "batch_field_mixed_64x8",
                                           "batch_field_mixed_64x8_r80"};
    static const char *f64[kVariants] = {"batch_field_fp64_128x4", "batch_field_fp64_256x2", "batch_field_fp64_64x8",
                                         "batch_field_fp64_64x8"};
    return prec == DD_MIXED ? mixed[v] : f64[v];
}

template <typename Cfg>
int persistent_grid() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ddk::batch_field_kernel<Cfg>, Cfg::kThreads, 0);
    return std::max(1, sms * std::max(1, per));
}

template <typename Cfg>
void launch_field(dd_batch *b, int grid, cudaStream_t st) {
    ddk::batch_field_kernel<Cfg><<<grid, Cfg::kThreads, 0, st>>>(
        b->d_sc, b->d_items, b->n_items, b->d_counter, b->d_X, b->d_Y, b->d_F,
        (const typename Cfg::Rec *)b->d_rec, b->sb, b->d_part);
}

// Enqueue the whole batch evaluation on `st` (used for capture and for tuning).
dd_status enqueue(dd_batch *b, const double *pts, double *out, int variant, cudaStream_t st) {
    const unsigned nb_pts = (unsigned)((b->total_pts + 255) / 256);
    // two branches: the points on `st`, the coefficient records beside them on `side`
    // (they only read the scans); with the tensor-core contraction, it follows the records
    // on `side` while the grid tiles run on `st`; both join before the reduce
    DD_CUDA_TRY(cudaEventRecord(b->ev_fork, st));
    DD_CUDA_TRY(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
    DD_CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), st));
    ddk::batch_prep_kernel<<<nb_pts, 256, 0, st>>>(b->d_sc, b->d_pt_offs, b->n_scans, pts, b->total_pts, b->d_X, b->d_Y, b->d_F);
    if (b->total_rec > 0) {
        const unsigned nb = (unsigned)((b->total_rec + 127) / 128);
        if (b->prec == DD_MIXED)
            ddk::batch_coef_kernel<ddk::RecF32><<<nb, 128, 0, b->side>>>(b->d_sc, b->d_rec_offs, b->n_scans,
                                                                       b->total_rec, (ddk::RecF32 *)b->d_rec);
        else
            ddk::batch_coef_kernel<ddk::RecF64><<<nb, 128, 0, b->side>>>(b->d_sc, b->d_rec_offs, b->n_scans,
                                                                       b->total_rec, (ddk::RecF64 *)b->d_rec);
    }
    DD_CUDA_TRY(cudaEventRecord(b->ev_coef, b->side));
    DD_CUDA_TRY(cudaStreamWaitEvent(st, b->ev_coef, 0));
    if (b->n_t2 + b->n_t4 > 0) {
        // the older visits of the larger grids on the tensor cores (after the points)
        DD_CUDA_TRY(cudaEventRecord(b->ev_fork, st));
        DD_CUDA_TRY(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
        DD_CUDA_TRY(dd::launch_field_tc(2, b->d_tcs, (const ddk::RecF32 *)b->d_rec, b->d_titems, b->n_t2, b->cta_t2,
                                        b->side));
        DD_CUDA_TRY(dd::launch_field_tc(4, b->d_tcs, (const ddk::RecF32 *)b->d_rec, b->d_titems + b->n_t2, b->n_t4,
                                        b->cta_t4, b->side));
    }
    DD_CUDA_TRY(cudaEventRecord(b->ev_join, b->side));
    if (b->n_items > 0 && b->grid_tiles) {
        ddk::batch_grid_kernel<<<b->grid[0], ddk::kBgThreads, 0, st>>>(b->d_sc, b->d_items, b->n_items, b->d_counter,
                                                                      b->d_F, (const ddk::RecF32 *)b->d_rec, b->sb,
                                                                      b->d_part);
    } else if (b->n_items > 0) {
        const int g = b->grid[variant];
        if (b->prec == DD_MIXED) {
            if (variant == 0) launch_field<ddk::CfgMixed>(b, g, st);
            else if (variant == 1) launch_field<ddk::CfgMixed256>(b, g, st);
            else if (variant == 2) launch_field<ddk::CfgMixed64>(b, g, st);
            else launch_field<ddk::CfgMixed64x12>(b, g, st);
        } else {
            if (variant == 0) launch_field<ddk::CfgF64>(b, g, st);   // 128 x 2 (256-point tile)
            else if (variant == 1) launch_field<ddk::CfgF64x256>(b, g, st);
            else launch_field<ddk::CfgF64>(b, g, st);
        }
    }
    DD_CUDA_TRY(cudaStreamWaitEvent(st, b->ev_join, 0));
    ddk::batch_reduce_kernel<<<nb_pts, 256, 0, st>>>(b->d_sc, b->d_pt_offs, b->n_scans, b->total_pts, b->d_part,
                                                     b->d_tpart, b->grid_tiles, out);
    DD_CUDA_TRY(cudaGetLastError());
    return DD_OK;
}

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;

void tune_cache_load() {
    static bool loaded = false;
    if (loaded) return;
    loaded = true;
    const char *path = std::getenv("DD_TUNE_CACHE");
    if (!path) return;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {      // one "key": variant pair per line
        const size_t a = line.find('"'), b = line.find('"', a + 1), c = line.find(':', b);
        if (a == std::string::npos || b == std::string::npos || c == std::string::npos) continue;
        g_tune[line.substr(a + 1, b - a - 1)] = std::atoi(line.c_str() + c + 1);
    }
}

void tune_cache_store() {
    const char *path = std::getenv("DD_TUNE_CACHE");
    if (!path) return;
    std::ofstream f(path);
    f << "{\n";
    size_t k = 0;
    for (auto &kv : g_tune) f << "  \"" << kv.first << "\": " << kv.second << (++k < g_tune.size() ? ",\n" : "\n");
    f << "}\n";
}

int grid_kernel_ctas() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(ddk::batch_grid_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        cudaGetLastError();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ddk::batch_grid_kernel, ddk::kBgThreads, 0);
    return std::max(1, sms * std::max(1, std::min(per, 8)));
}

// Plan of a batch: explicit points (grid_xy == NULL, pt_offsets given) or per-scan grids
// (grid_xy: x0, y0, dx, dy per scan [m]; grid_wh: columns, rows per scan).
dd_status create_plan(const dd_scan *const *scans, int32_t n_scans, const int64_t *pt_offsets_in,
                      const double *grid_xy, const int64_t *grid_wh, const double *times_s, dd_precision prec,
                      dd_batch **out) {
    std::vector<int64_t> offs_grid;
    const int64_t *pt_offsets = pt_offsets_in;
    if (grid_xy) {
        offs_grid.assign((size_t)n_scans + 1, 0);
        for (int k = 0; k < n_scans; ++k) {
            const int64_t W = grid_wh[2 * k], H = grid_wh[2 * k + 1];
            if (W < 0 || H < 0 || W > (int64_t(1) << 31) || H > (int64_t(1) << 31))
                return dd::fail(DD_EINVAL, "dd_batch_create_grid: grid sizes must be in [0, 2^31]");
            for (int q = 0; q < 4; ++q)
                if (!std::isfinite(grid_xy[4 * k + q]))
                    return dd::fail(DD_EINVAL, "dd_batch_create_grid: grid origin and spacing must be finite");
            offs_grid[(size_t)k + 1] = offs_grid[(size_t)k] + W * H;
            if (offs_grid[(size_t)k + 1] > (int64_t(1) << 31))
                return dd::fail(DD_EINVAL, "dd_batch_create_grid: more than 2^31 points");
        }
        pt_offsets = offs_grid.data();
    }
    if (pt_offsets[0] != 0) return dd::fail(DD_EINVAL, "dd_batch_create: pt_offsets[0] must be 0");
    for (int k = 0; k < n_scans; ++k) {
        if (!scans[k]) return dd::fail(DD_EINVAL, "dd_batch_create: NULL scan");
        if (pt_offsets[k + 1] < pt_offsets[k]) return dd::fail(DD_EINVAL, "dd_batch_create: pt_offsets must not decrease");
        if (!std::isfinite(times_s[k])) return dd::fail(DD_EINVAL, "dd_batch_create: non-finite time");
    }
    std::unique_ptr<dd_batch> b(new dd_batch());
    b->prec = prec;
    b->n_scans = n_scans;
    b->on_grid = grid_xy != nullptr;
    b->grid_tiles = b->on_grid && prec == DD_MIXED;
    DD_CUDA_TRY(cudaGetDevice(&b->device));
    const int tile = prec == DD_MIXED ? kTile : ddk::CfgF64::kThreads * ddk::CfgF64::kPPT;
    std::vector<ddk::BScan> sc((size_t)n_scans);
    std::vector<int64_t> pt_offs((size_t)n_scans), rec_offs((size_t)n_scans);
    std::vector<std::pair<int64_t, int4>> items;
    // tensor-core work items (FP32-mixed grid plans): degree 2 and degree 4, each at most
    // kTcMaxItemStages stages long (the FP32 accumulation's error budget), times the tiles
    std::vector<std::pair<int64_t, ddk::TcItem>> titems2, titems4;
    std::vector<ddk::TcScan> tcs((size_t)n_scans, ddk::TcScan{});
    int64_t tpart_total = 0;
    int64_t rec = 0, part = 0;
    for (int k = 0; k < n_scans; ++k) {
        const dd_scan *s = scans[k];
        dd_status st = DD_OK;
        const double *src = dd::device_sources(s, nullptr, &st);
        if (!src) return st;
        dd::scan_shared(s);                  // the plan may run on any stream
        ddk::BScan &S = sc[(size_t)k];
        S.src = src;
        S.srcF = dd::device_sources_ff(s, nullptr, &st);
        S.n = s->n;
        S.pt_off = pt_offsets[k];
        S.n_pts = pt_offsets[k + 1] - pt_offsets[k];
        S.s = s->s; S.kappa = s->kappa; S.pref = s->pref; S.inv_pitch = 1.0 / s->pitch;
        S.tdim = times_s[k] / s->dwell;
        S.nact = (int)(std::lower_bound(s->T.begin(), s->T.end(), S.tdim) - s->T.begin());
        if (S.n_pts == 0) S.nact = 0;
        S.nblk = (S.nact + b->sb - 1) / b->sb;
        S.rec_off = rec;
        S.part_off = part;
        S.gx0 = S.gy0 = S.gdx = S.gdy = 0.0;
        S.gW = S.gH = S.n_tc = 0;
        if (grid_xy) {
            S.gx0 = grid_xy[4 * k]; S.gy0 = grid_xy[4 * k + 1];
            S.gdx = grid_xy[4 * k + 2]; S.gdy = grid_xy[4 * k + 3];
            S.gW = grid_wh[2 * k]; S.gH = grid_wh[2 * k + 1];
            S.n_tc = (S.gW + ddk::kBgCols - 1) / ddk::kBgCols;
        }
        S.k_tc = S.nq_tc = 0;
        S.t_off = S.t_stride = 0;
        if (b->grid_tiles && S.nact > 0) {
            int K2 = 0, K = 0;
            dd::tc_prefixes(s, S.gx0, S.gy0, S.gdx, S.gdy, S.gW, S.gH, S.tdim, S.nact, &K2, &K);
            if (K > 0) {
                const int64_t n_tcols = (S.gW + ddk::kTcTile - 1) / ddk::kTcTile;
                const int n_ttiles = (int)(n_tcols * ((S.gH + ddk::kTcTile - 1) / ddk::kTcTile));
                constexpr int kPiece = ddk::kTcMaxItemStages * ddk::kTcStage;
                int row = 0;
                auto pieces = [&](int lo, int hi, std::vector<std::pair<int64_t, ddk::TcItem>> &list) {
                    for (int vb = lo; vb < hi; vb += kPiece, ++row) {
                        const int ve = std::min(hi, vb + kPiece);
                        for (int t = 0; t < n_ttiles; ++t)
                            list.push_back({(int64_t)(ve - vb), ddk::TcItem{vb, ve, t, row, S.rec_off, k, 0}});
                    }
                };
                pieces(0, K2, titems2);
                pieces(K2, K, titems4);
                S.k_tc = K;
                S.nq_tc = row;
                S.t_stride = (S.n_pts + 3) / 4 * 4;             // 16-byte aligned rows
                S.t_off = tpart_total;
                tpart_total += (int64_t)row * S.t_stride;
                // the points and partial rows are filled in once the plan's buffers exist
                tcs[(size_t)k] = ddk::TcScan{S.gW, S.gH, n_tcols, S.srcF, nullptr, nullptr, S.t_stride};
            }
        }
        S.blk0 = S.k_tc >= S.nact ? S.nblk : S.k_tc / b->sb;
        pt_offs[(size_t)k] = S.pt_off;
        rec_offs[(size_t)k] = rec;
        rec += S.nact;
        part += (int64_t)S.nblk * S.n_pts;
        // grid tiles of 32 x 32 points (items cost by their valid points), else point tiles
        const int64_t n_tr = b->grid_tiles ? (S.gH + ddk::kBgRows - 1) / ddk::kBgRows : 0;
        const int64_t tiles = S.n_pts == 0 ? 0 : b->grid_tiles ? S.n_tc * n_tr : (S.n_pts + tile - 1) / tile;
        for (int blk = S.blk0; blk < S.nblk; ++blk) {
            const int64_t nsrc = std::min<int64_t>(S.nact, (int64_t)(blk + 1) * b->sb) -
                                 std::max<int64_t>((int64_t)blk * b->sb, S.k_tc);
            for (int64_t t = 0; t < tiles; ++t) {
                int64_t npt;
                if (b->grid_tiles) {
                    const int64_t tc = t % S.n_tc, tr = t / S.n_tc;
                    npt = std::min<int64_t>(ddk::kBgCols, S.gW - tc * ddk::kBgCols) *
                          std::min<int64_t>(ddk::kBgRows, S.gH - tr * ddk::kBgRows);
                } else {
                    npt = std::min<int64_t>(tile, S.n_pts - t * tile);
                }
                items.push_back({nsrc * npt, make_int4(k, (int)t, blk, 0)});
            }
        }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<int64_t, int4> &x, const std::pair<int64_t, int4> &y) { return x.first > y.first; });
    auto longest_first = [](const std::pair<int64_t, ddk::TcItem> &x, const std::pair<int64_t, ddk::TcItem> &y) {
        return x.first > y.first;
    };
    std::stable_sort(titems2.begin(), titems2.end(), longest_first);
    std::stable_sort(titems4.begin(), titems4.end(), longest_first);
    b->n_t2 = (int)titems2.size();
    b->n_t4 = (int)titems4.size();
    b->total_pts = pt_offsets[n_scans];
    b->total_rec = rec;
    b->total_part = part;
    b->n_items = (int)items.size();
    const size_t rec_size = prec == DD_MIXED ? sizeof(ddk::RecF32) : sizeof(ddk::RecF64);
    size_t bytes = 0;
    auto add = [&](size_t x) { size_t o = (bytes + 255) & ~size_t(255); bytes = o + x; return o; };
    const size_t o_sc = add(sc.size() * sizeof(ddk::BScan));
    const size_t o_pt = add(pt_offs.size() * sizeof(int64_t));
    const size_t o_ro = add(rec_offs.size() * sizeof(int64_t));
    const size_t o_it = add(std::max<size_t>(1, items.size()) * sizeof(int4));
    const size_t o_ct = add(sizeof(unsigned));
    const size_t o_x = add(2 * (size_t)std::max<int64_t>(1, b->total_pts) * sizeof(double));
    const size_t o_f = add((size_t)std::max<int64_t>(1, b->total_pts) * sizeof(float4));
    const size_t o_rec = add((size_t)std::max<int64_t>(1, rec) * rec_size);
    const size_t o_part = add((size_t)std::max<int64_t>(1, part) * sizeof(double));
    const size_t o_tcs = add(tcs.size() * sizeof(ddk::TcScan));
    const size_t o_ti = add((size_t)std::max(1, b->n_t2 + b->n_t4) * sizeof(ddk::TcItem));
    const size_t o_tp = add((size_t)std::max<int64_t>(4, tpart_total) * sizeof(float));
    cudaError_t err = cudaMalloc(&b->ws, bytes);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return dd::fail(DD_ENOMEM, std::string("dd_batch_create: cudaMalloc: ") + cudaGetErrorString(err));
    }
    char *base = (char *)b->ws;
    b->d_sc = (ddk::BScan *)(base + o_sc);
    b->d_pt_offs = (int64_t *)(base + o_pt);
    b->d_rec_offs = (int64_t *)(base + o_ro);
    b->d_items = (int4 *)(base + o_it);
    b->d_counter = (unsigned *)(base + o_ct);
    b->d_X = (double *)(base + o_x);
    b->d_Y = b->d_X + std::max<int64_t>(1, b->total_pts);
    b->d_F = (float4 *)(base + o_f);
    b->d_rec = base + o_rec;
    b->d_part = (double *)(base + o_part);
    b->d_tcs = (ddk::TcScan *)(base + o_tcs);
    b->d_titems = (ddk::TcItem *)(base + o_ti);
    b->d_tpart = (float *)(base + o_tp);
    if (b->n_t2 + b->n_t4 > 0) {
        for (int k = 0; k < n_scans; ++k) {
            if (sc[(size_t)k].nq_tc == 0) continue;
            tcs[(size_t)k].ptsF = b->d_F + sc[(size_t)k].pt_off;
            tcs[(size_t)k].partial = b->d_tpart + sc[(size_t)k].t_off;
        }
        std::vector<ddk::TcItem> ti;
        ti.reserve(titems2.size() + titems4.size());
        for (auto &x : titems2) ti.push_back(x.second);
        for (auto &x : titems4) ti.push_back(x.second);
        DD_CUDA_TRY(cudaMemcpy(b->d_tcs, tcs.data(), tcs.size() * sizeof(ddk::TcScan), cudaMemcpyHostToDevice));
        DD_CUDA_TRY(cudaMemcpy(b->d_titems, ti.data(), ti.size() * sizeof(ddk::TcItem), cudaMemcpyHostToDevice));
        DD_CUDA_TRY(dd::prepare_field_tc());
        b->cta_t2 = (int)std::min<int64_t>(b->n_t2, std::max<int64_t>(1, dd::field_tc_resident(2)));
        b->cta_t4 = (int)std::min<int64_t>(b->n_t4, std::max<int64_t>(1, dd::field_tc_resident(4)));
    }
    std::vector<int4> it(items.size());
    for (size_t k = 0; k < items.size(); ++k) it[k] = items[k].second;
    DD_CUDA_TRY(cudaMemcpy(b->d_sc, sc.data(), sc.size() * sizeof(ddk::BScan), cudaMemcpyHostToDevice));
    DD_CUDA_TRY(cudaMemcpy(b->d_pt_offs, pt_offs.data(), pt_offs.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    DD_CUDA_TRY(cudaMemcpy(b->d_rec_offs, rec_offs.data(), rec_offs.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    if (!it.empty()) DD_CUDA_TRY(cudaMemcpy(b->d_items, it.data(), it.size() * sizeof(int4), cudaMemcpyHostToDevice));
    DD_CUDA_TRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    DD_CUDA_TRY(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
    DD_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    DD_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_coef, cudaEventDisableTiming));
    DD_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
    if (b->grid_tiles)
        b->grid = {grid_kernel_ctas(), grid_kernel_ctas(), grid_kernel_ctas(), grid_kernel_ctas()};
    else if (prec == DD_MIXED)
        b->grid = {persistent_grid<ddk::CfgMixed>(), persistent_grid<ddk::CfgMixed256>(), persistent_grid<ddk::CfgMixed64>(),
                   persistent_grid<ddk::CfgMixed64x12>()};
    else
        b->grid = {persistent_grid<ddk::CfgF64>(), persistent_grid<ddk::CfgF64x256>(), persistent_grid<ddk::CfgF64>(),
                   persistent_grid<ddk::CfgF64>()};
    // tuning key: device name, precision and a log2 bucket of the pair count
    cudaDeviceProp prop;
    DD_CUDA_TRY(cudaGetDeviceProperties(&prop, b->device));
    int64_t pairs = 0;
    for (auto &S : sc) pairs += (int64_t)S.nact * S.n_pts;
    b->pairs = pairs;
    int bucket = 0;
    while ((int64_t(1) << bucket) < pairs && bucket < 62) ++bucket;
    std::ostringstream key;
    key << prop.name << "/sm" << prop.major << prop.minor << "/" << (prec == DD_MIXED ? "mixed" : "fp64")
        << (b->on_grid ? "/grid" : "") << "/2^" << bucket;
    b->tune_key = key.str();
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_cache_load();
        auto f = g_tune.find(b->tune_key);
        b->variant = f != g_tune.end() ? std::min(std::max(f->second, 0), kVariants - 1) : 0;
    }
    if (b->grid_tiles) b->variant = 0;                  // one kernel for grid tiles
    *out = b.release();
    return DD_OK;
}

}  // namespace

extern "C" {

dd_status dd_batch_create(const dd_scan *const *scans, int32_t n_scans, const int64_t *pt_offsets,
                          const double *times_s, dd_precision prec, dd_batch **out) {
    dd::clear_error();
    if (!scans || !pt_offsets || !times_s || !out || n_scans < 1)
        return dd::fail(DD_EINVAL, "dd_batch_create: NULL argument or no scans");
    if (prec != DD_FP64 && prec != DD_MIXED) return dd::fail(DD_EINVAL, "dd_batch_create: unknown precision");
    return create_plan(scans, n_scans, pt_offsets, nullptr, nullptr, times_s, prec, out);
}

dd_status dd_batch_create_grid(const dd_scan *const *scans, int32_t n_scans, const double *grid_xy,
                               const int64_t *grid_wh, const double *times_s, dd_precision prec, dd_batch **out) {
    dd::clear_error();
    if (!scans || !grid_xy || !grid_wh || !times_s || !out || n_scans < 1)
        return dd::fail(DD_EINVAL, "dd_batch_create_grid: NULL argument or no scans");
    if (prec != DD_FP64 && prec != DD_MIXED) return dd::fail(DD_EINVAL, "dd_batch_create_grid: unknown precision");
    return create_plan(scans, n_scans, nullptr, grid_xy, grid_wh, times_s, prec, out);
}

dd_status dd_batch_tune(dd_batch *b, const double *pts_xy_m, int32_t *chosen) {
    dd::clear_error();
    if (!b || (!pts_xy_m && !b->on_grid)) return dd::fail(DD_EINVAL, "dd_batch_tune: NULL argument");
    if (b->on_grid) pts_xy_m = nullptr;                  // grid plans form their points
    else if (!dd::is_device_pointer(pts_xy_m))
        return dd::fail(DD_EINVAL, "dd_batch_tune: points must be on the device");
    double *tmp = nullptr;
    DD_CUDA_TRY(cudaMalloc(&tmp, (size_t)std::max<int64_t>(1, b->total_pts) * sizeof(double)));
    cudaEvent_t e0, e1;
    DD_CUDA_TRY(cudaEventCreate(&e0));
    DD_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_v = 0;
    const int nv = b->grid_tiles ? 1 : b->prec == DD_MIXED ? kVariants : 2;
    for (int v = 0; v < nv; ++v) {
        dd_status st = enqueue(b, pts_xy_m, tmp, v, b->cap);           // warm
        if (st != DD_OK) { cudaFree(tmp); return st; }
        cudaEventRecord(e0, b->cap);
        enqueue(b, pts_xy_m, tmp, v, b->cap);
        cudaEventRecord(e1, b->cap);
        DD_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_v = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(tmp);
    b->variant = best_v;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[b->tune_key] = best_v;
        tune_cache_store();
    }
    if (chosen) *chosen = best_v;
    return DD_OK;
}

dd_status dd_batch_run(dd_batch *b, const double *pts_xy_m, double *out, void *cuda_stream) {
    dd::clear_error();
    if (!b || (!pts_xy_m && !b->on_grid) || !out) return dd::fail(DD_EINVAL, "dd_batch_run: NULL argument");
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    if (b->on_grid) pts_xy_m = nullptr;                  // grid plans form their points
    const bool pts_host = pts_xy_m && !dd::is_device_pointer(pts_xy_m);
    const bool out_host = !dd::is_device_pointer(out);
    const size_t npt = (size_t)std::max<int64_t>(1, b->total_pts);
    if ((pts_host && !b->d_pts) || (out_host && !b->d_out)) {
        if (!b->d_pts) DD_CUDA_TRY(cudaMalloc(&b->d_pts, 2 * npt * sizeof(double)));
        if (!b->d_out) DD_CUDA_TRY(cudaMalloc(&b->d_out, npt * sizeof(double)));
    }
    const double *pts = pts_xy_m;
    double *dst = out;
    if (pts_host) {
        DD_CUDA_TRY(cudaMemcpyAsync(b->d_pts, pts_xy_m, 2 * (size_t)b->total_pts * sizeof(double),
                                    cudaMemcpyHostToDevice, stream));
        pts = b->d_pts;
    }
    if (out_host) dst = b->d_out;
    if (!b->exec || b->g_pts != pts || b->g_out != dst || b->g_variant != b->variant) {
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        cudaGraph_t graph;
        DD_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        dd_status st = enqueue(b, pts, dst, b->variant, b->cap);
        cudaError_t err = cudaStreamEndCapture(b->cap, &graph);
        if (st != DD_OK) return st;
        if (err != cudaSuccess) return dd::fail_cuda(err, "cudaStreamEndCapture");
        err = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (err != cudaSuccess) return dd::fail_cuda(err, "cudaGraphInstantiate");
        b->g_pts = pts;
        b->g_out = dst;
        b->g_variant = b->variant;
    }
    {
        dd::ProfScope ps(b->grid_tiles ? "batch_grid_mixed_32x32" : variant_name(b->prec, b->variant), stream);
        DD_CUDA_TRY(cudaGraphLaunch(b->exec, stream));
    }
    if (out_host)
        DD_CUDA_TRY(cudaMemcpyAsync(out, dst, (size_t)b->total_pts * sizeof(double), cudaMemcpyDeviceToHost, stream));
    if (out_host || pts_host) DD_CUDA_TRY(cudaStreamSynchronize(stream));
    return DD_OK;
}

void dd_batch_destroy(dd_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_coef) cudaEventDestroy(b->ev_coef);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    cudaFree(b->ws);
    cudaFree(b->d_pts);
    cudaFree(b->d_out);
    cudaGetLastError();
    delete b;
}

dd_status dd_batch_info(const dd_batch *b, int64_t *n_items, int64_t *pairs, int32_t *variant) {
    dd::clear_error();
    if (!b) return dd::fail(DD_EINVAL, "dd_batch_info: NULL plan");
    if (n_items) *n_items = b->n_items;
    if (variant) *variant = b->variant;
    if (pairs) *pairs = b->pairs;
    return DD_OK;
}

dd_status dd_field_batch(const dd_scan *const *scans, int32_t n_scans, const int64_t *pt_offsets,
                         const double *pts_xy_m, const double *times_s, dd_precision prec,
                         double *out, void *cuda_stream) {
    dd::clear_error();
    if (!pts_xy_m || !out) return dd::fail(DD_EINVAL, "dd_field_batch: NULL buffer");
    dd_batch *b = nullptr;
    dd_status st = dd_batch_create(scans, n_scans, pt_offsets, times_s, prec, &b);
    if (st != DD_OK) return st;
    st = dd_batch_run(b, pts_xy_m, out, cuda_stream);
    if (st == DD_OK) {
        cudaError_t err = cudaStreamSynchronize((cudaStream_t)cuda_stream);
        if (err != cudaSuccess) st = dd::fail_cuda(err, "dd_field_batch: stream");
    }
    dd_batch_destroy(b);
    return st;
}

}  // extern "C"
