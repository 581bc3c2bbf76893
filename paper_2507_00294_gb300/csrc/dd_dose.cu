// dd_dose.cu -- dwell-start dose of every visit: out[j] = psi_{j-1}(r_j, t_j)
// = sum_{i<j} phi_i(r_j, t_j)  (Eq. 5 evaluated at the probe position when its dwell
// starts; the paper's psi_j of Eq. 5 with j-1 visits).
//
// With a uniform dwell and no flyback the visit start times are t_k = k tau, so the
// pair (i, j) only depends on the lag k = j - i through w0, w1 (Eq. 1 at k = 1, where
// the beam of visit i switches off exactly at t_j, Eq. 2 for k > 1): one coefficient
// record per lag.  The kernel walks lags outermost, so all lanes of a warp read the
// same record (a shared-memory broadcast) while each lane's source index j - k is
// different and contiguous.  Work items are (target tile, lag block), cost-sorted;
// per-block partial sums are reduced in block order (deterministic).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "dd_coef.cuh"
#include "dd_e1.cuh"
#include "dd_field_impl.cuh"
#include "dd_internal.h"

namespace ddk {

// Lag blocks of the dose work items.  The smallest lags are the costliest pairs (at dwell
// start the source k visits back lies about k pitches away, so h = rho^2 dq stays near 1:
// the high series degrees and the two-E1 path), so the first lb lags come in kDoseSplit
// blocks of lb / kDoseSplit, and every later block holds lb lags: block b covers lags
// [k0, k1) below.  lb is a multiple of kDoseSplit.
constexpr int kDoseSplit = 8;
__host__ __device__ inline void dose_block_lags(int64_t b, int lb, int64_t &k0, int64_t &k1) {
    const int q = lb / kDoseSplit;
    if (b < kDoseSplit) { k0 = 1 + b * q; k1 = k0 + q; }
    else { k0 = 1 + (b - kDoseSplit + 1) * (int64_t)lb; k1 = k0 + lb; }
}
// Blocks needed for the lags 1 .. t1 - 1 of a tile whose last target is t1 - 1.
__host__ __device__ inline int64_t dose_blocks(int64_t t1, int lb) {
    const int64_t kmax = t1 - 1;                     // largest lag
    if (kmax < 1) return 0;
    const int q = lb / kDoseSplit;
    if (kmax <= lb) return (kmax - 1) / q + 1;
    return kDoseSplit + (kmax - lb - 1) / lb + 1;
}

// FP64 dose: PPT = Cfg::kDosePPT targets per thread (strided by the block size), lags
// outermost, one pair term per (target, lag) at the pair's own series class.
template <typename Cfg>
__global__ void __launch_bounds__(Cfg::kThreads)
dose_kernel(const double *__restrict__ srcX, const double *__restrict__ srcY, int64_t n,
            const typename Cfg::Rec *__restrict__ lagrec, const int2 *__restrict__ items, int lb,
            typename Cfg::Real *__restrict__ partial) {
    using Rec = typename Cfg::Rec;
    using Real = typename Cfg::Real;
    static_assert(std::is_same<Real, double>::value, "the FP32 dose runs dose_kernel_f32");
    constexpr int NT = Cfg::kThreads, PPT = Cfg::kDosePPT, TILE = NT * PPT, LBMAX = Cfg::kDoseLB;
    constexpr int RV = sizeof(Rec) / 16;
    __shared__ Real s_x[TILE + LBMAX], s_y[TILE + LBMAX];
    __shared__ __align__(16) Rec s_rec[Cfg::kDoseSTILE];

    const int2 item = items[blockIdx.x];
    const int tid = threadIdx.x;
    const int64_t t0 = (int64_t)item.x * TILE;             // first target of the tile
    const int64_t t1 = min((int64_t)n, t0 + TILE);
    int64_t kb0, kb1;
    dose_block_lags(item.y, lb, kb0, kb1);
    const int k0 = (int)kb0;                               // lags [k0, k1)
    const int k1 = (int)min(kb1, t1);                      // lag < target index <= t1 - 1
    // sources needed: i = j - k for j in [t0, t1), k in [k0, k1): i in [t0 - k1 + 1, t1 - k0)
    const int64_t w0 = t0 - k1 + 1;
    const int64_t w1 = t1 - k0;
    // coordinates relative to the tile's first target
    const double cx = srcX[t0], cy = srcY[t0];
    for (int64_t i = w0 + tid; i < w1; i += NT) {
        const int64_t ic = i < 0 ? 0 : i;                  // i < 0 never used
        s_x[i - w0] = (Real)(srcX[ic] - cx);
        s_y[i - w0] = (Real)(srcY[ic] - cy);
    }
    Real px[PPT], py[PPT];
    int64_t jt[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        jt[q] = t0 + q * NT + tid;
        const int64_t jj = jt[q] < n ? jt[q] : t0;
        px[q] = (Real)(srcX[jj] - cx);
        py[q] = (Real)(srcY[jj] - cy);
    }
    Real acc[PPT];
    BlockSum<Real> tot[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) acc[q] = 0;

    for (int kk = k0; kk < k1; kk += Cfg::kDoseSTILE) {
        const int cnt = min(Cfg::kDoseSTILE, k1 - kk);
        __syncthreads();
        {
            const float4 *row = reinterpret_cast<const float4 *>(lagrec + kk);
            float4 *dst = reinterpret_cast<float4 *>(&s_rec[0]);
            for (int v = tid; v < cnt * RV; v += NT) dst[v] = row[v];
        }
        __syncthreads();
        for (int c = 0; c < cnt; ++c) {
            const int k = kk + c;
            const Rec &R = s_rec[c];
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                const int64_t i = jt[q] - k;
                if (i >= 0 && jt[q] < n) {
                    const Real dx = px[q] - s_x[i - w0], dy = py[q] - s_y[i - w0];
                    acc[q] += pair_term(dx * dx + dy * dy, R);
                }
            }
            if (Cfg::kFlush < Cfg::kDoseSTILE && (c % Cfg::kFlush) == Cfg::kFlush - 1) {
#pragma unroll
                for (int q = 0; q < PPT; ++q) { tot[q].add(acc[q]); acc[q] = 0; }
            }
        }
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            tot[q].add(acc[q]);
            acc[q] = 0;
        }
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q)
        if (jt[q] < n) partial[(int64_t)item.y * n + jt[q]] = tot[q].result();
}

// The lags [kk, kk + cnt) of one staged round of the FP32 dose for this thread's PPT targets
// (target pairs (2m, 2m + 1) on f32x2).  rel[q]: the target's index in the coordinate
// window, whose entry rel[q] - k is the source of lag k (always inside the window).
// kFull: every (target, lag) pair of the item exists; otherwise pair q exists when bit q
// of live is set (target < n) and rel[q] - k >= lo_idx (source index >= 0).  One exponent-series
// degree per warp and lag, from the largest h and the smallest a over its lanes (the
// classes of the field kernel); degree 2, the common case, settled by one vote.
template <int PPT, bool kFull>
__device__ __forceinline__ void dose_lags_f32(const RecF32 *s_rec, int cnt, int kk, const float2 *s_xy,
                                              const float (&px)[PPT], const float (&py)[PPT], const int (&rel)[PPT],
                                              uint32_t live, int lo_idx, float2 (&acc2)[PPT / 2]) {
    static_assert(PPT <= 32, "pair flags in one word");
    for (int c = 0; c < cnt; ++c) {
        const int k = kk + c;
        const RecF32 &R = s_rec[c];
        const float dqR = R.dq();
        float r2[PPT];
        // bit q: pair q exists (flags in a word rather than PPT predicates)
        uint32_t ok = kFull ? (1u << PPT) - 1u : 0u;
        float rmax = 0.0f;
#pragma unroll
        for (int m = 0; m < PPT / 2; ++m) {
            const int ia = rel[2 * m] - k, ib = rel[2 * m + 1] - k;
            if (!kFull) {
                ok |= (((live >> (2 * m)) & 1u) && ia >= lo_idx ? 1u : 0u) << (2 * m);
                ok |= (((live >> (2 * m + 1)) & 1u) && ib >= lo_idx ? 1u : 0u) << (2 * m + 1);
            }
            // a pair that does not exist takes its own target as the source (rho^2 = 0)
            const float2 sa = ((ok >> (2 * m)) & 1u) ? s_xy[ia] : make_float2(px[2 * m], py[2 * m]);
            const float2 sb = ((ok >> (2 * m + 1)) & 1u) ? s_xy[ib] : make_float2(px[2 * m + 1], py[2 * m + 1]);
            const float2 dx = __fadd2_rn(make_float2(px[2 * m], px[2 * m + 1]), make_float2(-sa.x, -sb.x));
            const float2 dy = __fadd2_rn(make_float2(py[2 * m], py[2 * m + 1]), make_float2(-sa.y, -sb.y));
            const float2 q2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
            r2[2 * m] = q2.x;
            r2[2 * m + 1] = q2.y;
            rmax = fmaxf(rmax, fmaxf(q2.x, q2.y));
        }
        // use: the pairs whose terms are added.  When the whole warp is on degree 2 (one
        // vote: every pair's h, culled or not, is in that series' range) every existing
        // pair; else the class is the largest of the pairs' own classes, and a pair whose
        // own a is 87 or more (its term below 2e-38) is left out: its h can lie far beyond
        // the range of the warp's series, whose polynomial would then overflow.
        uint32_t use = ok;
        uint32_t cls = kCodeD2;
        if (!__all_sync(0xffffffffu, rmax * dqR <= kL2H && dqR >= kMinDqX)) {
            cls = kCodeSkip;
            use = 0u;
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                const uint32_t cq = !((ok >> q) & 1u) ? kCodeSkip : series_class(r2[q] * dqR, r2[q] * R.q1(), dqR);
                use |= (cq != kCodeSkip ? 1u : 0u) << q;
                cls = max(cls, cq);
            }
            cls = __reduce_max_sync(0xffffffffu, cls);
        }
        if (cls == kCodeSkip) continue;
        if (cls == kCodeD2) {
            // degree 2 on f32x2 over target pairs; a pair left out gets the exponent -inf
            // (term 0)
            const float4 v0 = R.v0;                        // (g_0, g_1x, g_2x, g_3x)
            const float2 g2 = make_float2(v0.z, v0.z), g1 = make_float2(v0.y, v0.y);
#pragma unroll
            for (int m = 0; m < PPT / 2; ++m) {
                const float2 r = make_float2(r2[2 * m], r2[2 * m + 1]);
                const float2 g0 = make_float2(((use >> (2 * m)) & 1u) ? v0.x : -INFINITY,
                                              ((use >> (2 * m + 1)) & 1u) ? v0.x : -INFINITY);
                const float2 g = __ffma2_rn(__ffma2_rn(g2, r, g1), r, g0);
                acc2[m] = __fadd2_rn(acc2[m], make_float2(ex2_approx(g.x), ex2_approx(g.y)));
            }
            continue;
        }
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            float t;
            if (cls == kCodeD4) t = log_term<4>(r2[q], R);
            else if (cls == kCodeD8) t = log_term<8>(r2[q], R);
            else if (cls == kCodeD12) t = log_term<12>(r2[q], R);
            else t = pair_term(r2[q], R);
            if ((use >> q) & 1u) { if (q & 1) acc2[q >> 1].y += t; else acc2[q >> 1].x += t; }
        }
    }
}

// FP32 dose: PPT targets per thread (strided by the block size: a warp's lanes hold
// consecutive targets), lags outermost, so all lanes of a warp read one lag record (a
// shared-memory broadcast) while each lane's source is its own.  More targets per thread
// share each lag's record, vote and loop over more pairs (the large scans take 4); the
// coordinates are FP32 differences from the float-float copy (no FP64 arithmetic).
template <typename Cfg, int PPT>
__global__ void __launch_bounds__(Cfg::kThreads)
dose_kernel_f32(int64_t n, const RecF32 *__restrict__ lagrec, const int2 *__restrict__ items, int lb,
                float *__restrict__ partial, const float4 *__restrict__ srcF) {
    static_assert(std::is_same<typename Cfg::Real, float>::value, "FP32 records and sums");
    static_assert(PPT % 2 == 0, "the FP32 path takes targets in pairs");
    constexpr int NT = Cfg::kThreads, TILE = NT * PPT, LBMAX = Cfg::kDoseLB;
    constexpr int RV = sizeof(RecF32) / 16;
    __shared__ float2 s_xy[TILE + LBMAX];
    __shared__ __align__(16) RecF32 s_rec[Cfg::kDoseSTILE];

    const int2 item = items[blockIdx.x];
    const int tid = threadIdx.x;
    const int64_t t0 = (int64_t)item.x * TILE;             // first target of the tile
    const int64_t t1 = min((int64_t)n, t0 + TILE);
    int64_t kb0, kb1;
    dose_block_lags(item.y, lb, kb0, kb1);
    const int k0 = (int)kb0;                               // lags [k0, k1)
    const int k1 = (int)min(kb1, t1);                      // lag < target index <= t1 - 1
    // sources needed: i = j - k for j in [t0, t1), k in [k0, k1): the window
    // [t0 - k1 + 1, t1 - k0), at most TILE + lb - 1 visits
    const int64_t w0 = t0 - k1 + 1;
    const int64_t w1 = t1 - k0;
    const float4 org = srcF[t0];
    for (int64_t i = w0 + tid; i < w1; i += NT) {
        const int64_t ic = i < 0 ? 0 : i;                  // i < 0 never used
        s_xy[i - w0] = ff_diff(srcF[ic], org);
    }
    float px[PPT], py[PPT];
    int rel[PPT];
    uint32_t live = 0;                                     // bit q: target q < n
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int64_t jt = t0 + q * NT + tid;
        live |= (jt < n ? 1u : 0u) << q;
        const float2 d = ff_diff(srcF[jt < n ? jt : t0], org);
        px[q] = d.x;
        py[q] = d.y;
        rel[q] = (int)(jt - w0);
    }
    // source index i = w0 + (rel - k) >= 0
    const int lo_idx = (int)(w0 < 0 ? -w0 : 0);
    // every (target, lag) pair of this item exists: the whole tile lies in [0, n) and its
    // first target is beyond the block's largest lag
    const bool full = t0 + TILE <= n && (int64_t)k1 - 1 <= t0;
    // FP32 sums of one staged round of lags, added into a compensated running sum
    float2 acc2[PPT / 2];
    BlockSum<float> tot[PPT];
#pragma unroll
    for (int m = 0; m < PPT / 2; ++m) acc2[m] = make_float2(0.f, 0.f);

    for (int kk = k0; kk < k1; kk += Cfg::kDoseSTILE) {
        const int cnt = min(Cfg::kDoseSTILE, k1 - kk);
        __syncthreads();
        {
            const float4 *row = reinterpret_cast<const float4 *>(lagrec + kk);
            float4 *dst = reinterpret_cast<float4 *>(&s_rec[0]);
            for (int v = tid; v < cnt * RV; v += NT) dst[v] = row[v];
        }
        __syncthreads();
        if (full) dose_lags_f32<PPT, true>(s_rec, cnt, kk, s_xy, px, py, rel, live, lo_idx, acc2);
        else dose_lags_f32<PPT, false>(s_rec, cnt, kk, s_xy, px, py, rel, live, lo_idx, acc2);
#pragma unroll
        for (int q = 0; q < PPT; ++q) tot[q].add((q & 1) ? acc2[q >> 1].y : acc2[q >> 1].x);
#pragma unroll
        for (int m = 0; m < PPT / 2; ++m) acc2[m] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q)
        if ((live >> q) & 1u) partial[(int64_t)item.y * n + t0 + q * NT + tid] = tot[q].result();
}

// Dose for arbitrary visit timing (per-visit dwells, flyback): the pair (i, j) has its
// own elapsed time t_j - t_i, so its coefficients are formed per pair in FP64 from the
// same formulas as the (snapshot, visit) records (pair_geometry, moment_coefficients)
// and evaluated with the precision's pair_term.  One thread per target j; the visits
// before the CTA's last target are staged through shared memory in visit order.
template <typename Cfg>
__global__ void __launch_bounds__(128)
dose_general_kernel(const double *__restrict__ src, int64_t n, int64_t j0, int64_t j1, double s,
                    double kappa, double *__restrict__ out_partial) {
    using Rec = typename Cfg::Rec;
    using Real = typename Cfg::Real;
    constexpr int TILE = 64;
    __shared__ double s_x[TILE], s_y[TILE], s_t[TILE], s_tau[TILE];
    const double *X = src, *Y = src + n, *T = src + 2 * n, *TAU = src + 3 * n;
    // targets j0 + [blockIdx.x * blockDim.x, ...) of the range [j0, j1)
    const int64_t j = j0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j_last = min(j1, j0 + (int64_t)(blockIdx.x + 1) * blockDim.x) - 1;
    const bool live = j < j1;
    const double xj = live ? X[j] : 0.0, yj = live ? Y[j] : 0.0, tj = live ? T[j] : 0.0;
    double tot = 0.0;
    for (int64_t i0 = 0; i0 < j_last; i0 += TILE) {
        const int cnt = (int)min((int64_t)TILE, j_last - i0);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
            s_x[q] = X[i0 + q]; s_y[q] = Y[i0 + q]; s_t[q] = T[i0 + q]; s_tau[q] = TAU[i0 + q];
        }
        __syncthreads();
        Real acc = 0;
        for (int q = 0; q < cnt; ++q) {
            if (!live || i0 + q >= j) break;
            double q1, dq, r, ell;
            pair_geometry<RecTraits<Rec>::kFP64Ell>(tj - s_t[q], s_tau[q], s, kappa, q1, dq, r, ell);
            Rec R;
            RecTraits<Rec>::fill(R, q1, dq, r, ell);
            const Real dx = (Real)(xj - s_x[q]), dy = (Real)(yj - s_y[q]);
            acc += pair_term(dx * dx + dy * dy, R);
        }
        tot += (double)acc;
    }
    if (live) out_partial[j - j0] = tot;
}

__global__ void scale_kernel(const double *__restrict__ v, int64_t n, double pref, double *__restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = pref * v[j];
}

// out[j - j0] = pref * sum over the lag blocks of target j, j in [j0, j1).  A block of 256 threads serves 32
// targets: lane t of warp q sums the blocks b = q, q + 8, q + 16, ... of target t (in
// order), and warp 0 adds the eight results in q order -- a fixed association, so the
// result is deterministic, with eight times the loads in flight of one thread per target.
constexpr int kDoseReduceSplit = 8;
template <typename Part>
__global__ void __launch_bounds__(32 * kDoseReduceSplit)
dose_reduce_kernel(const Part *__restrict__ partial, int64_t n, int64_t j0, int64_t j1, int tile, int lb,
                   double pref, double *__restrict__ out) {
    __shared__ double s_sum[kDoseReduceSplit][32];
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int64_t j = j0 + (int64_t)blockIdx.x * 32 + lane;
    double v = 0.0;
    if (j < j1) {
        // blocks written for target j: every lag block that starts below the tile's last target
        const int64_t tile_last = min(n, (j / tile + 1) * tile) - 1;
        const int64_t nb = dose_blocks(tile_last + 1, lb);
        BlockSum<Part> acc;
#pragma unroll 4
        for (int64_t b = q; b < nb; b += kDoseReduceSplit) acc.add(partial[b * n + j]);
        v = acc.value();
    }
    s_sum[q][lane] = v;
    __syncthreads();
    if (q == 0 && j < j1) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kDoseReduceSplit; ++k) t += s_sum[k][lane];
        out[j - j0] = pref * t;
    }
}

}  // namespace ddk

namespace {

int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 1;
    }
    return sms;
}

// Work items (target tile, lag block) of the tiles [tile_lo, tile_hi) of `tile` targets.
int64_t dose_items(int64_t n, int64_t tile_lo, int64_t tile_hi, int tile, int lb) {
    int64_t items = 0;
    for (int64_t t = tile_lo; t < tile_hi; ++t) items += ddk::dose_blocks(std::min(n, t * tile + tile), lb);
    return items;
}

// Lag block of the dose work items: the largest power-of-two fraction of kDoseLB, down to
// kDoseLBMin lags, that still gives at least 8 items per SM (the triangle of a few
// thousand visits is otherwise cut into too few CTAs to fill the GPU).
template <typename Cfg>
int dose_lag_block(int64_t n, int64_t j0, int64_t j1, int tile) {
    const int64_t want = 8 * (int64_t)device_sms();
    const int64_t tile_lo = j0 / tile, tile_hi = (j1 + tile - 1) / tile;
    int lb = Cfg::kDoseLB;
    while (lb > Cfg::kDoseLBMin && dose_items(n, tile_lo, tile_hi, tile, lb) < want) lb /= 2;
    return lb;
}

// Targets per thread of the FP32 dose: kDoseWidePPT when the wide tiles still give at least
// 8 items per SM at the largest lag block (large scans), else Cfg::kDosePPT.
constexpr int kDoseWidePPT = 4;
template <typename Cfg>
int dose_ppt(int64_t n, int64_t j0, int64_t j1) {
    if (!std::is_same<typename Cfg::Real, float>::value) return Cfg::kDosePPT;
    const int tile = Cfg::kThreads * kDoseWidePPT;
    return dose_items(n, j0 / tile, (j1 + tile - 1) / tile, tile, Cfg::kDoseLB) >= 8 * (int64_t)device_sms()
               ? kDoseWidePPT : Cfg::kDosePPT;
}

// One launch of the dose kernel over `count` items: the FP32 kernel at `ppt` targets per
// thread, or the FP64 kernel.
template <typename Cfg>
cudaError_t launch_dose(unsigned count, int ppt, cudaStream_t stream, const double *srcX, const double *srcY,
                        int64_t n, const typename Cfg::Rec *rec, const int2 *items, int lb,
                        typename Cfg::Real *part, const float4 *srcF) {
    if constexpr (std::is_same<typename Cfg::Real, float>::value) {
        if (ppt == kDoseWidePPT)
            ddk::dose_kernel_f32<Cfg, kDoseWidePPT><<<count, Cfg::kThreads, 0, stream>>>(n, rec, items, lb, part, srcF);
        else
            ddk::dose_kernel_f32<Cfg, Cfg::kDosePPT><<<count, Cfg::kThreads, 0, stream>>>(n, rec, items, lb, part, srcF);
    } else {
        ddk::dose_kernel<Cfg><<<count, Cfg::kThreads, 0, stream>>>(srcX, srcY, n, rec, items, lb, part);
    }
    return cudaGetLastError();
}

// Valid (target j, lag k) pairs of a dose work item: targets [t0, t1), lags [k0, k1) with
// k1 <= t1, pair valid when k <= j, i.e. sum_k (t1 - max(t0, k)): t1 - t0 for every lag up
// to t0, then t1 - k (an arithmetic series) for the lags beyond.
inline int64_t dose_item_pairs(int64_t t0, int64_t t1, int64_t k0, int64_t k1) {
    const int64_t full = std::max<int64_t>(0, std::min(k1, t0 + 1) - k0) * (t1 - t0);
    const int64_t a = std::max(k0, t0 + 1), b = k1 - 1;
    return full + (a <= b ? (b - a + 1) * t1 - (a + b) * (b - a + 1) / 2 : 0);
}

// Dose of the targets [j0, j1): the target tiles that overlap the range are evaluated
// whole, and only the range is reduced and written (out[j - j0]).
template <typename Cfg>
dd_status run_dose(const dd_scan *scan, int64_t j0, int64_t j1, double *out, cudaStream_t stream) {
    using Rec = typename Cfg::Rec;
    const int64_t n = scan->n;
    const int64_t m = j1 - j0;
    const dd::MemKind out_kind = dd::memory_kind(out);
    const bool out_host = out_kind != dd::MemKind::Device;
    const bool out_copy = out_host;
    const int ppt = dose_ppt<Cfg>(n, j0, j1);
    const int TILE = Cfg::kThreads * ppt;
    const int64_t tile_lo = j0 / TILE, tile_hi = (j1 + TILE - 1) / TILE;
    const int lb = dose_lag_block<Cfg>(n, j0, j1, TILE);
    const int64_t n_items = dose_items(n, tile_lo, tile_hi, TILE, lb);   // lags 1 .. t1-1 per tile
    const int64_t nblk = ddk::dose_blocks(std::min(n, tile_hi * TILE), lb);
    size_t bytes = 0;
    auto add = [&](size_t b) { bytes = ((bytes + 255) & ~size_t(255)) + b; };
    add((size_t)std::max<int64_t>(n, 1) * sizeof(Rec));
    add((size_t)n_items * sizeof(int2) + 16);
    add((size_t)std::max<int64_t>(nblk, 1) * n * sizeof(typename Cfg::Real));
    if (out_copy) add((size_t)m * sizeof(double));
    bytes += 256;

    dd_status st = DD_OK;
    const double *src = dd::device_sources(scan, stream, &st);
    if (!src) return st;
    const dd::ScanUse use{scan, stream};
    const float4 *srcF = dd::device_sources_ff(scan, stream, &st);
    void *ws = nullptr;
    cudaError_t err = dd::workspace_alloc(&ws, bytes, stream);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return dd::fail(err == cudaErrorMemoryAllocation ? DD_ENOMEM : DD_ECUDA,
                        std::string("dose workspace allocation: ") + cudaGetErrorString(err));
    }
    char *base = (char *)ws;
    size_t off = 0;
    auto take = [&](size_t b) { off = (off + 255) & ~size_t(255); char *p = base + off; off += b; return p; };
    Rec *d_rec = (Rec *)take((size_t)std::max<int64_t>(n, 1) * sizeof(Rec));
    int2 *d_items = (int2 *)take((size_t)n_items * sizeof(int2) + 16);
    using Part = typename Cfg::Real;
    Part *d_part = (Part *)take((size_t)std::max<int64_t>(nblk, 1) * n * sizeof(Part));
    double *out_dev = out_copy ? (double *)take((size_t)m * sizeof(double)) : out;

    // work list, kept until the stream has consumed its upload (pinned staging when available)
    struct Keep {
        std::vector<int2> items;
        dd::CallStaging staging;
    };
    auto *keep = new Keep();
    if (n >= 2) {
        // the lag table first: the GPU builds it while the host sorts the work list
        DD_PROFILED(Cfg::kLagCoefName, stream,
                    (ddk::lag_coef_kernel<Rec><<<(unsigned)((n + 31) / 32), 32, 0, stream>>>(n, scan->s, scan->kappa, d_rec)));
        DD_CUDA_TRY(cudaGetLastError());
        std::vector<std::pair<int64_t, int2>> its;
        its.reserve((size_t)n_items);
        for (int64_t t = tile_lo; t < tile_hi; ++t) {
            const int64_t t0 = t * TILE, t1 = std::min(n, t0 + TILE);
            if (t1 - 1 < 1) continue;                                // target 0 has no source
            const int64_t nb = ddk::dose_blocks(t1, lb);             // lags 1 .. t1-1
            for (int64_t b = 0; b < nb; ++b) {
                int64_t k0, k1;
                ddk::dose_block_lags(b, lb, k0, k1);
                k1 = std::min(k1, t1);
                its.push_back({dose_item_pairs(t0, t1, k0, k1), make_int2((int)t, (int)b)});
            }
        }
        std::stable_sort(its.begin(), its.end(),
                         [](const std::pair<int64_t, int2> &a, const std::pair<int64_t, int2> &b) { return a.first > b.first; });
        keep->items.resize(its.size());
        for (size_t k = 0; k < its.size(); ++k) keep->items[k] = its[k].second;
        DD_CUDA_TRY(keep->staging.upload(d_items, keep->items.data(), keep->items.size() * sizeof(int2), stream));
        DD_PROFILED(Cfg::kDoseName, stream,
                    DD_CUDA_TRY(launch_dose<Cfg>((unsigned)keep->items.size(), ppt, stream, src, src + n, n, d_rec,
                                                 d_items, lb, d_part, srcF)));
    }
    DD_PROFILED("dose_reduce", stream,
                (ddk::dose_reduce_kernel<Part><<<(unsigned)((m + 31) / 32), 32 * ddk::kDoseReduceSplit, 0, stream>>>(d_part, n, j0, j1, TILE, lb, scan->pref, out_dev)));
    DD_CUDA_TRY(cudaGetLastError());
    if (out_copy)
        DD_CUDA_TRY(cudaMemcpyAsync(out, out_dev, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, stream));
    DD_CUDA_TRY(dd::workspace_release(ws, stream));
    DD_CUDA_TRY(dd::defer_release(stream, keep, [](void *p) { delete static_cast<Keep *>(p); }));
    if (dd::host_sync_needed(stream, {out_kind})) DD_CUDA_TRY(cudaStreamSynchronize(stream));
    return DD_OK;
}

template <typename Cfg>
dd_status run_dose_general(const dd_scan *scan, int64_t j0, int64_t j1, double *out, cudaStream_t stream) {
    const int64_t n = scan->n;
    const int64_t m = j1 - j0;
    const dd::MemKind out_kind = dd::memory_kind(out);
    const bool out_host = out_kind != dd::MemKind::Device;
    dd_status st = DD_OK;
    const double *src = dd::device_sources(scan, stream, &st);
    if (!src) return st;
    const dd::ScanUse use{scan, stream};
    void *ws = nullptr;
    const size_t bytes = (size_t)m * sizeof(double) * (out_host ? 2 : 1) + 512;
    cudaError_t err = dd::workspace_alloc(&ws, bytes, stream);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return dd::fail(err == cudaErrorMemoryAllocation ? DD_ENOMEM : DD_ECUDA,
                        std::string("dose workspace allocation: ") + cudaGetErrorString(err));
    }
    double *sums = (double *)ws;
    double *out_dev = out_host ? sums + m : out;
    DD_PROFILED(Cfg::kDoseName, stream,
                (ddk::dose_general_kernel<Cfg><<<(unsigned)((m + 127) / 128), 128, 0, stream>>>(
                    src, n, j0, j1, scan->s, scan->kappa, sums)));
    DD_CUDA_TRY(cudaGetLastError());
    DD_PROFILED("dose_scale", stream,
                (ddk::scale_kernel<<<(unsigned)((m + 255) / 256), 256, 0, stream>>>(sums, m, scan->pref, out_dev)));
    DD_CUDA_TRY(cudaGetLastError());
    if (out_host)
        DD_CUDA_TRY(cudaMemcpyAsync(out, out_dev, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, stream));
    DD_CUDA_TRY(dd::workspace_release(ws, stream));
    if (dd::host_sync_needed(stream, {out_kind})) DD_CUDA_TRY(cudaStreamSynchronize(stream));
    return DD_OK;
}

}  // namespace

namespace {

dd_status dose_range(const dd_scan *scan, dd_precision prec, int64_t j0, int64_t j1, double *out,
                     void *cuda_stream) {
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    if (!scan->uniform) {
        // per-visit dwells, flyback or blanker travel: no lag table, coefficients per pair
        if (prec == DD_MIXED) return run_dose_general<ddk::CfgMixed>(scan, j0, j1, out, stream);
        return run_dose_general<ddk::CfgF64>(scan, j0, j1, out, stream);
    }
    if (prec == DD_MIXED) return run_dose<ddk::CfgMixed>(scan, j0, j1, out, stream);
    return run_dose<ddk::CfgF64>(scan, j0, j1, out, stream);
}

}  // namespace

extern "C" dd_status dd_per_probe_dose(const dd_scan *scan, dd_precision prec, double *out, void *cuda_stream) {
    dd::clear_error();
    if (!scan || !out) return dd::fail(DD_EINVAL, "dd_per_probe_dose: NULL argument");
    if (prec != DD_FP64 && prec != DD_MIXED) return dd::fail(DD_EINVAL, "dd_per_probe_dose: unknown precision");
    return dose_range(scan, prec, 0, scan->n, out, cuda_stream);
}

extern "C" dd_status dd_per_probe_dose_range(const dd_scan *scan, dd_precision prec, int64_t j0, int64_t j1,
                                             double *out, void *cuda_stream) {
    dd::clear_error();
    if (!scan) return dd::fail(DD_EINVAL, "dd_per_probe_dose_range: NULL scan");
    if (prec != DD_FP64 && prec != DD_MIXED)
        return dd::fail(DD_EINVAL, "dd_per_probe_dose_range: unknown precision");
    if (j0 < 0 || j1 < j0 || j1 > scan->n)
        return dd::fail(DD_EINVAL, "dd_per_probe_dose_range: need 0 <= j0 <= j1 <= n_visits");
    if (j1 == j0) return DD_OK;
    if (!out) return dd::fail(DD_EINVAL, "dd_per_probe_dose_range: NULL output");
    return dose_range(scan, prec, j0, j1, out, cuda_stream);
}

// ---------------------------------------------------------------------------------
// Allocation-free dose.  Some callers cannot allocate device memory during a run: a
// microscope acquisition loop that reserves its whole memory budget before the scan
// starts, a host that hands the device allocator to another framework, or code on a
// path where cudaMalloc's implicit synchronisation is not allowed.  This entry point
// keeps its scratch (visit coordinates, lag records, work list, partial sums) in one
// file-scope device array and calls no device allocator.
namespace {

constexpr size_t kNoAllocBytes = size_t(8) << 20;       // 8 MiB: up to 16384 visits
constexpr int64_t kNoAllocMaxVisits = 16384;
constexpr int kNoAllocMaxItems = 4096;
constexpr int kNoAllocMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_dose_scratch[kNoAllocBytes];

namespace {

std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of g_dose_scratch on the current device; looked up once per device.
dd_status noalloc_scratch(char **addr) {
    int dev = 0;
    DD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return dd::fail(DD_ENOTSUP, "dd_per_probe_dose_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t err = cudaGetSymbolAddress(&p, g_dose_scratch);
        if (err != cudaSuccess) return dd::fail_cuda(err, "cudaGetSymbolAddress(g_dose_scratch)");
        g_noalloc_addr[dev] = p;
    }
    *addr = (char *)g_noalloc_addr[dev];
    return DD_OK;
}

// Float-float copy (hi, lo, hi, lo) of FP64 coordinates: hi = x rounded to FP32, lo = the
// FP64 remainder x - hi (exact) rounded to FP32 -- the same values as the scan's cached
// float-float copy, which is built on the host by the same two roundings.
__global__ void ff_coords_kernel(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
                                 float4 *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double xv = x[i], yv = y[i];
    const float xh = __double2float_rn(xv), yh = __double2float_rn(yv);
    out[i] = make_float4(xh, __double2float_rn(xv - (double)xh), yh, __double2float_rn(yv - (double)yh));
}

template <typename Cfg>
dd_status run_dose_noalloc(const dd_scan *scan, double *out, cudaStream_t stream, char *scratch) {
    using Rec = typename Cfg::Rec;
    const int64_t n = scan->n;
    constexpr int TILE = Cfg::kThreads * Cfg::kDosePPT;
    const int lb = Cfg::kDoseLB;
    const int64_t n_tiles = (n + TILE - 1) / TILE;
    const int64_t nblk = ddk::dose_blocks(n, lb);
    size_t off = 0;
    auto take = [&](size_t bytes) { off = (off + 255) & ~size_t(255); size_t o = off; off += bytes; return o; };
    const size_t o_x = take(2 * (size_t)n * sizeof(double));
    const size_t o_f = take((size_t)n * sizeof(float4));
    const size_t o_rec = take((size_t)n * sizeof(Rec));
    using Part = typename Cfg::Real;
    const size_t o_part = take((size_t)std::max<int64_t>(nblk, 1) * n * sizeof(Part));
    const size_t o_items = take((size_t)kNoAllocMaxItems * sizeof(int2));
    if (off > kNoAllocBytes)
        return dd::fail(DD_EINVAL, "dd_per_probe_dose_noalloc: scan needs more scratch than the 8 MiB built-in area");

    // work list on the host (fixed storage, no heap), same cost order as dd_per_probe_dose
    static thread_local std::pair<int64_t, int2> its[kNoAllocMaxItems];
    static thread_local int2 flat[kNoAllocMaxItems];
    int count = 0;
    for (int64_t t = 0; t < n_tiles; ++t) {
        const int64_t t0 = t * TILE, t1 = std::min(n, t0 + TILE);
        if (t1 - 1 < 1) continue;
        const int64_t nb = ddk::dose_blocks(t1, lb);
        for (int64_t bk = 0; bk < nb; ++bk) {
            int64_t k0, k1;
            ddk::dose_block_lags(bk, lb, k0, k1);
            k1 = std::min(k1, t1);
            const int64_t cost = dose_item_pairs(t0, t1, k0, k1);
            if (count >= kNoAllocMaxItems)
                return dd::fail(DD_EINVAL, "dd_per_probe_dose_noalloc: work list exceeds its fixed size");
            its[count++] = {cost, make_int2((int)t, (int)bk)};
        }
    }
    std::sort(its, its + count, [](const std::pair<int64_t, int2> &a, const std::pair<int64_t, int2> &b) {
        if (a.first != b.first) return a.first > b.first;
        return a.second.x != b.second.x ? a.second.x < b.second.x : a.second.y < b.second.y;
    });
    for (int k = 0; k < count; ++k) flat[k] = its[k].second;

    double *d_x = (double *)(scratch + o_x);
    double *d_y = d_x + n;
    float4 *d_f = (float4 *)(scratch + o_f);
    Rec *d_rec = (Rec *)(scratch + o_rec);
    Part *d_part = (Part *)(scratch + o_part);
    int2 *d_items = (int2 *)(scratch + o_items);
    // every scratch byte a kernel reads below is written earlier in this call, so
    // nothing left by a previous call can leak into the result
    DD_CUDA_TRY(cudaMemcpyAsync(d_x, scan->X.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, stream));
    DD_CUDA_TRY(cudaMemcpyAsync(d_y, scan->Y.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, stream));
    // float-float copy of the coordinates, built on the device from the FP64 ones
    ff_coords_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(d_x, d_y, n, d_f);
    DD_CUDA_TRY(cudaGetLastError());
    if (n >= 2) {
        ddk::lag_coef_kernel<Rec><<<(unsigned)((n + 31) / 32), 32, 0, stream>>>(n, scan->s, scan->kappa, d_rec);
        DD_CUDA_TRY(cudaGetLastError());
        DD_CUDA_TRY(cudaMemcpyAsync(d_items, flat, (size_t)count * sizeof(int2), cudaMemcpyHostToDevice, stream));
        DD_CUDA_TRY(launch_dose<Cfg>((unsigned)count, Cfg::kDosePPT, stream, d_x, d_y, n, d_rec, d_items, lb, d_part,
                                     d_f));
    }
    ddk::dose_reduce_kernel<Part><<<(unsigned)((n + 31) / 32), 32 * ddk::kDoseReduceSplit, 0, stream>>>(d_part, n, 0, n, TILE, lb, scan->pref, out);
    DD_CUDA_TRY(cudaGetLastError());
    // the work list above lives in this thread's fixed host storage, which the next call
    // on this thread rewrites: wait until the stream has copied it
    DD_CUDA_TRY(cudaStreamSynchronize(stream));
    return DD_OK;
}

}  // namespace

extern "C" dd_status dd_per_probe_dose_noalloc(const dd_scan *scan, dd_precision prec, double *out,
                                               void *cuda_stream) {
    dd::clear_error();
    if (!scan || !out) return dd::fail(DD_EINVAL, "dd_per_probe_dose_noalloc: NULL argument");
    if (prec != DD_FP64 && prec != DD_MIXED)
        return dd::fail(DD_EINVAL, "dd_per_probe_dose_noalloc: unknown precision");
    if (!scan->uniform)
        return dd::fail(DD_ENOTSUP, "dd_per_probe_dose_noalloc: needs a uniform dwell without flyback");
    if (scan->n > kNoAllocMaxVisits)
        return dd::fail(DD_EINVAL, "dd_per_probe_dose_noalloc: at most 16384 visits fit the 8 MiB built-in scratch");
    if (!dd::is_device_pointer(out))
        return dd::fail(DD_EINVAL, "dd_per_probe_dose_noalloc: out must be device memory");
    char *scratch = nullptr;
    dd_status st = noalloc_scratch(&scratch);
    if (st != DD_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    if (prec == DD_MIXED) return run_dose_noalloc<ddk::CfgMixed>(scan, out, stream, scratch);
    return run_dose_noalloc<ddk::CfgF64>(scan, out, stream, scratch);
}
