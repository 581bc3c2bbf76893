// dd_field_impl.cuh -- the field tile kernel shared by the field, dose and batch paths.
#pragma once
#include <cstdint>

#include "dd_e1.cuh"

namespace ddk {

// Per (snapshot, visit) coefficients.  FP32-mixed: alpha = -log2(e)/w1 (so that
// e^-a = 2^(rho^2 alpha)), dq = 1/w0 - 1/w1, q1 = 1/w1 and the moment coefficients
// c_0..c_8 (c_0 = ln(w1/w0)); 48 bytes, read as three 16-byte vectors.
struct __align__(16) RecF32 {
    static constexpr int kTerms = 9;
    float alpha, dq, q1;
    float c[kTerms];
};
static_assert(sizeof(RecF32) == 48, "RecF32 layout");

// FP64: q1, dq and c_0..c_15; 144 bytes.
struct __align__(16) RecF64 {
    static constexpr int kTerms = 16;
    double q1, dq;
    double c[kTerms];
};
static_assert(sizeof(RecF64) == 144, "RecF64 layout");

template <typename Rec>
struct RecTraits;

// Largest h handled by the moment series: its truncation after c_8 (FP32) or c_15
// (FP64) is below e^h h^(M+1)/(M+1)! = 9e-9 resp. 1.2e-18 relative at h = 1/2.
constexpr float kHMaxF = 0.5f;
constexpr double kHMaxD = 0.5;

// One pair term E1(a) - E1(b), a = rho^2 q1, b = a + rho^2 dq, FP32 arithmetic.
__device__ __forceinline__ float pair_term(float r2, const RecF32 &R) {
    const float a = r2 * R.q1;
    const float h = r2 * R.dq;
    if (a >= 87.0f) return 0.0f;                  // e^-a below the FP32 normal range
    if (h <= kHMaxF) {
        float p = R.c[8];
#pragma unroll
        for (int m = 7; m >= 0; --m) p = fmaf(p, h, R.c[m]);
        return ex2_approx(r2 * R.alpha) * p;
    }
    return e1diff_general_f32(a, h, R.c[0]);
}

// The same in FP64.
__device__ __forceinline__ double pair_term(double r2, const RecF64 &R) {
    const double a = r2 * R.q1;
    const double h = r2 * R.dq;
    if (a >= 745.0) return 0.0;
    if (h <= kHMaxD) {
        double p = R.c[15];
#pragma unroll
        for (int m = 14; m >= 0; --m) p = fma(p, h, R.c[m]);
        return exp(-a) * p;
    }
    return e1diff_general_f64(a, h, R.c[0]);
}

// Tile configurations.  kThreads threads x kPPT points per thread form a point tile;
// kTCH snapshots share each staged visit; kSTILE visits are staged per round; kSB
// visits form one work item's block; FP32 partial sums are folded into FP64 every
// kFlush visits.
struct CfgMixed {
    using Rec = RecF32;
    using Real = float;
    static constexpr int kThreads = 128, kPPT = 4, kTCH = 4, kSTILE = 64, kSB = 512, kFlush = 32;
    static constexpr const char *kFieldName = "field_mixed", *kCoefName = "coef_mixed",
                                *kDoseName = "dose_mixed", *kLagCoefName = "lag_coef_mixed";
};
struct CfgF64 {
    using Rec = RecF64;
    using Real = double;
    static constexpr int kThreads = 128, kPPT = 2, kTCH = 4, kSTILE = 32, kSB = 512, kFlush = 1 << 30;
    static constexpr const char *kFieldName = "field_fp64", *kCoefName = "coef_fp64",
                                *kDoseName = "dose_fp64", *kLagCoefName = "lag_coef_fp64";
};

// Shared memory of one tile pass: kSTILE staged visits (coordinates relative to the
// tile origin) and their records for TCH snapshots.
template <typename Cfg, int TCH>
struct TileSmem {
    typename Cfg::Real x[Cfg::kSTILE], y[Cfg::kSTILE];
    __align__(16) typename Cfg::Rec rec[TCH][Cfg::kSTILE];
};

// Sum of pair terms over visits [s_begin, s_end) for the point tile starting at point
// tile0 and TCH snapshots:  partial[jc * part_stride + p] = sum_{i < na[jc]} term(p, i, jc)
// for jc < nj.  rec points at the record row of the first snapshot (row stride
// rec_stride); records exist for visits below na[jc].  All threads of the CTA call it.
template <typename Cfg, int TCH>
__device__ __forceinline__ void field_tile(TileSmem<Cfg, TCH> &sm, const double *__restrict__ srcX,
                                           const double *__restrict__ srcY, const double *__restrict__ X,
                                           const double *__restrict__ Y, int64_t n_pts, int64_t tile0,
                                           const typename Cfg::Rec *__restrict__ rec, int64_t rec_stride,
                                           const int (&na)[TCH], int nj, int s_begin, int s_end,
                                           double *__restrict__ partial, int64_t part_stride) {
    using Rec = typename Cfg::Rec;
    using Real = typename Cfg::Real;
    constexpr int NT = Cfg::kThreads, PPT = Cfg::kPPT, STILE = Cfg::kSTILE;
    constexpr int RV = sizeof(Rec) / 16;   // 16-byte vectors per record
    const int tid = threadIdx.x;

    // points relative to the tile's first point (keeps FP32 differences exact-ish)
    const double cx = X[tile0], cy = Y[tile0];
    Real px[PPT], py[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int64_t p = tile0 + k * NT + tid;
        px[k] = p < n_pts ? (Real)(X[p] - cx) : (Real)0;
        py[k] = p < n_pts ? (Real)(Y[p] - cy) : (Real)0;
    }
    Real acc[TCH][PPT];
    double tot[TCH][PPT];
#pragma unroll
    for (int jc = 0; jc < TCH; ++jc)
#pragma unroll
        for (int k = 0; k < PPT; ++k) { acc[jc][k] = 0; tot[jc][k] = 0.0; }

    for (int s0 = s_begin; s0 < s_end; s0 += STILE) {
        const int cnt = min(STILE, s_end - s0);
        __syncthreads();
        for (int i = tid; i < cnt; i += NT) {
            sm.x[i] = (Real)(srcX[s0 + i] - cx);
            sm.y[i] = (Real)(srcY[s0 + i] - cy);
        }
#pragma unroll
        for (int jc = 0; jc < TCH; ++jc) {
            const float4 *row = reinterpret_cast<const float4 *>(rec + (int64_t)jc * rec_stride + s0);
            const int lim = na[jc] - s0;           // records exist for visits below n_active
            float4 *dst = reinterpret_cast<float4 *>(&sm.rec[jc][0]);
            for (int v = tid; v < cnt * RV; v += NT)
                dst[v] = (v / RV < lim) ? row[v] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        for (int s = 0; s < cnt; ++s) {
            const Real sx = sm.x[s], sy = sm.y[s];
            Real r2[PPT];
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const Real dx = px[k] - sx, dy = py[k] - sy;
                r2[k] = dx * dx + dy * dy;
            }
            const int gs = s0 + s;
#pragma unroll
            for (int jc = 0; jc < TCH; ++jc) {
                if (gs < na[jc]) {
                    const Rec &R = sm.rec[jc][s];
#pragma unroll
                    for (int k = 0; k < PPT; ++k) acc[jc][k] += pair_term(r2[k], R);
                }
            }
            if (Cfg::kFlush < STILE && (s % Cfg::kFlush) == Cfg::kFlush - 1) {
#pragma unroll
                for (int jc = 0; jc < TCH; ++jc)
#pragma unroll
                    for (int k = 0; k < PPT; ++k) { tot[jc][k] += (double)acc[jc][k]; acc[jc][k] = 0; }
            }
        }
#pragma unroll
        for (int jc = 0; jc < TCH; ++jc)
#pragma unroll
            for (int k = 0; k < PPT; ++k) { tot[jc][k] += (double)acc[jc][k]; acc[jc][k] = 0; }
    }
#pragma unroll
    for (int jc = 0; jc < TCH; ++jc) {
        if (jc >= nj) continue;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int64_t p = tile0 + k * NT + tid;
            if (p < n_pts) partial[(int64_t)jc * part_stride + p] = tot[jc][k];
        }
    }
}

// One work item per CTA: item = (point tile, snapshot chunk, visit block).
// partial[(block * n_tg + j) * n_pts + p] receives sum_{i in block, i < nact[j]} pair_term.
template <typename Cfg>
__global__ void __launch_bounds__(Cfg::kThreads)
field_kernel(const double *__restrict__ srcX, const double *__restrict__ srcY,
             const double *__restrict__ X, const double *__restrict__ Y, int64_t n_pts,
             const typename Cfg::Rec *__restrict__ rec, int64_t rec_stride,
             const int *__restrict__ nact, const int4 *__restrict__ items, int n_tg, int sb,
             double *__restrict__ partial) {
    constexpr int TCH = Cfg::kTCH;
    __shared__ TileSmem<Cfg, TCH> sm;
    const int4 item = items[blockIdx.x];
    const int j0 = item.y * TCH;
    int na[TCH];
    int nmax = 0;
#pragma unroll
    for (int jc = 0; jc < TCH; ++jc) {
        na[jc] = (j0 + jc < n_tg) ? nact[j0 + jc] : 0;
        nmax = max(nmax, na[jc]);
    }
    const int s_begin = item.z * sb;
    const int s_end = min(s_begin + sb, nmax);
    field_tile<Cfg, TCH>(sm, srcX, srcY, X, Y, n_pts, (int64_t)item.x * (Cfg::kThreads * Cfg::kPPT),
                         rec + (int64_t)j0 * rec_stride, rec_stride, na, min(TCH, n_tg - j0), s_begin,
                         s_end, partial + ((int64_t)item.z * n_tg + j0) * n_pts, n_pts);
}

}  // namespace ddk
