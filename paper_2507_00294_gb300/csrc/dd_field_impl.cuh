// dd_field_impl.cuh -- the field tile kernel shared by the field, dose and batch paths.
#pragma once
#include <cstdint>
#include <type_traits>

#include "dd_e1.cuh"

namespace ddk {

// Per (snapshot, visit) coefficients, FP32-mixed, 80 bytes read as five 16-byte vectors.
// The FP32 path evaluates the pair term as one power of two,
//   E1(a) - E1(b) = e^-a P(h),  P(h) = sum_m c_m h^m,  h = rho^2 dq,  a = rho^2 q1,
//   log2(e^-a P(h)) = g_0 - log2(e) a + log2(e) sum_{m>=1} l_m h^m,
// where g_0 = log2(c_0), c_0 = ln(w1/w0), and l_m are the coefficients of the power series
// of ln(P(h)/c_0) (the cumulants of the moment weight r/(1+rs) on [0,1], up to sign and
// factorials; |l_m| <= 0.5, 0.042, 3.9e-3, 4.0e-4, 5.3e-5, 9.1e-6, 1.3e-6, 1.7e-7,
// 3.1e-8 for m = 1..9 over r in [1e-6, 1e6], i.e. about (2 pi)^-m).  Layout:
//   v0 = (g_0, g_1x, g_2x, g_3x),  v1 = (g_4x, dq, q1, c_0),  v2 = (k_1, k_2, k_3, k_4),
//   v3 = (k_5, k_6, k_7, k_8),      v4 = (k_9, k_10, k_11, k_12)
// with the exponent's coefficients in rho^2 for the low degrees,
//   g_1x = log2(e) (l_1 dq - q1),  g_mx = log2(e) l_m dq^m  (m = 2..4),
// and in h for the high degrees (the -a term folded in as -h/r, since a = h/r),
//   k_1 = log2(e) (l_1 - 1/r),  k_m = log2(e) l_m  (m = 2..12).
// A snapshot for which the visit has not started carries the zero record, g_0 = -inf and
// everything else 0: every path then yields 2^-inf = 0.
struct __align__(16) RecF32 {
    float4 v0, v1, v2, v3, v4;
    __device__ __forceinline__ float g0() const { return v0.x; }
    __device__ __forceinline__ float dq() const { return v1.y; }
    __device__ __forceinline__ float q1() const { return v1.z; }
    __device__ __forceinline__ float c0() const { return v1.w; }
    // exponent coefficient of (rho^2)^m, m = 1..4
    __device__ __forceinline__ float gx(int m) const {
        return m == 1 ? v0.y : m == 2 ? v0.z : m == 3 ? v0.w : v1.x;
    }
    // exponent coefficient of h^m, m = 1..12
    __device__ __forceinline__ float k(int m) const {
        switch (m) {
            case 1: return v2.x; case 2: return v2.y; case 3: return v2.z; case 4: return v2.w;
            case 5: return v3.x; case 6: return v3.y; case 7: return v3.z; case 8: return v3.w;
            case 9: return v4.x; case 10: return v4.y; case 11: return v4.z; default: return v4.w;
        }
    }
};
static_assert(sizeof(RecF32) == 80, "RecF32 layout");

// FP64: q1, dq and c_0..c_15; 144 bytes.
struct __align__(16) RecF64 {
    static constexpr int kTerms = 16;
    double q1, dq;
    double c[kTerms];
};
static_assert(sizeof(RecF64) == 144, "RecF64 layout");

template <typename Rec>
struct RecTraits;

// Largest h of each FP32 class: the truncated exponent series of degree d stays within
// 2.5e-7 of ln(P(h)/c_0) for every r in [1e-12, 1e6] (checked against FP64 adaptive
// quadrature of P(h), relative 1e-13, at half-decade steps of r: worst 2.49e-7 at degree 2;
// about four FP32 roundings of the term, below the exponent's own rounding for all but the
// largest terms): degree 2 up to h = 0.04, 4 up to 0.33, 8 up to 1.25 and 12 up to 2.0.
// FP64: the moment polynomial of degree 15 up to h = 1/2 (1.2e-18).
constexpr float kL2H = 0.04f, kL4H = 0.33f, kL8H = 1.25f, kL12H = 2.0f;
constexpr double kHMaxD = 0.5;
// The rho^2 forms of degree 2 and 4 need dq^4 and dq^3 in the FP32 normal range; records
// with a smaller dq (far beyond any scan's duration) take the h forms.
constexpr float kMinDqX = 1.0e-8f;

// Degree-D exponent of one pair: rho^2 form for D = 2, 4, h form for D = 8, 12.
template <int D, typename RV>
__device__ __forceinline__ float log_exponent(float r2, const RV &R) {
    if (D == 2) return fmaf(fmaf(R.gx(2), r2, R.gx(1)), r2, R.g0());
    if (D == 4)
        return fmaf(fmaf(fmaf(fmaf(R.gx(4), r2, R.gx(3)), r2, R.gx(2)), r2, R.gx(1)), r2, R.g0());
    const float h = r2 * R.dq();
    float p = R.k(D);
#pragma unroll
    for (int m = D - 1; m >= 1; --m) p = fmaf(p, h, R.k(m));
    return fmaf(p, h, R.g0());
}

template <int D, typename RV>
__device__ __forceinline__ float log_term(float r2, const RV &R) {
    return ex2_approx(log_exponent<D>(r2, R));
}

// One pair term E1(a) - E1(b), a = rho^2 q1, b = a + rho^2 dq, FP32 arithmetic, with a
// per-lane regime test: zero (a >= 87: below the FP32 normal range), the degree-12
// exponent series (h <= 2.0), or the two E1 values (dd_e1.cuh).
template <typename RV>
__device__ __forceinline__ float pair_term(float r2, const RV &R) {
    const float a = r2 * R.q1();
    const float h = r2 * R.dq();
    if (a >= 87.0f) return 0.0f;
    if (h <= kL12H) return log_term<12>(r2, R);
    return e1diff_general_f32(a, h, R.c0());
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

// FP64 moment term of degree D (truncation e^{2h} h^{D+1}/(D+1)! <= 1e-17 at the class
// limits below): e^-a times Horner in h over c_0..c_D.
constexpr double kDeg4HD = 1.0e-3, kDeg8HD = 5.2e-2, kDeg11HD = 0.19;
template <int D>
__device__ __forceinline__ double moment_term_f64(double r2, const RecF64 &R) {
    const double h = r2 * R.dq;
    double p = R.c[D];
#pragma unroll
    for (int m = D - 1; m >= 0; --m) p = fma(p, h, R.c[m]);
    return exp(-r2 * R.q1) * p;
}

// Tile configurations.  kThreads threads x kPPT points per thread form a point tile;
// kTCH snapshots share each staged visit; kSTILE visits are staged per round; kSB
// visits form one work item's block; FP32 partial sums are folded into FP64 every
// kFlush visits; kDoseLB lags form the dose kernel's largest work-item block.
struct CfgMixed {
    using Rec = RecF32;
    using Real = float;
    static constexpr int kThreads = 128, kPPT = 4, kTCH = 4, kSTILE = 32, kSB = 512, kFlush = 32;
    static constexpr int kMinBlocks = 8;     // 32 warps per SM: at most 64 registers, 12 KB shared
    static constexpr int kCarveout = 58;     // percent of the L1/shared array as shared memory (132 KB)
    static constexpr int kDoseLB = 512;      // largest lag block of the dose kernel
    static constexpr int kDoseSTILE = 64;    // lags staged per round by the dose kernel
    static constexpr int kDosePPT = 2;       // targets per thread in the dose kernel (256-target tiles)
    static constexpr int kDoseLBMin = 32;    // smallest lag block of the dose kernel
    static constexpr const char *kFieldName = "field_mixed", *kCoefName = "coef_mixed",
                                *kDoseName = "dose_mixed", *kLagCoefName = "lag_coef_mixed";
};
struct CfgF64 {
    using Rec = RecF64;
    using Real = double;
    static constexpr int kThreads = 128, kPPT = 2, kTCH = 4, kSTILE = 32, kSB = 512, kFlush = 1 << 30;
    static constexpr int kMinBlocks = 1;
    static constexpr int kCarveout = (int)cudaSharedmemCarveoutMaxShared;
    static constexpr int kDoseLB = 512;
    static constexpr int kDoseSTILE = 32;
    static constexpr int kDosePPT = 2;
    static constexpr int kDoseLBMin = 64;
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

// ---- FP32-mixed tile with warp-uniform regime selection -------------------------
//
// For every staged visit, each warp bounds its own a and h from the bounding box of its
// points (one visit per lane): a_min = rho2_min q1 and h_max = rho2_max dq.
// Per snapshot that gives a class: skip (a_min >= 87: every term is below the FP32 normal
// range), the smallest exponent-series degree whose range holds h_max (2, 4, 8, 12), or
// the per-lane regime test of pair_term.  When every snapshot of the chunk is on degree 2,
// or on degree 2 or 4, the warp runs the whole visit on that degree, two snapshots per
// f32x2 instruction; otherwise one snapshot at a time, each at its own class.  Lanes whose
// own a is 87 or more inside a series class add terms below 2e-38, flushed to zero once
// they leave the normal range, so the series paths need no per-lane test.
enum : uint32_t { kCodeSkip = 0, kCodeD2 = 1, kCodeD4 = 2, kCodeD8 = 3, kCodeD12 = 4, kCodeGeneral = 5 };
// classes are packed 3 bits per snapshot in one word (up to 10 snapshots)
constexpr uint32_t kCodeBits = 3, kCodeMask = 7;
// per (warp, visit): all snapshots skipped / all on degree 2 / all on degree <= 4 / mixed
enum : uint32_t { kModeSkip = 0, kModeAllD2 = 1, kModeAllD4 = 2, kModePerSnapshot = 3 };

// Class of one (snapshot, visit) record for h_max and a_min over a set of pairs.
__device__ __forceinline__ uint32_t series_class(float hmax, float amin, float dq) {
    const bool x_ok = dq >= kMinDqX;
    return amin >= 87.0f ? kCodeSkip
         : (hmax <= kL2H && x_ok) ? kCodeD2
         : (hmax <= kL4H && x_ok) ? kCodeD4
         : hmax <= kL8H ? kCodeD8
         : hmax <= kL12H ? kCodeD12 : kCodeGeneral;
}

// acc[k] (one half of each pair: H = 0 for .x, 1 for .y) += term of point k
template <int D, int PPT, int H>
__device__ __forceinline__ void moment_pass(float2 (&acc)[PPT], const float (&r2)[PPT], const RecF32 &R) {
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const float t = log_term<D>(r2[k], R);
        if (H) acc[k].y += t; else acc[k].x += t;
    }
}

// One snapshot at PPT points, the h form of degree D (8, 12) on f32x2 instructions over
// point pairs: acc[m] += (2^G(r_2m), 2^G(r_2m+1)), each half rounded as log_exponent<D>
// rounds it.
template <int D, int PPT>
__device__ __forceinline__ void point_pass_h2(float2 (&acc)[PPT], const float (&r2)[PPT], const RecF32 &R) {
    const float2 dq = make_float2(R.dq(), R.dq()), g0 = make_float2(R.g0(), R.g0());
    float2 h[PPT / 2], p[PPT / 2];
#pragma unroll
    for (int m = 0; m < PPT / 2; ++m) {
        h[m] = __fmul2_rn(make_float2(r2[2 * m], r2[2 * m + 1]), dq);
        p[m] = make_float2(R.k(D), R.k(D));
    }
#pragma unroll
    for (int j = D - 1; j >= 1; --j) {
        const float2 c = make_float2(R.k(j), R.k(j));
#pragma unroll
        for (int m = 0; m < PPT / 2; ++m) p[m] = __ffma2_rn(p[m], h[m], c);
    }
#pragma unroll
    for (int m = 0; m < PPT / 2; ++m) {
        const float2 g = __ffma2_rn(p[m], h[m], g0);
        acc[m] = __fadd2_rn(acc[m], make_float2(ex2_approx(g.x), ex2_approx(g.y)));
    }
}

// The zero record's leading vector (g_0 = -inf): a snapshot for which the visit has not
// started, or a padding snapshot, adds 2^-inf = 0 on every path.
__device__ __forceinline__ float4 zero_rec_v0() { return make_float4(-INFINITY, 0.f, 0.f, 0.f); }

// Shared memory of the FP32-mixed tile: the staged visits' coordinates, the running sums,
// and
//  * snapshot-pair tiles (even TCH): the low-degree exponent coefficients of a visit,
//    laid out so that one f32x2 instruction evaluates the two snapshots of a pair
//    (2P, 2P+1) and a degree-2 visit needs few 16-byte loads:
//      pa[P] = (g_0, g_0', g_1x, g_1x') of pair P,  gm[m - 2] = g_mx of the TCH snapshots
//    (m = 2, 3, 4), and (dq, q1) of every snapshot for the classification (the minority
//    classes read whole records from global memory);
//  * one-snapshot tiles: the leading record vectors and whole records.
template <typename Cfg, int TCH, bool kPacked = TCH % 2 == 0>
struct TileSmemMixed;

template <typename Cfg, int TCH>
struct TileSmemMixed<Cfg, TCH, true> {
    static constexpr int NP = TCH / 2, ST = Cfg::kSTILE;
    static_assert(TCH == 4, "gm holds the coefficients of four snapshots as one vector");
    float run[TCH * Cfg::kPPT][Cfg::kThreads];          // per-thread running sums over stages
    float4 xy[ST];                                      // (-x, -x, -y, -y) of each staged visit
    float4 pa[NP][ST];
    float4 gm[3][ST];
    float2 cls[TCH][ST];                                // (dq, q1)
};

template <typename Cfg, int TCH>
struct TileSmemMixed<Cfg, TCH, false> {
    float run[TCH * Cfg::kPPT][Cfg::kThreads];
    float4 xy[Cfg::kSTILE];
    float4 lo[TCH][Cfg::kSTILE];                        // record vector v0: (g_0, g_1x, g_2x, g_3x)
    float4 hi[TCH][Cfg::kSTILE];                        // record vector v1: (g_4x, dq, q1, c_0)
    __align__(16) RecF32 rec[Cfg::kSTILE];              // whole records (minority classes)
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Coordinate difference a - b of two float-float values (x_hi, x_lo, y_hi, y_lo): FP32
// arithmetic only, within about one FP32 rounding of the exact difference.
__device__ __forceinline__ float2 ff_diff(const float4 &a, const float4 &b) {
    return make_float2((a.x - b.x) + (a.y - b.y), (a.z - b.z) + (a.w - b.w));
}

// Bounds of rho^2 between a visit at (sx, sy) and any point of the box [bx0, bx1] x
// [by0, by1], widened (relative 1e-4, absolute 1e-6) to cover the FP32 rounding of each
// pair's own rho^2.
__device__ __forceinline__ void box_rho2(float sx, float sy, float bx0, float bx1, float by0, float by1,
                                         float &r2min, float &r2max) {
    const float dx1 = fmaxf(fabsf(sx - bx0), fabsf(sx - bx1));
    const float dy1 = fmaxf(fabsf(sy - by0), fabsf(sy - by1));
    const float dx0 = fmaxf(0.0f, fmaxf(bx0 - sx, sx - bx1));
    const float dy0 = fmaxf(0.0f, fmaxf(by0 - sy, sy - by1));
    r2max = (dx1 * dx1 + dy1 * dy1) * 1.0001f + 1e-6f;
    r2min = (dx0 * dx0 + dy0 * dy0) * 0.9999f;
}

// Points in a tile are held as an integer offset from the tile's integer origin plus a
// fraction (|f| <= 1/2 pitch): P.i = (x_2m, x_2m+1) - origin (exact integers), P.f the
// fractions, and likewise in y.  Visits sit on the integer probe grid, so visit minus
// origin is an exact integer too: dx = (P.i - visit) + P.f is within 2^-24 |dx| + 2^-25
// pitch of the exact difference (the final rounding and the fraction's own) wherever the
// points lie.  (One FP32 offset per point
// would carry an error of 2^-24 times the distance to the tile origin instead, which at a
// few thousand pitches and a sub-pitch probe is a 1e-3 error in e^-a.)
struct PointPair {
    float2 xi, xf, yi, yf;
};

// rho^2 of PPT points (pairs m: points 2m, 2m+1) to the visit nxy = (-x, -x, -y, -y)
// (integer, relative to the tile origin) on f32x2 instructions.  split (uniform over the
// CTA): add the fractions; otherwise P.xi, P.yi hold the whole offsets, which are then exact
// in FP32 (points on the probe grid, its halves, quarters, ...), and the two adds are skipped.
template <int PPT>
__device__ __forceinline__ void rho2_points(const PointPair (&P)[PPT / 2], const float4 &nxy, bool split,
                                            float (&r2)[PPT]) {
    float2 dx[PPT / 2], dy[PPT / 2];
#pragma unroll
    for (int m = 0; m < PPT / 2; ++m) {
        dx[m] = __fadd2_rn(P[m].xi, f2(nxy.x, nxy.y));
        dy[m] = __fadd2_rn(P[m].yi, f2(nxy.z, nxy.w));
    }
    if (split) {
#pragma unroll
        for (int m = 0; m < PPT / 2; ++m) {
            dx[m] = __fadd2_rn(dx[m], P[m].xf);
            dy[m] = __fadd2_rn(dy[m], P[m].yf);
        }
    }
#pragma unroll
    for (int m = 0; m < PPT / 2; ++m) {
        const float2 q = __ffma2_rn(dx[m], dx[m], __fmul2_rn(dy[m], dy[m]));
        r2[2 * m] = q.x;
        r2[2 * m + 1] = q.y;
    }
}

// srcF: visit coordinates, ptsF: point coordinates, both float-float in pitch units.
template <typename Cfg, int TCH, typename Part>
__device__ __forceinline__ void field_tile_mixed(TileSmemMixed<Cfg, TCH> &sm, const float4 *__restrict__ srcF,
                                                 const float4 *__restrict__ ptsF, int64_t n_pts, int64_t tile0,
                                                 const RecF32 *const (&rows)[TCH], const int (&na)[TCH], int nj,
                                                 int s_begin, int s_end, Part *__restrict__ partial,
                                                 int64_t part_stride) {
    constexpr int NT = Cfg::kThreads, PPT = Cfg::kPPT, STILE = Cfg::kSTILE;
    constexpr bool kPacked = TCH % 2 == 0;       // snapshot pairs on f32x2 instructions
    constexpr bool kSingle = TCH == 1;           // one snapshot: point pairs on f32x2 instead
    static_assert(kPacked || kSingle, "snapshot chunks of one or an even number");
    constexpr int NP = (TCH + 1) / 2;            // accumulator pairs (acc[0][k / 2] holds
                                                 // points (k, k + 1) when kSingle)
    static_assert(PPT % 2 == 0, "points are processed in pairs");
    const int tid = threadIdx.x, lane = tid & 31;

    // coordinates relative to the integer grid position nearest the tile's first point:
    // integer offset + fraction per point (PointPair), exact integers for the visits;
    // points k = 2m, 2m+1 in one pair
    const float4 org = ptsF[tile0];
    const float ox = rintf(org.x), oy = rintf(org.z);
    PointPair pp[PPT / 2];
    float bx0 = 3.0e38f, bx1 = -3.0e38f, by0 = 3.0e38f, by1 = -3.0e38f;
    bool exact = true;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int64_t p = tile0 + k * NT + tid;
        const float4 q = p < n_pts ? ptsF[p] : org;
        const float ix = rintf(q.x), iy = rintf(q.z);
        const float fx = (q.x - ix) + q.y, fy = (q.z - iy) + q.w;     // q.x - ix is exact
        const float xi = ix - ox, yi = iy - oy;                        // exact integers
        if (k & 1) { pp[k >> 1].xi.y = xi; pp[k >> 1].xf.y = fx; pp[k >> 1].yi.y = yi; pp[k >> 1].yf.y = fy; }
        else       { pp[k >> 1].xi.x = xi; pp[k >> 1].xf.x = fx; pp[k >> 1].yi.x = yi; pp[k >> 1].yf.x = fy; }
        const float x = xi + fx, y = yi + fy;
        // (x - xi) is computed exactly (|fx| <= 1/2, xi an integer), so it equals fx only
        // when x lost no bit of xi + fx
        exact = exact && (x - xi) == fx && (y - yi) == fy;
        bx0 = fminf(bx0, x); bx1 = fmaxf(bx1, x);
        by0 = fminf(by0, y); by1 = fmaxf(by1, y);
    }
    // one vote of the CTA: split offsets only where some point of the tile needs them
    const bool split = __syncthreads_or(!exact) != 0;
    if (!split) {
#pragma unroll
        for (int m = 0; m < PPT / 2; ++m) {
            pp[m].xi = __fadd2_rn(pp[m].xi, pp[m].xf);
            pp[m].yi = __fadd2_rn(pp[m].yi, pp[m].yf);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bx0 = fminf(bx0, __shfl_xor_sync(0xffffffffu, bx0, o));
        bx1 = fmaxf(bx1, __shfl_xor_sync(0xffffffffu, bx1, o));
        by0 = fminf(by0, __shfl_xor_sync(0xffffffffu, by0, o));
        by1 = fmaxf(by1, __shfl_xor_sync(0xffffffffu, by1, o));
    }

    // per (snapshot, point): FP32 sum of the current stage of STILE visits in registers
    // (acc[jc / 2][k], .x for even jc, .y for odd), added after each stage to an FP32
    // running sum in shared memory (sm.run, one column per thread: conflict-free) (the
    // dispatcher keeps blocks at or below 32 stages, so that sum adds at most 32 u = 2e-6
    // relative error), converted to FP64 at the end of the item.
    float2 acc[NP][PPT];
#pragma unroll
    for (int m = 0; m < NP; ++m)
#pragma unroll
        for (int k = 0; k < PPT; ++k) acc[m][k] = f2(0.0f, 0.0f);
#pragma unroll
    for (int jc = 0; jc < TCH; ++jc)
#pragma unroll
        for (int k = 0; k < PPT; ++k) sm.run[jc * PPT + k][tid] = 0.0f;

    constexpr int NCW = (STILE + 31) / 32;
    for (int s0 = s_begin; s0 < s_end; s0 += STILE) {
        const int cnt = min(STILE, s_end - s0);
        __syncthreads();
        for (int i = tid; i < cnt; i += NT) {
            // probe positions are integers in pitch units: visit - origin is exact
            const float4 v = srcF[s0 + i];
            const float dx = (v.x - ox) + v.y, dy = (v.z - oy) + v.w;
            sm.xy[i] = make_float4(-dx, -dx, -dy, -dy);
        }
        // records; a snapshot for which the visit has not started gets the zero record,
        // whose terms are 0
        constexpr int RV = sizeof(RecF32) / 16;
        constexpr int NV = kSingle ? RV : 2;          // record vectors staged per visit
#pragma unroll
        for (int jc = 0; jc < TCH; ++jc) {
            const float4 *row = reinterpret_cast<const float4 *>(rows[jc] + s0);
            const int lim = na[jc] - s0;
            for (int v = tid; v < cnt * NV; v += NT) {
                const int i = v / NV, q = v - i * NV;
                const float4 r = i < lim ? row[i * RV + q] : (q == 0 ? zero_rec_v0() : make_float4(0.f, 0.f, 0.f, 0.f));
                if constexpr (kPacked) {
                    // half jc & 1 of snapshot pair jc / 2, element jc of the g_mx vectors
                    if (q == 0) {
                        float *a = reinterpret_cast<float *>(&sm.pa[jc >> 1][i]) + (jc & 1);
                        a[0] = r.x; a[2] = r.y;
                        reinterpret_cast<float *>(&sm.gm[0][i])[jc] = r.z;
                        reinterpret_cast<float *>(&sm.gm[1][i])[jc] = r.w;
                    } else {
                        reinterpret_cast<float *>(&sm.gm[2][i])[jc] = r.x;
                        sm.cls[jc][i] = make_float2(r.y, r.z);
                    }
                } else {
                    if (q == 0) sm.lo[jc][i] = r;
                    else if (q == 1) sm.hi[jc][i] = r;
                    reinterpret_cast<float4 *>(&sm.rec[i])[q] = r;
                }
            }
        }
        __syncthreads();                   // staged coordinates and records visible
        // Class words: lane i of each warp classifies staged visits i, i + 32, .. against
        // its own warp's box.  Per snapshot: skip (a_min >= 87: every term is below the
        // FP32 normal range), the smallest exponent-series degree whose range holds h_max,
        // or the per-lane regime test.  A snapshot for which the visit has not started
        // counts as degree 2 for the warp's mode (its zero record yields 0 there) and as
        // skip for the one-snapshot-at-a-time path (which reads records from global memory).
        uint32_t my_word[NCW], my_mode[NCW];
#pragma unroll
        for (int cw = 0; cw < NCW; ++cw) {
            const int i = cw * 32 + lane;
            my_word[cw] = 0;
            my_mode[cw] = kModeSkip;
            if (i < cnt) {
                float r2min, r2max;
                box_rho2(-sm.xy[i].x, -sm.xy[i].z, bx0, bx1, by0, by1, r2min, r2max);
                uint32_t codes = 0, cmin = kCodeGeneral, cmax = kCodeSkip;
                bool any = false;
#pragma unroll
                for (int jc = 0; jc < TCH; ++jc) {
                    uint32_t c = kCodeD2, code = kCodeSkip;
                    if (s0 + i < na[jc]) {
                        float dq, q1;
                        if constexpr (kPacked) { const float2 h = sm.cls[jc][i]; dq = h.x; q1 = h.y; }
                        else { const float4 h = sm.hi[jc][i]; dq = h.y; q1 = h.z; }
                        c = code = series_class(r2max * dq, r2min * q1, dq);
                        any = any || c != kCodeSkip;
                    }
                    cmin = min(cmin, c);
                    cmax = max(cmax, c);
                    codes |= code << (kCodeBits * jc);
                }
                my_word[cw] = codes;
                my_mode[cw] = !any ? kModeSkip
                            : (cmin >= kCodeD2 && cmax == kCodeD2) ? kModeAllD2
                            : (cmin >= kCodeD2 && cmax == kCodeD4) ? kModeAllD4 : kModePerSnapshot;
            }
        }
        // The warp's visits by mode, as bit masks (bit b of word cw: staged visit 32 cw + b);
        // each mode runs its visits in a loop of its own, without per-visit dispatch.
#pragma unroll
        for (int cw = 0; cw < NCW; ++cw) {
            const uint32_t m2 = __ballot_sync(0xffffffffu, my_mode[cw] == kModeAllD2);
            const uint32_t m4 = __ballot_sync(0xffffffffu, my_mode[cw] == kModeAllD4);
            const uint32_t mp = __ballot_sync(0xffffffffu, my_mode[cw] == kModePerSnapshot);
            if constexpr (kPacked) {
                // every snapshot of the chunk on degree 2 (then on degree 4): both
                // snapshots of a pair in one f32x2 instruction,
                //   term = 2^(g_0 + g_1x r + g_2x r^2 [+ g_3x r^3 + g_4x r^4]),  r = rho^2;
                // the coefficient vectors first, so their shared-memory latency overlaps
                for (uint32_t m = m2; m; m &= m - 1) {
                    const int s = cw * 32 + __ffs(m) - 1;
                    float4 va[NP];
#pragma unroll
                    for (int P = 0; P < NP; ++P) va[P] = sm.pa[P][s];
                    const float4 g2 = sm.gm[0][s];
                    const float2 g2p[2] = {f2(g2.x, g2.y), f2(g2.z, g2.w)};
                    float r2[PPT];
                    rho2_points<PPT>(pp, sm.xy[s], split, r2);
#pragma unroll
                    for (int P = 0; P < NP; ++P)
#pragma unroll
                        for (int k = 0; k < PPT; ++k) {
                            const float2 r = f2(r2[k], r2[k]);
                            const float2 g = __ffma2_rn(__ffma2_rn(g2p[P], r, f2(va[P].z, va[P].w)), r,
                                                        f2(va[P].x, va[P].y));
                            acc[P][k] = __fadd2_rn(acc[P][k], f2(ex2_approx(g.x), ex2_approx(g.y)));
                        }
                }
                for (uint32_t m = m4; m; m &= m - 1) {
                    const int s = cw * 32 + __ffs(m) - 1;
                    float4 va[NP];
#pragma unroll
                    for (int P = 0; P < NP; ++P) va[P] = sm.pa[P][s];
                    const float4 g2 = sm.gm[0][s], g3 = sm.gm[1][s], g4 = sm.gm[2][s];
                    const float2 g2p[2] = {f2(g2.x, g2.y), f2(g2.z, g2.w)};
                    const float2 g3p[2] = {f2(g3.x, g3.y), f2(g3.z, g3.w)};
                    const float2 g4p[2] = {f2(g4.x, g4.y), f2(g4.z, g4.w)};
                    float r2[PPT];
                    rho2_points<PPT>(pp, sm.xy[s], split, r2);
#pragma unroll
                    for (int P = 0; P < NP; ++P)
#pragma unroll
                        for (int k = 0; k < PPT; ++k) {
                            const float2 r = f2(r2[k], r2[k]);
                            float2 g = __ffma2_rn(g4p[P], r, g3p[P]);
                            g = __ffma2_rn(g, r, g2p[P]);
                            g = __ffma2_rn(g, r, f2(va[P].z, va[P].w));
                            g = __ffma2_rn(g, r, f2(va[P].x, va[P].y));
                            acc[P][k] = __fadd2_rn(acc[P][k], f2(ex2_approx(g.x), ex2_approx(g.y)));
                        }
                }
                // the rest: one snapshot at a time, each at its own class, whole records
                // from global memory
                for (uint32_t m = mp; m; m &= m - 1) {
                    const int b = __ffs(m) - 1, s = cw * 32 + b;
                    const uint32_t word = __shfl_sync(0xffffffffu, my_word[cw], b);
                    float r2[PPT];
                    rho2_points<PPT>(pp, sm.xy[s], split, r2);
#pragma unroll
                    for (int jc = 0; jc < TCH; ++jc) {
                        const uint32_t c = (word >> (kCodeBits * jc)) & kCodeMask;
                        if (c == kCodeSkip) continue;
                        const RecF32 &Rs = rows[jc][s0 + s];            // active: the record exists
                        float2 (&A)[PPT] = acc[jc >> 1];
                        if (c == kCodeD2) {
                            if (jc & 1) moment_pass<2, PPT, 1>(A, r2, Rs); else moment_pass<2, PPT, 0>(A, r2, Rs);
                        } else if (c == kCodeD4) {
                            if (jc & 1) moment_pass<4, PPT, 1>(A, r2, Rs); else moment_pass<4, PPT, 0>(A, r2, Rs);
                        } else if (c == kCodeD8) {
                            if (jc & 1) moment_pass<8, PPT, 1>(A, r2, Rs); else moment_pass<8, PPT, 0>(A, r2, Rs);
                        } else if (c == kCodeD12) {
                            if (jc & 1) moment_pass<12, PPT, 1>(A, r2, Rs); else moment_pass<12, PPT, 0>(A, r2, Rs);
                        } else {
#pragma unroll
                            for (int k = 0; k < PPT; ++k) {
                                const float t = pair_term(r2[k], Rs);
                                if (jc & 1) A[k].y += t; else A[k].x += t;
                            }
                        }
                    }
                }
            } else {
                // one snapshot: points (2m, 2m+1) in one f32x2 instruction instead
                for (uint32_t m = m2 | m4; m; m &= m - 1) {
                    const int b = __ffs(m) - 1, s = cw * 32 + b;
                    const bool d4 = (m4 >> b) & 1u;
                    const float4 v0 = sm.lo[0][s];                     // (g_0, g_1x, g_2x, g_3x)
                    const float g4 = d4 ? sm.hi[0][s].x : 0.0f;
                    float r2[PPT];
                    rho2_points<PPT>(pp, sm.xy[s], split, r2);
#pragma unroll
                    for (int mm = 0; mm < PPT / 2; ++mm) {
                        const float2 r = f2(r2[2 * mm], r2[2 * mm + 1]);
                        float2 g;
                        if (!d4) {
                            g = __ffma2_rn(f2(v0.z, v0.z), r, f2(v0.y, v0.y));
                        } else {
                            g = __ffma2_rn(f2(g4, g4), r, f2(v0.w, v0.w));
                            g = __ffma2_rn(g, r, f2(v0.z, v0.z));
                            g = __ffma2_rn(g, r, f2(v0.y, v0.y));
                        }
                        g = __ffma2_rn(g, r, f2(v0.x, v0.x));
                        acc[0][mm] = __fadd2_rn(acc[0][mm], f2(ex2_approx(g.x), ex2_approx(g.y)));
                    }
                }
                // another class: per point, into the point-pair accumulators
                for (uint32_t m = mp; m; m &= m - 1) {
                    const int b = __ffs(m) - 1, s = cw * 32 + b;
                    const uint32_t c = __shfl_sync(0xffffffffu, my_word[cw], b) & kCodeMask;
                    if (c == kCodeSkip) continue;
                    float r2[PPT];
                    rho2_points<PPT>(pp, sm.xy[s], split, r2);
                    const RecF32 &Rs = sm.rec[s];
                    if (c == kCodeD8) {
                        point_pass_h2<8, PPT>(acc[0], r2, Rs);
                    } else if (c == kCodeD12) {
                        point_pass_h2<12, PPT>(acc[0], r2, Rs);
                    } else if (c == kCodeGeneral) {
#pragma unroll
                        for (int k = 0; k < PPT; ++k) {
                            const float t = pair_term(r2[k], Rs);
                            if (k & 1) acc[0][k >> 1].y += t; else acc[0][k >> 1].x += t;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int jc = 0; jc < TCH; ++jc)
#pragma unroll
            for (int k = 0; k < PPT; ++k)
                sm.run[jc * PPT + k][tid] += kSingle ? ((k & 1) ? acc[0][k >> 1].y : acc[0][k >> 1].x)
                                                     : ((jc & 1) ? acc[jc >> 1][k].y : acc[jc >> 1][k].x);
#pragma unroll
        for (int m = 0; m < NP; ++m)
#pragma unroll
            for (int k = 0; k < PPT; ++k) acc[m][k] = f2(0.0f, 0.0f);
    }
#pragma unroll
    for (int jc = 0; jc < TCH; ++jc) {
        if (jc >= nj) continue;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int64_t p = tile0 + k * NT + tid;
            if (p < n_pts) partial[(int64_t)jc * part_stride + p] = (Part)sm.run[jc * PPT + k][tid];
        }
    }
}

// Sum of pair terms over visits [s_begin, s_end) for the point tile starting at point
// tile0 and TCH snapshots:  partial[jc * part_stride + p] = sum_{i < na[jc]} term(p, i, jc)
// for jc < nj.  rec points at the record row of the first snapshot (row stride
// rec_stride); records exist for visits below na[jc].  All threads of the CTA call it.
template <typename Cfg, int TCH>
__device__ __forceinline__ void field_tile(TileSmem<Cfg, TCH> &sm, const double *__restrict__ srcX,
                                           const double *__restrict__ srcY, const double *__restrict__ X,
                                           const double *__restrict__ Y, int64_t n_pts, int64_t tile0,
                                           const typename Cfg::Rec *const (&rows)[TCH], const int (&na)[TCH],
                                           int nj, int s_begin, int s_end, double *__restrict__ partial,
                                           int64_t part_stride) {
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
            const float4 *row = reinterpret_cast<const float4 *>(rows[jc] + s0);
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
                    if constexpr (std::is_same<Rec, RecF64>::value) {
                        // one polynomial degree for the warp, from every lane's own h and a
                        uint32_t cls = 0;
#pragma unroll
                        for (int k = 0; k < PPT; ++k) {
                            const double h = r2[k] * R.dq, a = r2[k] * R.q1;
                            const uint32_t c = a >= 745.0 ? 0u : h <= kDeg4HD ? 1u : h <= kDeg8HD ? 2u
                                             : h <= kDeg11HD ? 3u : 4u;
                            cls = max(cls, c);
                        }
                        cls = __reduce_max_sync(0xffffffffu, cls);
#pragma unroll
                        for (int k = 0; k < PPT; ++k) {
                            if (cls == 1u) acc[jc][k] += moment_term_f64<4>(r2[k], R);
                            else if (cls == 2u) acc[jc][k] += moment_term_f64<8>(r2[k], R);
                            else if (cls == 3u) acc[jc][k] += moment_term_f64<11>(r2[k], R);
                            else if (cls == 4u) acc[jc][k] += pair_term(r2[k], R);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < PPT; ++k) acc[jc][k] += pair_term(r2[k], R);
                    }
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

// Running sum of FP32 (mixed path) or FP64 values.  FP32 values are added with Knuth's
// two-sum, so s + c carries the sum to about one FP32 rounding without any FP64
// arithmetic: FP64 runs at about 1/70 of the FP32 rate on this part, and a plain FP64
// reduction of the FP32 partial sums ran at 0.8 TB/s instead of streaming them from HBM.
// FP64 values are summed in FP64.
template <typename Part>
struct BlockSum;
template <>
struct BlockSum<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        const float b = t - s;
        c += (s - (t - b)) + (x - b);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
    // s + c rounded to FP32 (one rounding; no FP64 arithmetic)
    __device__ __forceinline__ float result() const { return s + c; }
};
template <>
struct BlockSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
    __device__ __forceinline__ double result() const { return s; }
};

// Four consecutive per-item sums of one partial row, read at L2 (written by other SMs);
// the row offset is a multiple of 4 elements.
__device__ __forceinline__ void load4_cg(const float *p, float (&v)[4]) {
    const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4_cg(const double *p, double (&v)[4]) {
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// One work item per CTA: item = (point tile, snapshot chunk, visit block).  The items are
// the (chunk, block) descriptors desc[] (in cost order) times the point tiles in tile
// order: CTA item0 + blockIdx.x takes descriptor (item0 + blockIdx.x) / n_tiles and tile
// (item0 + blockIdx.x) % n_tiles.
// partial[(block * n_tg + j) * pstride + p] receives sum_{i in block, i < nact[j]} pair_term
// (pstride = n_pts rounded up to a multiple of 4, so that rows are 16-byte aligned).
template <typename Cfg>
__global__ void __launch_bounds__(Cfg::kThreads, Cfg::kMinBlocks)
field_kernel(const double *__restrict__ srcX, const double *__restrict__ srcY,
             const double *__restrict__ X, const double *__restrict__ Y, int64_t n_pts,
             const typename Cfg::Rec *__restrict__ rec, const int64_t *__restrict__ row_off,
             const int *__restrict__ nact, const int2 *__restrict__ desc, int64_t n_tiles, int64_t item0,
             int n_tg, int sb, typename Cfg::Real *__restrict__ partial, int64_t pstride,
             const float4 *__restrict__ srcF, const float4 *__restrict__ ptsF) {
    using Rec = typename Cfg::Rec;
    constexpr int TCH = Cfg::kTCH;
    const int64_t q = item0 + blockIdx.x;
    const int2 dc = desc[q / n_tiles];                     // (chunk, block)
    const int4 item = make_int4((int)(q % n_tiles), dc.x, dc.y, 0);
    const int j0 = item.y * TCH;
    int na[TCH];
    const Rec *rows[TCH];
    int nmax = 0;
#pragma unroll
    for (int jc = 0; jc < TCH; ++jc) {
        const bool live = j0 + jc < n_tg;
        na[jc] = live ? nact[j0 + jc] : 0;
        rows[jc] = live ? rec + row_off[j0 + jc] : rec;     // record of visit i: rows[jc][i]
        nmax = max(nmax, na[jc]);
    }
    const int s_begin = item.z * sb;
    const int s_end = min(s_begin + sb, nmax);
    const int64_t tile0 = (int64_t)item.x * (Cfg::kThreads * Cfg::kPPT);
    // per-item sums: FP32 on the mixed path (they are FP32 sums already), FP64 otherwise
    typename Cfg::Real *part = partial + ((int64_t)item.z * n_tg + j0) * pstride;
    if constexpr (std::is_same<typename Cfg::Real, float>::value) {
        __shared__ TileSmemMixed<Cfg, TCH> sm;
        field_tile_mixed<Cfg, TCH>(sm, srcF, ptsF, n_pts, tile0, rows, na, min(TCH, n_tg - j0), s_begin,
                                   s_end, part, pstride);
    } else {
        __shared__ TileSmem<Cfg, TCH> sm;
        field_tile<Cfg, TCH>(sm, srcX, srcY, X, Y, n_pts, tile0, rows, na, min(TCH, n_tg - j0), s_begin, s_end,
                             part, pstride);
    }

}

}  // namespace ddk
