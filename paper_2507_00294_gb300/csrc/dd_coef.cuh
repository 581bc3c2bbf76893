// dd_coef.cuh -- FP64 per-(visit, snapshot) coefficients of the pair term (Eq. 1/2).
#pragma once
#include <cstdint>

#include "dd_field_impl.cuh"

namespace ddk {

// --------------------------------------------------------------- coefficients

// c_m = (-1)^m J_m(r) / m!,  J_m(r) = int_0^1 r s^m / (1 + r s) ds,  m = 0..M, c_0 = ln(1+r).
// J_m = 1/m - J_{m-1}/r (forward) is stable for r >= 1.  For r < 1 the same recurrence
// is run downward from J_M, which comes from the positive series
//   J_M = rho sum_k rho^k B(M+1, k+1),  rho = r/(1+r)  (expand 1/(1+rs) about s = 1).
// 1/n for n = 0..95 (entry 0 unused), exact to FP64 rounding.
struct RecipTable {
    double v[96];
    constexpr RecipTable() : v() {
        for (int n = 1; n < 96; ++n) v[n] = 1.0 / n;
    }
};
static __device__ __constant__ RecipTable kRecipTable = RecipTable();
#define kRecip kRecipTable.v
// The same rounded to FP32 (bit for bit (float)kRecip[n]), for the FP32 recurrences: an
// FP64 -> FP32 conversion per use would run on the FP64 unit, a small fraction of the
// FP32 rate on this part, inside each thread's serial chain.
struct RecipTableF {
    float v[96];
    constexpr RecipTableF() : v() {
        for (int n = 1; n < 96; ++n) v[n] = (float)(1.0 / n);
    }
};
static __device__ __constant__ RecipTableF kRecipFTable = RecipTableF();
#define kRecipF kRecipFTable.v

template <int M>
__device__ void moment_coefficients(double r, double ell, double *c) {
    double J[M + 1];
    if (r >= 1.0) {
        const double ir = 1.0 / r;
        J[0] = ell;
#pragma unroll
        for (int m = 1; m <= M; ++m) J[m] = kRecip[m] - J[m - 1] * ir;
    } else {
        const double rho = r / (1.0 + r);
        double term = rho * kRecip[M + 1], sum = 0.0;
        // rho < 1/2 here, so the terms shrink at least geometrically: 64 suffice
        for (int k = 1; k < 64; ++k) {
            sum += term;
            term *= rho * k * kRecip[M + 1 + k];
            if (term <= 1e-18 * sum) break;
        }
        J[M] = sum;
#pragma unroll
        for (int m = M; m >= 1; --m) J[m - 1] = r * (kRecip[m] - J[m]);
        J[0] = ell;
    }
    double inv_fact = 1.0;
#pragma unroll
    for (int m = 0; m <= M; ++m) {
        c[m] = (m & 1) ? -J[m] * inv_fact : J[m] * inv_fact;
        inv_fact *= kRecip[m + 1];
    }
}

// The same in FP32 (for the FP32 record's exponent series, whose coefficients beyond
// c_0 only enter as corrections l_m h^m next to the FP64-computed exponent terms; the
// recurrences are the stable ones above, so FP32 keeps them to a few ulp, and the
// dependent chain is a few hundred cycles instead of the FP64 unit's tens of thousands).
template <int M>
__device__ void moment_coefficients_f32(float r, float ell, float *c) {
    float J[M + 1];
    if (r >= 1.0f) {
        const float ir = 1.0f / r;
        J[0] = ell;
#pragma unroll
        for (int m = 1; m <= M; ++m) J[m] = kRecipF[m] - J[m - 1] * ir;
    } else {
        const float rho = r / (1.0f + r);
        float term = rho * kRecipF[M + 1], sum = 0.0f;
        for (int k = 1; k < 64; ++k) {
            sum += term;
            term *= rho * (float)k * kRecipF[M + 1 + k];
            if (term <= 1e-9f * sum) break;
        }
        J[M] = sum;
#pragma unroll
        for (int m = M; m >= 1; --m) J[m - 1] = r * (kRecipF[m] - J[m]);
        J[0] = ell;
    }
    float inv_fact = 1.0f;
#pragma unroll
    for (int m = 0; m <= M; ++m) {
        c[m] = (m & 1) ? -J[m] * inv_fact : J[m] * inv_fact;
        inv_fact *= kRecipF[m + 1];
    }
}

// kEll: also ell = ln(w1/w0) in FP64 (the FP64 record needs it; the FP32 record forms
// its own in FP32, which is all its rounding to FP32 keeps).
template <bool kEll = true>
__device__ __forceinline__ void pair_geometry(double dT, double tau, double s, double kappa,
                                              double &q1, double &dq, double &r, double &ell) {
    const bool on = dT <= tau;                         // Eq. 1 while t_i <= t <= t_i + tau_i
    const double w1 = 2.0 * s + 4.0 * kappa * dT;
    const double w0 = on ? 2.0 * s : 2.0 * s + 4.0 * kappa * (dT - tau);
    const double dw = 4.0 * kappa * (on ? dT : tau);   // w1 - w0 without cancellation
    q1 = 1.0 / w1;
    r = dw / w0;
    dq = r * q1;                                       // 1/w0 - 1/w1
    ell = kEll ? log1p(r) : 0.0;                       // ln(w1/w0) = ln(b/a)
}

template <typename Rec>
__global__ void coef_kernel(const double *__restrict__ srcT, const double *__restrict__ srcTAU,
                            const double *__restrict__ tsnap, const int *__restrict__ nact,
                            double s, double kappa, Rec *__restrict__ rec, int64_t stride) {
    const int j = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nact[j]) return;
    double q1, dq, r, ell;
    pair_geometry<RecTraits<Rec>::kFP64Ell>(tsnap[j] - srcT[i], srcTAU[i], s, kappa, q1, dq, r, ell);
    Rec out;
    RecTraits<Rec>::fill(out, q1, dq, r, ell);
    rec[(int64_t)j * stride + i] = out;
}

template <>
struct RecTraits<RecF32> {
    // The exponent series of the FP32 record (see RecF32): l_m, the coefficients of
    // ln(P(h)/c_0) with P(h) = sum_m c_m h^m, from the power-series logarithm
    //   l_m = p_m - (1/m) sum_{k=1}^{m-1} k l_k p_{m-k},  p_m = c_m / c_0
    // (P'/P = (ln P)').
    static constexpr bool kFP64Ell = false;
    // ell: unused (c_0 = ln(1 + r) is formed here in FP32)
    static __device__ void fill(RecF32 &o, double q1, double dq, double r, double) {
        constexpr int M = 12;
        constexpr double kLog2e = 1.44269504088896340736;
        const float kLog2eF = (float)kLog2e;
        // the exponent's leading terms: q1 and dq from FP64 (rounded once), the logs and
        // 1/r in FP32 (they enter as g_0 = log2 c_0 and k_1, both kept to FP32 rounding);
        // the corrections l_m (|l_m h^m| <= 0.85) in FP32
        const float rf = (float)r, ellf = log1pf(rf);
        float cf[M + 1], p[M + 1], l[M + 1];
        moment_coefficients_f32<M>(rf, ellf, cf);
        const float ic0 = 1.0f / cf[0];
#pragma unroll
        for (int m = 1; m <= M; ++m) p[m] = cf[m] * ic0;
#pragma unroll
        for (int m = 1; m <= M; ++m) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 1; k < m; ++k) acc = fmaf((float)k * l[k], p[m - k], acc);
            l[m] = p[m] - acc * kRecipF[m];
        }
        const float dqf = (float)dq, dq2 = dqf * dqf;
        o.v0 = make_float4(log2f(ellf), (float)(kLog2e * ((double)l[1] * dq - q1)),
                           kLog2eF * dq2 * l[2], kLog2eF * dq2 * dqf * l[3]);
        o.v1 = make_float4(kLog2eF * dq2 * dq2 * l[4], dqf, (float)q1, ellf);
        o.v2 = make_float4(kLog2eF * (l[1] - 1.0f / rf), kLog2eF * l[2], kLog2eF * l[3], kLog2eF * l[4]);
        o.v3 = make_float4(kLog2eF * l[5], kLog2eF * l[6], kLog2eF * l[7], kLog2eF * l[8]);
        o.v4 = make_float4(kLog2eF * l[9], kLog2eF * l[10], kLog2eF * l[11], kLog2eF * l[12]);
    }
    // a visit that has not started: every path yields 2^-inf = 0
    static __device__ RecF32 zero() {
        RecF32 z;
        z.v0 = make_float4(-INFINITY, 0.f, 0.f, 0.f);
        z.v1 = z.v2 = z.v3 = z.v4 = make_float4(0.f, 0.f, 0.f, 0.f);
        return z;
    }
};

template <>
struct RecTraits<RecF64> {
    static __device__ void fill(RecF64 &o, double q1, double dq, double r, double ell) {
        moment_coefficients<RecF64::kTerms - 1>(r, ell, o.c);
        o.q1 = q1;
        o.dq = dq;
    }
    static __device__ RecF64 zero() { return RecF64{}; }
    static constexpr bool kFP64Ell = true;
};

// Record for lag k = 1..n-1 of a scan with a uniform dwell (time unit = dwell):
// visit i seen from the start of visit i + k, i.e. dT = k, tau = 1.
template <typename Rec>
__global__ void lag_coef_kernel(int64_t n, double s, double kappa, Rec *__restrict__ rec) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (k == 0) { rec[0] = RecTraits<Rec>::zero(); return; }
    double q1, dq, r, ell;
    pair_geometry<RecTraits<Rec>::kFP64Ell>((double)k, 1.0, s, kappa, q1, dq, r, ell);
    Rec out;
    RecTraits<Rec>::fill(out, q1, dq, r, ell);
    rec[k] = out;
}

// Reversed lag table for snapshots on the dwell lattice of a uniform scan:
// rev[u] = record of lag L = M - u (dT = L dwells, tau = 1) for u < M, zero for u = M.
// Snapshot t_j (an integer number of dwells) then reads visit i's record at
// rev[M - t_j + i], contiguous in i.
template <typename Rec>
__device__ __forceinline__ void rev_lag_record(int64_t u, int64_t M, double s, double kappa, Rec *__restrict__ rev) {
    if (u > M) return;
    const int64_t L = M - u;
    if (L == 0) { rev[u] = RecTraits<Rec>::zero(); return; }
    double q1, dq, r, ell;
    pair_geometry<RecTraits<Rec>::kFP64Ell>((double)L, 1.0, s, kappa, q1, dq, r, ell);
    Rec out;
    RecTraits<Rec>::fill(out, q1, dq, r, ell);
    rev[u] = out;
}

}  // namespace ddk
