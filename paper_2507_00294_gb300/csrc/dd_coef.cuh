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

__device__ __forceinline__ void pair_geometry(double dT, double tau, double s, double kappa,
                                              double &q1, double &dq, double &r, double &ell) {
    const bool on = dT <= tau;                         // Eq. 1 while t_i <= t <= t_i + tau_i
    const double w1 = 2.0 * s + 4.0 * kappa * dT;
    const double w0 = on ? 2.0 * s : 2.0 * s + 4.0 * kappa * (dT - tau);
    const double dw = 4.0 * kappa * (on ? dT : tau);   // w1 - w0 without cancellation
    q1 = 1.0 / w1;
    r = dw / w0;
    dq = r * q1;                                       // 1/w0 - 1/w1
    ell = log1p(r);                                    // ln(w1/w0) = ln(b/a)
}

template <typename Rec>
__global__ void coef_kernel(const double *__restrict__ srcT, const double *__restrict__ srcTAU,
                            const double *__restrict__ tsnap, const int *__restrict__ nact,
                            double s, double kappa, Rec *__restrict__ rec, int64_t stride) {
    const int j = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nact[j]) return;
    double q1, dq, r, ell;
    pair_geometry(tsnap[j] - srcT[i], srcTAU[i], s, kappa, q1, dq, r, ell);
    Rec out;
    RecTraits<Rec>::fill(out, q1, dq, r, ell);
    rec[(int64_t)j * stride + i] = out;
}

template <>
struct RecTraits<RecF32> {
    static __device__ void fill(RecF32 &o, double q1, double dq, double r, double ell) {
        double c[RecF32::kTerms];
        moment_coefficients<RecF32::kTerms - 1>(r, ell, c);
        const double dq2 = dq * dq;
        o.v0 = make_float4((float)(-q1 * 1.44269504088896340736), (float)c[0], (float)(c[1] * dq), (float)(c[2] * dq2));
        o.v1 = make_float4((float)(c[3] * dq2 * dq), (float)(c[4] * dq2 * dq2), (float)dq, (float)c[1]);
        o.v2 = make_float4((float)c[2], (float)c[3], (float)c[4], (float)c[5]);
        o.v3 = make_float4((float)c[6], (float)c[7], (float)c[8], (float)c[9]);
        o.v4 = make_float4((float)c[10], (float)c[11], (float)c[12], 0.0f);
    }
};

template <>
struct RecTraits<RecF64> {
    static __device__ void fill(RecF64 &o, double q1, double dq, double r, double ell) {
        moment_coefficients<RecF64::kTerms - 1>(r, ell, o.c);
        o.q1 = q1;
        o.dq = dq;
    }
};

// Record for lag k = 1..n-1 of a scan with a uniform dwell (time unit = dwell):
// visit i seen from the start of visit i + k, i.e. dT = k, tau = 1.
template <typename Rec>
__global__ void lag_coef_kernel(int64_t n, double s, double kappa, Rec *__restrict__ rec) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (k == 0) { rec[0] = Rec{}; return; }
    double q1, dq, r, ell;
    pair_geometry((double)k, 1.0, s, kappa, q1, dq, r, ell);
    Rec out;
    RecTraits<Rec>::fill(out, q1, dq, r, ell);
    rec[k] = out;
}

// Reversed lag table for snapshots on the dwell lattice of a uniform scan:
// rev[u] = record of lag L = M - u (dT = L dwells, tau = 1) for u < M, zero for u = M.
// Snapshot t_j (an integer number of dwells) then reads visit i's record at
// rev[M - t_j + i], contiguous in i.
template <typename Rec>
__global__ void rev_lag_coef_kernel(int64_t M, double s, double kappa, Rec *__restrict__ rev) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u > M) return;
    const int64_t L = M - u;
    if (L == 0) { rev[u] = Rec{}; return; }
    double q1, dq, r, ell;
    pair_geometry((double)L, 1.0, s, kappa, q1, dq, r, ell);
    Rec out;
    RecTraits<Rec>::fill(out, q1, dq, r, ell);
    rev[u] = out;
}

}  // namespace ddk
