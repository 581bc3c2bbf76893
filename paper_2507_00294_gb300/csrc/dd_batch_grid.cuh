// dd_batch_grid.cuh -- FP32-mixed batch tile for scans evaluated on rectilinear grids of
// points (dd_batch_create_grid): one snapshot per scan, so the pair term of degree 2 takes
// the separable form of dd_field_grid.cuh with the sharing spread over rows instead of
// snapshots.  A tile is 32 grid columns x 32 grid rows; thread (warp w, lane l) holds
// column c0 + l at the rows r0 + 8 w .. r0 + 8 w + 7.  Per staged visit the CTA forms the
// row tables of its 32 rows (dy^2, Y = 2^(g_1x dy^2 + g_2x dy^4) and Y dy^2); a thread's
// degree-2 pairs then cost the column factor X = 2^(g_0 + g_1x dx^2 + g_2x dx^4) (one ex2,
// shared by its 8 rows) and one FMA per pair (two with the cross term), two rows per f32x2
// instruction.  Degree 4 and the higher classes run per point as in the general tile, with
// rho^2 = dx^2 + dy^2.
#pragma once
#include <cstdint>

#include "dd_field_grid.cuh"
#include "dd_field_impl.cuh"

namespace ddk {

constexpr int kBgCols = 32, kBgRowsPerThread = 8, kBgRows = 32, kBgThreads = 128, kBgStage = 32;

struct BGridSmem {
    float run[kBgRowsPerThread][kBgThreads];            // per-thread running sums over stages
    float vx[kBgStage], vy[kBgStage];                   // visit minus tile origin (integers)
    float4 v0[kBgStage], v1[kBgStage];                  // record vectors (g_0, g_1x, g_2x, g_3x), (g_4x, dq, q1, c_0)
    float4 yf[kBgStage][kBgRows / 4];                   // row factor Y per (visit, row)
    float4 bf[kBgStage][kBgRows / 4];                   // Y dy^2
    float4 dy2[kBgStage][kBgRows / 4];                  // dy^2
    float yin[kBgRows], yfr[kBgRows];                   // the rows' y: integer offset + fraction
};

// Degree 8 / 12 in h form for a thread's 8 points on f32x2 over row pairs (m: rows 2m, 2m+1).
template <int D>
__device__ __forceinline__ void rows_pass_h2(float2 (&acc)[4], const float (&r2)[8], const RecF32 &R) {
    const float2 dq = make_float2(R.dq(), R.dq()), g0 = make_float2(R.g0(), R.g0());
    float2 h[4], p[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        h[m] = __fmul2_rn(make_float2(r2[2 * m], r2[2 * m + 1]), dq);
        p[m] = make_float2(R.k(D), R.k(D));
    }
#pragma unroll
    for (int j = D - 1; j >= 1; --j) {
        const float2 c = make_float2(R.k(j), R.k(j));
#pragma unroll
        for (int m = 0; m < 4; ++m) p[m] = __ffma2_rn(p[m], h[m], c);
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float2 g = __ffma2_rn(p[m], h[m], g0);
        acc[m] = __fadd2_rn(acc[m], make_float2(ex2_approx(g.x), ex2_approx(g.y)));
    }
}

// Sum of the pair terms of visits [s_begin, s_end) (all started: one snapshot, rows[i] the
// record of visit i) at the tile's points; partial[r W + c] receives the sum at (c, r).
__device__ __forceinline__ void field_tile_bgrid(BGridSmem &sm, const float4 *__restrict__ srcF,
                                                 const float4 *__restrict__ ptsF, int64_t W, int64_t H, int64_t tc,
                                                 int64_t tr, const RecF32 *__restrict__ rows, int s_begin,
                                                 int s_end, double *__restrict__ partial) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c0 = tc * kBgCols, r0 = tr * kBgRows;
    const int64_t c = c0 + lane;
    const bool live_c = c < W;
    const int64_t cc = live_c ? c : W - 1;               // spare columns repeat the last one
    const float4 org = ptsF[r0 * W + c0];
    const float ox = rintf(org.x), oy = rintf(org.z);
    const float4 qx = ptsF[r0 * W + cc];
    const float ix = rintf(qx.x);
    const float xfr = (qx.x - ix) + qx.y;
    const float xin = ix - ox;
    bool exact = ((xin + xfr) - xin) == xfr;
    if (tid < kBgRows) {                                 // the tile's rows, once
        const int64_t rk = min(r0 + tid, H - 1);
        const float4 qy = ptsF[rk * W + c0];
        const float iy = rintf(qy.z);
        const float yf = (qy.z - iy) + qy.w, yi = iy - oy;
        exact = exact && ((yi + yf) - yi) == yf;
        sm.yin[tid] = yi;
        sm.yfr[tid] = yf;
    }
    const bool split = __syncthreads_or(!exact) != 0;   // also publishes the rows
    const float xs = xin + xfr;
    float bx0 = xs, bx1 = xs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bx0 = fminf(bx0, __shfl_xor_sync(0xffffffffu, bx0, o));
        bx1 = fmaxf(bx1, __shfl_xor_sync(0xffffffffu, bx1, o));
    }
    float by0 = 3.0e38f, by1 = -3.0e38f;                 // this warp's 8 rows
#pragma unroll
    for (int j = 0; j < kBgRowsPerThread; ++j) {
        const float y = sm.yin[kBgRowsPerThread * warp + j] + sm.yfr[kBgRowsPerThread * warp + j];
        by0 = fminf(by0, y);
        by1 = fmaxf(by1, y);
    }
    float2 acc[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[m] = f2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < kBgRowsPerThread; ++j) sm.run[j][tid] = 0.f;

    for (int s0 = s_begin; s0 < s_end; s0 += kBgStage) {
        const int cnt = min(kBgStage, s_end - s0);
        __syncthreads();
        if (tid < cnt) {
            const float4 v = srcF[s0 + tid];
            sm.vx[tid] = (v.x - ox) + v.y;
            sm.vy[tid] = (v.z - oy) + v.w;
        } else if (tid >= 64 && tid - 64 < 2 * cnt) {
            const int i = (tid - 64) >> 1, q = (tid - 64) & 1;
            const float4 r = reinterpret_cast<const float4 *>(rows + s0 + i)[q];
            if (q == 0) sm.v0[i] = r; else sm.v1[i] = r;
        }
        __syncthreads();
        // row tables: 32 visits x 32 rows, 8 (visit, row) pairs per thread
#pragma unroll 2
        for (int q = 0; q < (kBgStage * kBgRows) / kBgThreads; ++q) {
            const int idx = q * kBgThreads + tid, i = idx >> 5, r = idx & 31;
            if (i < cnt) {
                const float vy = sm.vy[i];
                const float dy = split ? (sm.yin[r] - vy) + sm.yfr[r] : (sm.yin[r] + sm.yfr[r]) - vy;
                const float d2 = dy * dy;
                const float4 v0 = sm.v0[i];
                const float y = ex2_approx(d2 * fmaf(v0.z, d2, v0.y));
                reinterpret_cast<float *>(&sm.yf[i][0])[r] = y;
                reinterpret_cast<float *>(&sm.bf[i][0])[r] = y * d2;
                reinterpret_cast<float *>(&sm.dy2[i][0])[r] = d2;
            }
        }
        // class of staged visit `lane` against this warp's box (32 columns x 8 rows)
        uint32_t my_code = kCodeSkip;
        bool sep1 = false;
        if (lane < cnt) {
            const float sx = sm.vx[lane], sy = sm.vy[lane];
            float r2min, r2max;
            box_rho2(sx, sy, bx0, bx1, by0, by1, r2min, r2max);
            const float4 v0 = sm.v0[lane], v1 = sm.v1[lane];
            my_code = series_class(r2max * v1.y, r2min * v1.z, v1.y);
            const float dxm = fmaxf(fabsf(sx - bx0), fabsf(sx - bx1));
            const float dym = fmaxf(fabsf(sy - by0), fabsf(sy - by1));
            sep1 = 2.0f * fabsf(v0.z) * ((dxm * dxm) * (dym * dym) * 1.0001f + 1e-6f) <= kSepCross;
        }
        __syncthreads();                                 // row tables visible
        const uint32_t m1 = __ballot_sync(0xffffffffu, my_code == kCodeD2 && sep1);
        const uint32_t m2 = __ballot_sync(0xffffffffu, my_code == kCodeD2 && !sep1);
        const uint32_t m4 = __ballot_sync(0xffffffffu, my_code == kCodeD4);
        const uint32_t mh = __ballot_sync(0xffffffffu, my_code > kCodeD4);
        const int q0 = 2 * warp;                         // this warp's rows: float4 q0, q0 + 1
        for (uint32_t m = m1; m; m &= m - 1) {           // X Y
            const int s = __ffs(m) - 1;
            const float4 v0 = sm.v0[s];
            const float vx = sm.vx[s];
            const float dx = split ? (xin - vx) + xfr : xs - vx;
            const float d2 = dx * dx;
            const float X = ex2_approx(fmaf(fmaf(v0.z, d2, v0.y), d2, v0.x));
            const float2 XX = f2(X, X);
            const float4 ya = sm.yf[s][q0], yb = sm.yf[s][q0 + 1];
            acc[0] = __ffma2_rn(XX, f2(ya.x, ya.y), acc[0]);
            acc[1] = __ffma2_rn(XX, f2(ya.z, ya.w), acc[1]);
            acc[2] = __ffma2_rn(XX, f2(yb.x, yb.y), acc[2]);
            acc[3] = __ffma2_rn(XX, f2(yb.z, yb.w), acc[3]);
        }
        for (uint32_t m = m2; m; m &= m - 1) {           // X Y + A B
            const int s = __ffs(m) - 1;
            const float4 v0 = sm.v0[s];
            const float vx = sm.vx[s];
            const float dx = split ? (xin - vx) + xfr : xs - vx;
            const float d2 = dx * dx;
            const float X = ex2_approx(fmaf(fmaf(v0.z, d2, v0.y), d2, v0.x));
            const float A = X * ((kTwoLn2 * v0.z) * d2);
            const float2 XX = f2(X, X), AA = f2(A, A);
            const float4 ya = sm.yf[s][q0], yb = sm.yf[s][q0 + 1];
            const float4 ba = sm.bf[s][q0], bb = sm.bf[s][q0 + 1];
            acc[0] = __ffma2_rn(AA, f2(ba.x, ba.y), __ffma2_rn(XX, f2(ya.x, ya.y), acc[0]));
            acc[1] = __ffma2_rn(AA, f2(ba.z, ba.w), __ffma2_rn(XX, f2(ya.z, ya.w), acc[1]));
            acc[2] = __ffma2_rn(AA, f2(bb.x, bb.y), __ffma2_rn(XX, f2(yb.x, yb.y), acc[2]));
            acc[3] = __ffma2_rn(AA, f2(bb.z, bb.w), __ffma2_rn(XX, f2(yb.z, yb.w), acc[3]));
        }
        for (uint32_t m = m4; m; m &= m - 1) {           // degree 4 per point, rows paired
            const int s = __ffs(m) - 1;
            const float4 v0 = sm.v0[s], v1 = sm.v1[s];
            const float vx = sm.vx[s];
            const float dx = split ? (xin - vx) + xfr : xs - vx;
            const float4 da = sm.dy2[s][q0], db = sm.dy2[s][q0 + 1];
            const float2 r2[4] = {f2(fmaf(dx, dx, da.x), fmaf(dx, dx, da.y)), f2(fmaf(dx, dx, da.z), fmaf(dx, dx, da.w)),
                                  f2(fmaf(dx, dx, db.x), fmaf(dx, dx, db.y)), f2(fmaf(dx, dx, db.z), fmaf(dx, dx, db.w))};
#pragma unroll
            for (int mm = 0; mm < 4; ++mm) {
                float2 g = __ffma2_rn(f2(v1.x, v1.x), r2[mm], f2(v0.w, v0.w));
                g = __ffma2_rn(g, r2[mm], f2(v0.z, v0.z));
                g = __ffma2_rn(g, r2[mm], f2(v0.y, v0.y));
                g = __ffma2_rn(g, r2[mm], f2(v0.x, v0.x));
                acc[mm] = __fadd2_rn(acc[mm], f2(ex2_approx(g.x), ex2_approx(g.y)));
            }
        }
        for (uint32_t m = mh; m; m &= m - 1) {           // degree 8 / 12 or two E1 values
            const int s = __ffs(m) - 1;
            const uint32_t code = __shfl_sync(0xffffffffu, my_code, s);
            const RecF32 &R = rows[s0 + s];
            const float vx = sm.vx[s];
            const float dx = split ? (xin - vx) + xfr : xs - vx;
            const float4 da = sm.dy2[s][q0], db = sm.dy2[s][q0 + 1];
            const float r2[8] = {fmaf(dx, dx, da.x), fmaf(dx, dx, da.y), fmaf(dx, dx, da.z), fmaf(dx, dx, da.w),
                                 fmaf(dx, dx, db.x), fmaf(dx, dx, db.y), fmaf(dx, dx, db.z), fmaf(dx, dx, db.w)};
            if (code == kCodeD8) {
                rows_pass_h2<8>(acc, r2, R);
            } else if (code == kCodeD12) {
                rows_pass_h2<12>(acc, r2, R);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float t = pair_term(r2[j], R);
                    if (j & 1) acc[j >> 1].y += t; else acc[j >> 1].x += t;
                }
            }
        }
#pragma unroll
        for (int mm = 0; mm < 4; ++mm) {
            sm.run[2 * mm][tid] += acc[mm].x;
            sm.run[2 * mm + 1][tid] += acc[mm].y;
            acc[mm] = f2(0.f, 0.f);
        }
    }
    if (live_c) {
#pragma unroll
        for (int j = 0; j < kBgRowsPerThread; ++j) {
            const int64_t r = r0 + kBgRowsPerThread * warp + j;
            if (r < H) partial[r * W + c] = (double)sm.run[j][tid];
        }
    }
}

}  // namespace ddk
