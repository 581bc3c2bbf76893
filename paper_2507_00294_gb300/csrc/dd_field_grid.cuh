// dd_field_grid.cuh -- FP32-mixed field tile for evaluation points on a rectilinear grid.
//
// A tile is 128 grid columns x 4 grid rows: thread t holds column c0 + t at the four rows
// r0..r0+3, for four snapshots (two f32x2 snapshot pairs).  Every point of a thread then
// shares its x and every point of a row shares its y, which the pair term can use.  With
// rho^2 = dx^2 + dy^2 the degree-2 exponent of the pair term (see RecF32)
//   G = g_0 + g_1x rho^2 + g_2x rho^4
// splits into a column part, a row part and a small cross term:
//   2^G = X * Y * 2^(2 g_2x dx^2 dy^2),
//   X = 2^(g_1x dx^2 + g_2x dx^4)        (one ex2 per thread, visit and snapshot),
//   Y = 2^(g_0 + g_1x dy^2 + g_2x dy^4)  (one ex2 per row, visit and snapshot: shared by
//                                         the whole CTA, formed once per staged visit).
// In the degree-2 class (h <= 0.04) |2 g_2x dx^2 dy^2| <= |g_2x| rho^4 / 2 < 5e-5, so
// 2^z = 1 + z ln 2 to 6e-10, and the term is X Y + A B with A = X (2 ln2 g_2x) dx^2 and
// B = Y dy^2; where the warp's bound of |2 g_2x dx^2 dy^2| is below the series classes'
// 2.5e-7 budget the cross term is dropped and the term is X Y.  A pair then costs one or
// two FMAs (f32x2, two snapshots per instruction) instead of two FMAs, an ex2 and an add:
// the exponentials leave the pair loop.  The other classes (degree 4, the per-snapshot
// path with degrees 8/12 and the two-E1 form) run as in the general tile, with
// rho^2 = dx^2 + dy^2 from the column's dx and the row's dy^2 -- the same roundings as
// the general tile's rho^2.
#pragma once
#include <climits>
#include <cstdint>

#include "dd_field_impl.cuh"

namespace ddk {

// Largest |2 g_2x dx^2 dy^2| (log2 units) for which the cross term is dropped: the series
// classes' truncation budget.
constexpr float kSepCross = 2.5e-7f;
constexpr float kTwoLn2 = 1.38629436112f;

// per (warp, visit): all skipped / degree 2 without the cross term / degree 2 with it /
// all on degree <= 4 / mixed classes
enum : uint32_t { kGModeSkip = 0, kGModeSep1 = 1, kGModeSep2 = 2, kGModeD4 = 3, kGModePer = 4 };

template <typename Cfg>
struct TileSmemGrid {
    static constexpr int ST = Cfg::kSTILE, TCH = 4, NP = 2, PPT = Cfg::kPPT;
    float run[TCH * PPT][Cfg::kThreads];                // per-thread running sums over stages
    float vx[ST], vy[ST];                               // visit minus tile origin (integers)
    float4 pa[NP][ST];                                  // (g_0, g_0', g_1x, g_1x') of pair P
    float4 gm[3][ST];                                   // g_2x, g_3x, g_4x of the 4 snapshots
    float4 g1[ST];                                      // g_1x of the 4 snapshots
    float2 cls[TCH][ST];                                // (dq, q1)
    float4 dy2[ST];                                     // dy^2 of the tile's rows
    float4 yf[ST][PPT];                                 // row factor Y of the 4 snapshots, per row
    float4 bf[ST][PPT];                                 // Y dy^2, per row
    float yin[PPT], yfr[PPT];                           // the rows' y: integer offset + fraction
};

// srcF: visit coordinates, ptsF: point coordinates (float-float, pitch units, row-major
// grid of W columns and H rows); the tile covers columns [128 tc, 128 tc + 128) and rows
// [4 tr, 4 tr + 4).  partial[jc * part_stride + r W + c] receives, for each snapshot jc of
// write_mask, the sum over visits i in [s_begin, s_end) with ks[jc] <= i < na[jc].
template <typename Cfg>
__device__ __forceinline__ void field_tile_grid_mixed(TileSmemGrid<Cfg> &sm, const float4 *__restrict__ srcF,
                                                      const float4 *__restrict__ ptsF, int64_t W, int64_t H,
                                                      int64_t tc, int64_t tr, const RecF32 *const (&rows)[4],
                                                      const int (&na)[4], const int (&ks)[4], uint32_t write_mask,
                                                      int s_begin, int s_end, float *__restrict__ partial,
                                                      int64_t part_stride) {
    constexpr int NT = Cfg::kThreads, PPT = Cfg::kPPT, STILE = Cfg::kSTILE, TCH = 4, NP = 2;
    static_assert(NT == 128 && PPT == 4 && STILE == 32, "grid tile: 128 columns x 4 rows, 32-visit stages");
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t c0 = tc * NT, r0 = tr * PPT;
    const int64_t c = c0 + tid;
    const bool live_c = c < W;
    const int64_t cc = live_c ? c : W - 1;               // a ragged tile's spare columns
                                                         // repeat the last one (not written)
    // Offsets from the integer grid position nearest the tile's first point, as an exact
    // integer plus a fraction (as in the general tile); the column's x for this thread,
    // the rows' y for every thread.
    const float4 org = ptsF[r0 * W + c0];
    const float ox = rintf(org.x), oy = rintf(org.z);
    const float4 qx = ptsF[r0 * W + cc];
    const float ix = rintf(qx.x);
    const float xfr = (qx.x - ix) + qx.y;                // qx.x - ix is exact
    const float xin = ix - ox;                           // exact integer
    // the rows (the same for every thread) go to shared memory
    bool exact = ((xin + xfr) - xin) == xfr;
    float by0 = 3.0e38f, by1 = -3.0e38f;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int64_t rk = min(r0 + k, H - 1);
        const float4 qy = ptsF[rk * W + c0];
        const float iy = rintf(qy.z);
        const float yf = (qy.z - iy) + qy.w, yi = iy - oy;
        exact = exact && ((yi + yf) - yi) == yf;
        by0 = fminf(by0, yi + yf);
        by1 = fmaxf(by1, yi + yf);
        if (tid == k) { sm.yin[k] = yi; sm.yfr[k] = yf; }
    }
    // one vote of the CTA: split offsets only where some point of the tile needs them
    // (the barrier also publishes the rows)
    const bool split = __syncthreads_or(!exact) != 0;
    const float xs = xin + xfr;                          // the whole offset (exact if !split)
    float bx0 = xs, bx1 = xs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bx0 = fminf(bx0, __shfl_xor_sync(0xffffffffu, bx0, o));
        bx1 = fmaxf(bx1, __shfl_xor_sync(0xffffffffu, bx1, o));
    }

    float2 acc[NP][PPT];
#pragma unroll
    for (int m = 0; m < NP; ++m)
#pragma unroll
        for (int k = 0; k < PPT; ++k) acc[m][k] = f2(0.0f, 0.0f);
#pragma unroll
    for (int jc = 0; jc < TCH; ++jc)
#pragma unroll
        for (int k = 0; k < PPT; ++k) sm.run[jc * PPT + k][tid] = 0.0f;

    for (int s0 = s_begin; s0 < s_end; s0 += STILE) {
        const int cnt = min(STILE, s_end - s0);
        __syncthreads();
        for (int i = tid; i < cnt; i += NT) {
            const float4 v = srcF[s0 + i];
            sm.vx[i] = (v.x - ox) + v.y;                 // probe positions are integers
            sm.vy[i] = (v.z - oy) + v.w;
        }
        // records of the four snapshots in the snapshot-pair layout; a snapshot for which
        // the visit has not started gets the zero record (g_0 = -inf, the rest 0)
        constexpr int RV = sizeof(RecF32) / 16;
#pragma unroll
        for (int jc = 0; jc < TCH; ++jc) {
            const float4 *row = reinterpret_cast<const float4 *>(rows[jc] + s0);
            const int lim = na[jc] - s0, lo = ks[jc] - s0;
            for (int v = tid; v < cnt * 2; v += NT) {
                const int i = v >> 1, q = v & 1;
                const float4 r = (i < lim && i >= lo) ? row[i * RV + q]
                                                      : (q == 0 ? zero_rec_v0() : make_float4(0.f, 0.f, 0.f, 0.f));
                if (q == 0) {
                    float *a = reinterpret_cast<float *>(&sm.pa[jc >> 1][i]) + (jc & 1);
                    a[0] = r.x; a[2] = r.y;
                    reinterpret_cast<float *>(&sm.g1[i])[jc] = r.y;
                    reinterpret_cast<float *>(&sm.gm[0][i])[jc] = r.z;
                    reinterpret_cast<float *>(&sm.gm[1][i])[jc] = r.w;
                } else {
                    reinterpret_cast<float *>(&sm.gm[2][i])[jc] = r.x;
                    sm.cls[jc][i] = make_float2(r.y, r.z);
                }
            }
        }
        __syncthreads();
        // Row tables: thread (visit i = tid / 4, row k = tid % 4) forms dy^2 and, for the
        // four snapshots, Y = 2^(g_0 + g_1x dy^2 + g_2x dy^4) and Y dy^2.
        {
            const int i = tid >> 2, k = tid & 3;
            if (i < cnt) {
                const float vy = sm.vy[i], yi = sm.yin[k], yf = sm.yfr[k];
                const float dy = split ? (yi - vy) + yf : (yi + yf) - vy;
                const float d2 = dy * dy;
                const float4 p0 = sm.pa[0][i], p1 = sm.pa[1][i], g2 = sm.gm[0][i];
                const float y0 = ex2_approx(fmaf(d2, fmaf(g2.x, d2, p0.z), p0.x));
                const float y1 = ex2_approx(fmaf(d2, fmaf(g2.y, d2, p0.w), p0.y));
                const float y2 = ex2_approx(fmaf(d2, fmaf(g2.z, d2, p1.z), p1.x));
                const float y3 = ex2_approx(fmaf(d2, fmaf(g2.w, d2, p1.w), p1.y));
                sm.yf[i][k] = make_float4(y0, y1, y2, y3);
                sm.bf[i][k] = make_float4(y0 * d2, y1 * d2, y2 * d2, y3 * d2);
                reinterpret_cast<float *>(&sm.dy2[i])[k] = d2;
            }
        }
        // Class words and modes per (warp, visit), lane i classifying staged visit i
        // against its warp's box (32 columns x the tile's rows), as in the general tile;
        // a visit whose every snapshot is on degree 2 (or not started) takes the separable
        // form, without the cross term where its bound allows.
        uint32_t my_word = 0, my_mode = kGModeSkip;
        if (lane < cnt) {
            const float sx = sm.vx[lane], sy = sm.vy[lane];
            float r2min, r2max;
            box_rho2(sx, sy, bx0, bx1, by0, by1, r2min, r2max);
            const float dxm = fmaxf(fabsf(sx - bx0), fabsf(sx - bx1));
            const float dym = fmaxf(fabsf(sy - by0), fabsf(sy - by1));
            const float xy4 = (dxm * dxm) * (dym * dym) * 1.0001f + 1e-6f;
            const float4 g2 = sm.gm[0][lane];
            uint32_t codes = 0, cmin = kCodeGeneral, cmax = kCodeSkip;
            bool any = false, small_cross = true;
#pragma unroll
            for (int jc = 0; jc < TCH; ++jc) {
                uint32_t cl = kCodeD2, code = kCodeSkip;
                if (s0 + lane < na[jc] && s0 + lane >= ks[jc]) {
                    const float2 h = sm.cls[jc][lane];
                    cl = code = series_class(r2max * h.x, r2min * h.y, h.x);
                    any = any || cl != kCodeSkip;
                    const float g2x = jc == 0 ? g2.x : jc == 1 ? g2.y : jc == 2 ? g2.z : g2.w;
                    small_cross = small_cross && 2.0f * fabsf(g2x) * xy4 <= kSepCross;
                }
                cmin = min(cmin, cl);
                cmax = max(cmax, cl);
                codes |= code << (kCodeBits * jc);
            }
            my_word = codes;
            my_mode = !any ? kGModeSkip
                    : (cmin >= kCodeD2 && cmax == kCodeD2) ? (small_cross ? kGModeSep1 : kGModeSep2)
                    : (cmin >= kCodeD2 && cmax == kCodeD4) ? kGModeD4 : kGModePer;
        }
        __syncthreads();                   // row tables visible
        const uint32_t m1 = __ballot_sync(0xffffffffu, my_mode == kGModeSep1);
        const uint32_t m2 = __ballot_sync(0xffffffffu, my_mode == kGModeSep2);
        const uint32_t m4 = __ballot_sync(0xffffffffu, my_mode == kGModeD4);
        const uint32_t mp = __ballot_sync(0xffffffffu, my_mode == kGModePer);
        // degree 2 without the cross term: term = X Y
        for (uint32_t m = m1; m; m &= m - 1) {
            const int s = __ffs(m) - 1;
            const float4 g1 = sm.g1[s], g2 = sm.gm[0][s];
            const float vx = sm.vx[s];
            const float dx = split ? (xin - vx) + xfr : xs - vx;
            const float d2 = dx * dx;
            const float2 dd = f2(d2, d2);
            const float2 e0 = __fmul2_rn(__ffma2_rn(f2(g2.x, g2.y), dd, f2(g1.x, g1.y)), dd);
            const float2 e1 = __fmul2_rn(__ffma2_rn(f2(g2.z, g2.w), dd, f2(g1.z, g1.w)), dd);
            const float2 X0 = f2(ex2_approx(e0.x), ex2_approx(e0.y));
            const float2 X1 = f2(ex2_approx(e1.x), ex2_approx(e1.y));
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const float4 y = sm.yf[s][k];
                acc[0][k] = __ffma2_rn(X0, f2(y.x, y.y), acc[0][k]);
                acc[1][k] = __ffma2_rn(X1, f2(y.z, y.w), acc[1][k]);
            }
        }
        // degree 2 with the cross term: term = X Y + A B
        for (uint32_t m = m2; m; m &= m - 1) {
            const int s = __ffs(m) - 1;
            const float4 g1 = sm.g1[s], g2 = sm.gm[0][s];
            const float vx = sm.vx[s];
            const float dx = split ? (xin - vx) + xfr : xs - vx;
            const float d2 = dx * dx;
            const float2 dd = f2(d2, d2);
            const float2 g20 = f2(g2.x, g2.y), g21 = f2(g2.z, g2.w);
            const float2 e0 = __fmul2_rn(__ffma2_rn(g20, dd, f2(g1.x, g1.y)), dd);
            const float2 e1 = __fmul2_rn(__ffma2_rn(g21, dd, f2(g1.z, g1.w)), dd);
            const float2 X0 = f2(ex2_approx(e0.x), ex2_approx(e0.y));
            const float2 X1 = f2(ex2_approx(e1.x), ex2_approx(e1.y));
            const float2 A0 = __fmul2_rn(X0, __fmul2_rn(__fmul2_rn(g20, f2(kTwoLn2, kTwoLn2)), dd));
            const float2 A1 = __fmul2_rn(X1, __fmul2_rn(__fmul2_rn(g21, f2(kTwoLn2, kTwoLn2)), dd));
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const float4 y = sm.yf[s][k], bb = sm.bf[s][k];
                acc[0][k] = __ffma2_rn(A0, f2(bb.x, bb.y), __ffma2_rn(X0, f2(y.x, y.y), acc[0][k]));
                acc[1][k] = __ffma2_rn(A1, f2(bb.z, bb.w), __ffma2_rn(X1, f2(y.z, y.w), acc[1][k]));
            }
        }
        // degree <= 4 for every snapshot: 2^(g_0 + g_1x r + ... + g_4x r^4) on snapshot pairs
        for (uint32_t m = m4; m; m &= m - 1) {
            const int s = __ffs(m) - 1;
            const float4 g2 = sm.gm[0][s], g3 = sm.gm[1][s], g4 = sm.gm[2][s], dy = sm.dy2[s];
            const float4 va[NP] = {sm.pa[0][s], sm.pa[1][s]};
            const float2 g2p[NP] = {f2(g2.x, g2.y), f2(g2.z, g2.w)};
            const float2 g3p[NP] = {f2(g3.x, g3.y), f2(g3.z, g3.w)};
            const float2 g4p[NP] = {f2(g4.x, g4.y), f2(g4.z, g4.w)};
            const float vx = sm.vx[s];
            const float dx = split ? (xin - vx) + xfr : xs - vx;
            const float r2[PPT] = {fmaf(dx, dx, dy.x), fmaf(dx, dx, dy.y), fmaf(dx, dx, dy.z), fmaf(dx, dx, dy.w)};
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
        // the rest: one snapshot at a time, each at its own class, whole records from
        // global memory
        for (uint32_t m = mp; m; m &= m - 1) {
            const int s = __ffs(m) - 1;
            const uint32_t word = __shfl_sync(0xffffffffu, my_word, s);
            const float4 dy = sm.dy2[s];
            const float vx = sm.vx[s];
            const float dx = split ? (xin - vx) + xfr : xs - vx;
            const float r2[PPT] = {fmaf(dx, dx, dy.x), fmaf(dx, dx, dy.y), fmaf(dx, dx, dy.z), fmaf(dx, dx, dy.w)};
#pragma unroll
            for (int jc = 0; jc < TCH; ++jc) {
                const uint32_t cl = (word >> (kCodeBits * jc)) & kCodeMask;
                if (cl == kCodeSkip) continue;
                const RecF32 &Rs = rows[jc][s0 + s];            // active: the record exists
                float2 (&A)[PPT] = acc[jc >> 1];
                if (cl == kCodeD2) {
                    if (jc & 1) moment_pass<2, PPT, 1>(A, r2, Rs); else moment_pass<2, PPT, 0>(A, r2, Rs);
                } else if (cl == kCodeD4) {
                    if (jc & 1) moment_pass<4, PPT, 1>(A, r2, Rs); else moment_pass<4, PPT, 0>(A, r2, Rs);
                } else if (cl == kCodeD8) {
                    if (jc & 1) moment_pass<8, PPT, 1>(A, r2, Rs); else moment_pass<8, PPT, 0>(A, r2, Rs);
                } else if (cl == kCodeD12) {
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
#pragma unroll
        for (int jc = 0; jc < TCH; ++jc)
#pragma unroll
            for (int k = 0; k < PPT; ++k)
                sm.run[jc * PPT + k][tid] += (jc & 1) ? acc[jc >> 1][k].y : acc[jc >> 1][k].x;
#pragma unroll
        for (int m = 0; m < NP; ++m)
#pragma unroll
            for (int k = 0; k < PPT; ++k) acc[m][k] = f2(0.0f, 0.0f);
    }
#pragma unroll
    for (int jc = 0; jc < TCH; ++jc) {
        if (!((write_mask >> jc) & 1u)) continue;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int64_t r = r0 + k;
            if (live_c && r < H) partial[(int64_t)jc * part_stride + r * W + c] = sm.run[jc * PPT + k][tid];
        }
    }
}

// One work item per CTA, as field_kernel, over grid tiles: CTA item0 + blockIdx.x takes
// descriptor (item0 + blockIdx.x) / n_tiles and grid tile (item0 + blockIdx.x) % n_tiles,
// tile q covering column block q % n_tc and row block q / n_tc.
// kst (NULL: none): snapshot j's visits below kst[j] are summed by the tensor-core
// contraction (dd_field_tc.cuh); this kernel takes visits [kst[j], nact[j]) and writes the
// partial row of block k only where the block reaches past kst[j] ((k + 1) sb > kst[j]).
template <typename Cfg>
__global__ void __launch_bounds__(Cfg::kThreads, Cfg::kMinBlocks)
field_grid_kernel(int64_t W, int64_t H, int64_t n_tc, const RecF32 *__restrict__ rec,
                  const int64_t *__restrict__ row_off, const int *__restrict__ nact, const int *__restrict__ kst,
                  const int2 *__restrict__ desc, int64_t n_tiles, int64_t item0, int n_tg, int sb,
                  float *__restrict__ partial, int64_t pstride, const float4 *__restrict__ srcF,
                  const float4 *__restrict__ ptsF) {
    constexpr int TCH = Cfg::kTCH;
    static_assert(TCH == 4, "grid tile: four snapshots");
    const int64_t q = item0 + blockIdx.x;
    const int2 dc = desc[q / n_tiles];                     // (chunk, block)
    const int64_t tile = q % n_tiles;
    const int j0 = dc.x * TCH;
    const int s_begin = dc.y * sb;
    int na[TCH], ks[TCH];
    const RecF32 *rows[TCH];
    int nmax = 0, kmin = INT_MAX;
    uint32_t write_mask = 0;
#pragma unroll
    for (int jc = 0; jc < TCH; ++jc) {
        const bool live = j0 + jc < n_tg;
        na[jc] = live ? nact[j0 + jc] : 0;
        ks[jc] = live && kst ? kst[j0 + jc] : 0;
        rows[jc] = live ? rec + row_off[j0 + jc] : rec;
        nmax = max(nmax, na[jc]);
        if (live) {
            kmin = min(kmin, ks[jc]);
            if (s_begin + sb > ks[jc]) write_mask |= 1u << jc;
        }
    }
    const int s_end = min(s_begin + sb, nmax);
    float *part = partial + ((int64_t)dc.y * n_tg + j0) * pstride;
    __shared__ TileSmemGrid<Cfg> sm;
    field_tile_grid_mixed<Cfg>(sm, srcF, ptsF, W, H, tile % n_tc, tile / n_tc, rows, na, ks, write_mask,
                               max(s_begin, kmin), s_end, part, pstride);
}

}  // namespace ddk
