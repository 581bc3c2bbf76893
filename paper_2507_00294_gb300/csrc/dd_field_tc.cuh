// dd_field_tc.cuh -- the older visits' part of the FP32-mixed field on a grid of points as
// a contraction on the 5th-generation tensor cores.
//
// For a grid point (column c, row r) and a visit i whose pair term is on the degree-2
// exponent series over a whole tile of points (h = rho^2 dq <= 0.04 for every point), the
// separable form of dd_field_grid.cuh gives, with x = dx^2, y = dy^2,
//   term(r, c; i) = Y_i(r) X_i(c) + B_i(r) A_i(c),
//   X = 2^(g_1x x + g_2x x^2),  A = X (2 ln2 g_2x) x,
//   Y = 2^(g_0 + g_1x y + g_2x y^2),  B = Y y,
// so the sum over such visits is a matrix product: F(r, c) = sum_i Y(r, i) X(i, c) +
// B(r, i) A(i, c), M = 128 rows x N = 128 columns per tile, K = visits.  The factors are
// formed in FP32 exactly as the CUDA-core tile forms them and split into BF16 pieces,
// X = X_h + X_m + X_l (each piece the round-to-nearest BF16 of what the earlier ones leave,
// |X - X_h - X_m - X_l| <= 2^-24 |X|); the six products X_h Y_h, X_h Y_m, X_m Y_h, X_h Y_l,
// X_l Y_h, X_m Y_m keep X Y to about 4 2^-24 relative, and the cross term, at most 3.5e-5
// of X Y in the degree-2 class, takes one product of the BF16 roundings (2^-7 of itself, at
// most 2.6e-7 of X Y).  Seven MMAs per 16 visits.
//
// Degree 4 (0.04 < h <= 0.33 at every point): the exponent G = g_0 + sum_m g_mx (x + y)^m,
// m <= 4, splits into X = 2^(sum_m g_mx x^m), Y = 2^(g_0 + sum_m g_mx y^m) and the cross part
// C = g_2x 2xy + g_3x (3x^2 y + 3x y^2) + g_4x (4x^3 y + 6x^2 y^2 + 4x y^3), |C| <= 3.5e-3
// (log2 units) in the class, so that with z = C ln2, 2^C = 1 + z + z^2/2 to 3e-9; of z^2/2
// only (2 ln2 g_2x xy)^2 / 2 exceeds 2.5e-7.  Grouped by powers of y:
//   term = X Y + A_1 B_1 + A_2 B_2 + A_3 B_3,  B_k = y^k Y,
//   A_1 = X ln2 x (2 g_2x + 3 g_3x x + 4 g_4x x^2),
//   A_2 = X x (3 ln2 g_3x + (6 ln2 g_4x + 2 ln2^2 g_2x^2) x),  A_3 = X ln2 4 g_4x x,
// |A_1 B_1| <= 2.3e-3, |A_2 B_2| <= 1.5e-4, |A_3 B_3| <= 4e-6 of X Y: A_1 and B_1 in two
// BF16 pieces (three products), A_2 in two and B_2 in one (two products), A_3 B_3 in one;
// twelve MMAs per 16 visits.
//
// The products accumulate in FP32 in tensor memory (kind::f16, tcgen05.mma issued by one
// thread): X_h Y_h into one accumulator and the small products (at most 2^-7 of it) into a
// second.  The tensor core's FP32 accumulation drops low bits in each MMA (the sums of
// positive terms come out slightly low); keeping the leading product apart makes that loss
// one MMA per 16 visits instead of seven or twelve, and the small products' losses 2^-7
// smaller.
//
// Work item: one 128 x 128 tile, one snapshot j and a range of the snapshot's degree-2 (or
// degree-4) visits (about one item per resident CTA), staged kTcMaxChunk visits at a time.
// Persistent CTAs walk the items (item blockIdx.x, then every gridDim.x-th).  Warps 0-7
// produce: thread t < 128 forms the factors of row r0 + t, thread 128 + t those of column
// c0 + t, 16 visits at a time, into one of three shared-memory stages, and arrives on the
// stage's "full" barrier; lane 0 of warp 8 waits for it, issues the stage's MMAs and commits
// them to the stage's "empty" barrier, which the producers wait on before they write that
// stage again -- no CTA-wide barrier inside the item.  After an item's last stage the MMA
// thread commits to the "done" barrier; the producers then read the accumulators (warp w:
// rows 32 (w % 4) .., columns 64 (w / 4) ..) into shared memory and write the FP32 partial
// sums of the item as whole rows.
#pragma once
#include <cstdint>

#include "dd_field_impl.cuh"
#include "dd_umma.cuh"

namespace ddk {

constexpr int kTcGenThreads = 256;         // warps 0-3: row factors, warps 4-7: column factors
constexpr int kTcThreads = kTcGenThreads + 32;                 // + warp 8: issues the MMAs
constexpr int kTcTile = 128;                 // rows = columns of a tile (M = N = 128)
constexpr int kTcStage = 16;                 // visits per stage: one K step of the BF16 MMA
constexpr int kTcBufs = 3;                   // stages in flight
constexpr int kTcMaxChunk = 256;             // visits per coefficient staging (segment of an item)
constexpr int kTcScratchStride = kTcTile + 4; // floats per row of the epilogue's transpose
constexpr int kTcPieceBytes = kTcTile * kTcStage * 2;          // 4 KB: 128 rows x 16 BF16
constexpr int kTcMaxItemStages = 32;         // stages per item (one partial row) at most: the
                                             // tensor core's FP32 accumulation drops up to an ulp
                                             // of the sum per MMA, so a sum takes at most 32
                                             // leading-product MMAs (<= 32 2^-23 relative)
constexpr int kTcWaitTries = 1 << 18;        // completion waits: at most about 0.26 s
constexpr float kTcLn2 = 0.693147180560f;
constexpr float kTcTwoLn2 = 1.38629436112f;

// Per degree: the BF16 pieces of a stage (rows, then columns: 4 + 4 or 7 + 8 of 4 KB), the
// coefficient vectors per visit pair, and the CTAs per SM (shared memory and 256 TMEM
// columns each).
template <int kDeg>
struct TcShape;
template <>
struct TcShape<2> {
    static constexpr int kRowPieces = 4, kColPieces = 4, kCoefVecs = 3, kCtasPerSm = 2;
};
template <>
struct TcShape<4> {
    static constexpr int kRowPieces = 7, kColPieces = 8, kCoefVecs = 6, kCtasPerSm = 1;
};
template <int kDeg>
struct TcConst {
    using S = TcShape<kDeg>;
    static constexpr int kBufBytes = (S::kRowPieces + S::kColPieces) * kTcPieceBytes;
    static constexpr int kCoefBytes = S::kCoefVecs * (kTcMaxChunk / 2) * 16;
    static constexpr int kSmemBytes = kTcBufs * kBufBytes + kCoefBytes + 128;
};
// set when a completion wait of the contraction gives up (its partial sums are then NaN)
static __device__ int g_field_tc_timeout;

// Work item: visits [v_begin, v_end) of one snapshot's degree-2 (degree-4) range on one tile (row
// block * n_tile_cols + column block); its sums go to partial row `row`; the snapshot's
// records start at rec + row_off.
struct TcItem {
    int v_begin, v_end, tile, row;
    int64_t row_off;
    int scan, pad;          // the item's entry in a batch's scan table (0 for one grid)
};
static_assert(sizeof(TcItem) == 32, "TcItem layout");

// The grid of points, the visits and the partial rows of the work items: one entry (a
// kernel argument) for dd_field_on_grid, a table indexed by TcItem::scan for a batch of
// scans, each on its own grid.  Item `row` writes partial + row * pstride + r W + c.
struct TcScan {
    int64_t W, H, n_tile_cols;
    const float4 *srcF, *ptsF;      // visits and points, float-float in pitch units
    float *partial;
    int64_t pstride;                // a multiple of 4 (16-byte aligned rows)
};
__device__ __forceinline__ TcScan tc_scan(const TcScan &one, const TcScan *many, const TcItem &it) {
    return many ? many[it.scan] : one;
}

__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ float2 bf16x2_to_f2(uint32_t w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
}
// v = h + m + l in BF16 pieces (packed pairs), each the rounding of what the earlier leave;
// the remainders are exact in FP32
__device__ __forceinline__ void split3_bf16(float2 v, uint32_t &h, uint32_t &m, uint32_t &l) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    h = bf16x2_rn(v.x, v.y);
    const float2 r1 = __ffma2_rn(bf16x2_to_f2(h), m1, v);
    m = bf16x2_rn(r1.x, r1.y);
    const float2 r2 = __ffma2_rn(bf16x2_to_f2(m), m1, r1);
    l = bf16x2_rn(r2.x, r2.y);
}

// v = h + l in BF16 pieces (packed pairs): |v - h - l| <= 2^-16 |v|
__device__ __forceinline__ void split2_bf16(float2 v, uint32_t &h, uint32_t &l) {
    h = bf16x2_rn(v.x, v.y);
    const float2 r1 = __ffma2_rn(bf16x2_to_f2(h), make_float2(-1.0f, -1.0f), v);
    l = bf16x2_rn(r1.x, r1.y);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}
// the 256 producer threads only (warps 0-7)
__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, %0;" :: "n"(kTcGenThreads) : "memory"); }

// The loads of one segment's inputs, issued early (the next segment's while the current one
// runs): the tile's first point and this thread's row or column point, and for thread p below
// the segment's pair count the coordinates and leading coefficients of its visits 2p, 2p + 1
// (record vector 0: g_0, g_1x, g_2x, g_3x; for degree 4 also vector 1: g_4x, ...).
template <int kDeg>
struct TcPrefetch {
    float4 org, pt, v[2], r[2], r1[2];
};
template <int kDeg>
__device__ __forceinline__ void tc_prefetch(TcPrefetch<kDeg> &f, const TcItem &it, int s0, const TcScan &S,
                                            const RecF32 *__restrict__ rec, int tid) {
    const int64_t W = S.W, H = S.H;
    const float4 *__restrict__ srcF = S.srcF;
    const float4 *__restrict__ ptsF = S.ptsF;
    const int64_t r0 = (it.tile / S.n_tile_cols) * (int64_t)kTcTile, c0 = (it.tile % S.n_tile_cols) * (int64_t)kTcTile;
    const int t = tid & (kTcTile - 1);
    f.org = ptsF[r0 * W + c0];
    f.pt = tid >= kTcTile ? ptsF[r0 * W + min(c0 + t, W - 1)] : ptsF[min(r0 + t, H - 1) * W + c0];
    const int nv = min(it.v_end - s0, kTcMaxChunk);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int i = 2 * tid + e;
        if (i < nv) {
            f.v[e] = srcF[s0 + i];
            const float4 *rv = reinterpret_cast<const float4 *>(rec + it.row_off + s0 + i);
            f.r[e] = rv[0];
            if (kDeg == 4) f.r1[e] = rv[1];
        }
    }
}

// Coefficient vectors of visit pair p (visits a, b), from the prefetched inputs; the padding
// to whole stages contributes 0 (g_0 = -inf: Y = 0 and every row piece is 0).
//   degree 2: (-x, -y), (g_1x, g_2x), (g_0, 2 ln2 g_2x)
//   degree 4: (-x, -y), (g_1x, g_2x), (g_0, g_3x), (g_4x, 2 ln2 g_2x), (3 ln2 g_3x,
//             4 ln2 g_4x), (6 ln2 g_4x + 2 ln2^2 g_2x^2, 0)
template <int kDeg>
__device__ __forceinline__ void tc_stage_coefs(float4 *cf, const TcPrefetch<kDeg> &pf, int p, int nv, float ox,
                                               float oy) {
    float vx[2], vy[2], g0[2], g1[2], g2[2], g3[2], g4[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        if (2 * p + e < nv) {
            vx[e] = (pf.v[e].x - ox) + pf.v[e].y;        // probe positions are integers
            vy[e] = (pf.v[e].z - oy) + pf.v[e].w;
            g0[e] = pf.r[e].x; g1[e] = pf.r[e].y; g2[e] = pf.r[e].z; g3[e] = pf.r[e].w;
            g4[e] = kDeg == 4 ? pf.r1[e].x : 0.0f;
        } else {
            vx[e] = vy[e] = 0.0f; g0[e] = -INFINITY; g1[e] = g2[e] = g3[e] = g4[e] = 0.0f;
        }
    }
    constexpr int NP = kTcMaxChunk / 2;
    cf[p] = make_float4(-vx[0], -vx[1], -vy[0], -vy[1]);
    cf[NP + p] = make_float4(g1[0], g1[1], g2[0], g2[1]);
    if (kDeg == 2) {
        cf[2 * NP + p] = make_float4(g0[0], g0[1], kTcTwoLn2 * g2[0], kTcTwoLn2 * g2[1]);
    } else {
        cf[2 * NP + p] = make_float4(g0[0], g0[1], g3[0], g3[1]);
        cf[3 * NP + p] = make_float4(g4[0], g4[1], kTcTwoLn2 * g2[0], kTcTwoLn2 * g2[1]);
        cf[4 * NP + p] = make_float4(3.0f * kTcLn2 * g3[0], 3.0f * kTcLn2 * g3[1], 4.0f * kTcLn2 * g4[0],
                                     4.0f * kTcLn2 * g4[1]);
        cf[5 * NP + p] = make_float4(fmaf(6.0f * kTcLn2, g4[0], 2.0f * kTcLn2 * kTcLn2 * g2[0] * g2[0]),
                                     fmaf(6.0f * kTcLn2, g4[1], 2.0f * kTcLn2 * kTcLn2 * g2[1] * g2[1]), 0.0f, 0.0f);
    }
}

// The BF16 pieces of four visit pairs (one K group of 8 visits) for this thread's row or
// column, stored as one 16-byte core-matrix row per piece: piece k at buf + k * 4 KB (rows
// first, then columns), K group kg at + kg * 2 KB, row (column) t at + t * 16.
template <int kDeg>
__device__ __forceinline__ void tc_produce_group(unsigned char *buf, const float4 *cf, int p0, int kg, int t,
                                                 bool col_side, float2 din2, float2 dfr2) {
    using S = TcShape<kDeg>;
    constexpr int NP = kTcMaxChunk / 2, PW = kTcPieceBytes / 16;
    constexpr int NPC = S::kColPieces > S::kRowPieces ? S::kColPieces : S::kRowPieces;
    uint32_t w[NPC][4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int p = p0 + u;
        const float4 P0 = cf[p], P1 = cf[NP + p], P2 = cf[2 * NP + p];
        const float2 g1 = f2(P1.x, P1.y), g2 = f2(P1.z, P1.w);
        const float2 nv2 = col_side ? f2(P0.x, P0.y) : f2(P0.z, P0.w);
        const float2 dd = __fadd2_rn(__fadd2_rn(din2, nv2), dfr2);
        const float2 d2 = __fmul2_rn(dd, dd);
        if (kDeg == 2) {
            // Row: F = Y = 2^(g_0 + g_1x y + g_2x y^2), cross piece B = Y y.  Column:
            // F = X = 2^(g_1x x + g_2x x^2) (the roundings of (g_2x x + g_1x) x), cross piece
            // A = X ((2 ln2 g_2x) x).
            const float2 g0 = col_side ? f2(0.0f, 0.0f) : f2(P2.x, P2.y);
            const float2 mul = col_side ? f2(P2.z, P2.w) : f2(1.0f, 1.0f);
            const float2 e = __ffma2_rn(__ffma2_rn(g2, d2, g1), d2, g0);
            const float2 F = f2(ex2_approx(e.x), ex2_approx(e.y));
            const float2 C = __fmul2_rn(F, __fmul2_rn(mul, d2));
            split3_bf16(F, w[0][u], w[1][u], w[2][u]);
            w[3][u] = bf16x2_rn(C.x, C.y);
        } else {
            const float4 P3 = cf[3 * NP + p], P4 = cf[4 * NP + p], P5 = cf[5 * NP + p];
            const float2 g3 = f2(P2.z, P2.w), g4 = f2(P3.x, P3.y);
            // exponent part of this row or column: sum_m g_mx d2^m (+ g_0 on a row)
            const float2 g0 = col_side ? f2(0.0f, 0.0f) : f2(P2.x, P2.y);
            const float2 e = __ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(g4, d2, g3), d2, g2), d2, g1), d2, g0);
            const float2 F = f2(ex2_approx(e.x), ex2_approx(e.y));
            split3_bf16(F, w[0][u], w[1][u], w[2][u]);
            if (col_side) {
                // A_1 = X x (2 ln2 g_2x + x (3 ln2 g_3x + x 4 ln2 g_4x)), A_2 = X x (3 ln2
                // g_3x + x (6 ln2 g_4x + 2 ln2^2 g_2x^2)), A_3 = X x 4 ln2 g_4x
                const float2 c1 = f2(P3.z, P3.w), c2 = f2(P4.x, P4.y), c3 = f2(P4.z, P4.w), c6 = f2(P5.x, P5.y);
                const float2 Fx = __fmul2_rn(F, d2);
                const float2 A1 = __fmul2_rn(Fx, __ffma2_rn(__ffma2_rn(c3, d2, c2), d2, c1));
                const float2 A2 = __fmul2_rn(Fx, __ffma2_rn(c6, d2, c2));
                const float2 A3 = __fmul2_rn(Fx, c3);
                split2_bf16(A1, w[3][u], w[4][u]);
                split2_bf16(A2, w[5][u], w[6][u]);
                w[7][u] = bf16x2_rn(A3.x, A3.y);
            } else {
                // B_k = y^k Y
                const float2 B1 = __fmul2_rn(F, d2), B2 = __fmul2_rn(B1, d2), B3 = __fmul2_rn(B2, d2);
                split2_bf16(B1, w[3][u], w[4][u]);
                w[5][u] = bf16x2_rn(B2.x, B2.y);
                w[6][u] = bf16x2_rn(B3.x, B3.y);
            }
        }
    }
    uint4 *const q = reinterpret_cast<uint4 *>(buf + (col_side ? S::kRowPieces * kTcPieceBytes : 0) +
                                               kg * (kTcPieceBytes / 2) + t * 16);
    const int np = col_side ? S::kColPieces : S::kRowPieces;
#pragma unroll
    for (int k = 0; k < NPC; ++k)
        if (k < np) q[k * PW] = make_uint4(w[k][0], w[k][1], w[k][2], w[k][3]);
}

// The MMAs of one stage: A = row pieces (M = rows), B = column pieces (N = columns); K-major,
// core matrices of 8 rows: SBO 128 bytes, LBO (next 8 visits) 2 KB.  tmem: the leading
// product's accumulator; tmem + 128: the rest.
template <int kDeg>
__device__ __forceinline__ void tc_issue_stage(uint32_t base, uint32_t tmem, int acc) {
    using S = TcShape<kDeg>;
    constexpr uint32_t idesc = umma_idesc_bf16(kTcTile, kTcTile);
    auto rowp = [&](int k) { return umma_smem_desc(base + k * kTcPieceBytes, kTcPieceBytes / 2, 128u); };
    auto colp = [&](int k) { return umma_smem_desc(base + (S::kRowPieces + k) * kTcPieceBytes, kTcPieceBytes / 2, 128u); };
    const uint32_t t2 = tmem + (uint32_t)kTcTile;
    umma_bf16(tmem, rowp(0), colp(0), idesc, acc);          // Y_h X_h
    umma_bf16(t2, rowp(0), colp(1), idesc, acc);            // Y_h X_m
    umma_bf16(t2, rowp(1), colp(0), idesc, 1);              // Y_m X_h
    umma_bf16(t2, rowp(0), colp(2), idesc, 1);              // Y_h X_l
    umma_bf16(t2, rowp(2), colp(0), idesc, 1);              // Y_l X_h
    umma_bf16(t2, rowp(1), colp(1), idesc, 1);              // Y_m X_m
    if (kDeg == 2) {
        umma_bf16(t2, rowp(3), colp(3), idesc, 1);          // B A
    } else {
        umma_bf16(t2, rowp(3), colp(3), idesc, 1);          // B1_h A1_h
        umma_bf16(t2, rowp(3), colp(4), idesc, 1);          // B1_h A1_l
        umma_bf16(t2, rowp(4), colp(3), idesc, 1);          // B1_l A1_h
        umma_bf16(t2, rowp(5), colp(5), idesc, 1);          // B2 A2_h
        umma_bf16(t2, rowp(5), colp(6), idesc, 1);          // B2 A2_l
        umma_bf16(t2, rowp(6), colp(7), idesc, 1);          // B3 A3
    }
}

// Item `row` of scan table entry S (tc_scan) writes S.partial[row * S.pstride + r W + c].
template <int kDeg>
__global__ void __launch_bounds__(kTcThreads, TcShape<kDeg>::kCtasPerSm)
field_grid_tc_kernel(const TcScan one, const TcScan *__restrict__ many, const RecF32 *__restrict__ rec,
                     const TcItem *__restrict__ items, int n_items, int withhold_mma) {
    using C = TcConst<kDeg>;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char *bufs = tc_smem;
    float4 *cf = reinterpret_cast<float4 *>(tc_smem + kTcBufs * C::kBufBytes);   // [vecs][kTcMaxChunk / 2]
    uint64_t *full = reinterpret_cast<uint64_t *>(tc_smem + kTcBufs * C::kBufBytes + C::kCoefBytes);
    uint64_t *empty = full + kTcBufs;
    uint64_t *done = empty + kTcBufs;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kGenWarps = kTcGenThreads / 32;
    static_assert(kTcTile * kTcScratchStride * 4 <= kTcBufs * C::kBufBytes, "epilogue scratch inside the stages");

    if (warp == kGenWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" :: "r"(smem_u32(s_tmem)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        if (lane == 0) {
            for (int k = 0; k < kTcBufs; ++k) {
                mbar_init(full + k, kGenWarps);          // one arrival per producer warp
                mbar_init(empty + k, 1);
            }
            mbar_init(done, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;                   // columns [0, 128): X_h Y_h; [128, 256): the rest

    bool ok = true;
    if (warp == kGenWarps) {
        // ---- the MMA thread
        if (lane == 0) {
            int gs = 0;
            for (int q = blockIdx.x; q < n_items; q += gridDim.x) {
                const TcItem it = items[q];
                const int nst = (it.v_end - it.v_begin + kTcStage - 1) / kTcStage;
                for (int st = 0; st < nst; ++st) {
                    const int g = gs + st, b = g % kTcBufs;
                    ok = mbar_wait_bounded(full + b, (uint32_t)(g / kTcBufs) & 1u, kTcWaitTries) && ok;
                    tc_fence_after();
                    if (!withhold_mma) tc_issue_stage<kDeg>(smem_u32(bufs + b * C::kBufBytes), tmem, st > 0 ? 1 : 0);
                    umma_commit(empty + b);                     // the stage may be rewritten
                }
                // DD_FAULT=field_tc_wait: the MMAs are withheld and so is this commit, so
                // that the producers' wait for the item runs out
                if (!withhold_mma) umma_commit(done);
                gs += nst;
            }
        }
        __syncwarp();
    } else {
        // ---- the producers
        const bool col_side = tid >= kTcTile;              // warp-uniform
        const int t = tid & (kTcTile - 1);
        const int G = (int)gridDim.x;
        int q = blockIdx.x;
        TcItem it = items[min(q, n_items - 1)];
        TcItem nxt = items[min(q + G, n_items - 1)];
        int s0 = it.v_begin;
        TcPrefetch<kDeg> pf;
        tc_prefetch<kDeg>(pf, it, s0, tc_scan(one, many, it), rec, tid);
        int gs = 0, n_done = 0;
        float *const scr = reinterpret_cast<float *>(bufs);
        while (q < n_items) {
            const int64_t n_tile_cols = tc_scan(one, many, it).n_tile_cols;
            const int64_t r0 = (it.tile / n_tile_cols) * (int64_t)kTcTile;
            const int64_t c0 = (it.tile % n_tile_cols) * (int64_t)kTcTile;
            const int s1 = min(s0 + kTcMaxChunk, it.v_end), nv = s1 - s0;
            const int nst = (nv + kTcStage - 1) / kTcStage;
            // this thread's row (or column): its offset from the integer grid position
            // nearest the tile's first point, as an exact integer plus a fraction (as in the
            // CUDA-core tile); a ragged tile's spare rows and columns repeat the last ones
            // (not written)
            const float ox = rintf(pf.org.x), oy = rintf(pf.org.z);
            float din, dfr;
            if (col_side) {
                const float ix = rintf(pf.pt.x);
                dfr = (pf.pt.x - ix) + pf.pt.y;
                din = ix - ox;
            } else {
                const float iy = rintf(pf.pt.z);
                dfr = (pf.pt.z - iy) + pf.pt.w;
                din = iy - oy;
            }
            // the segment's coefficients, once the previous segment's readers (and the
            // previous item's epilogue, whose scratch is the stage buffers) are done
            producers_sync();
            if (tid < nst * (kTcStage / 2)) tc_stage_coefs<kDeg>(cf, pf, tid, nv, ox, oy);
            producers_sync();
            // the next segment (of this item, else the next item's first), its inputs in
            // flight while this one runs
            const bool last_seg = s1 >= it.v_end;
            const int nq_ = last_seg ? q + G : q;
            const TcItem nit = last_seg ? nxt : it;
            const int ns0 = last_seg ? nit.v_begin : s1;
            if (nq_ < n_items) tc_prefetch<kDeg>(pf, nit, ns0, tc_scan(one, many, nit), rec, tid);
            const float2 din2 = f2(din, din), dfr2 = f2(dfr, dfr);
            for (int st = 0; st < nst; ++st) {
                const int g = gs + st, b = g % kTcBufs;
                unsigned char *buf = bufs + b * C::kBufBytes;
                // the stage's buffer is free once the MMAs of stage g - kTcBufs have completed
                if (g >= kTcBufs) ok = mbar_wait_bounded(empty + b, (uint32_t)(g / kTcBufs - 1) & 1u, kTcWaitTries) && ok;
#pragma unroll
                for (int kg = 0; kg < 2; ++kg)
                    tc_produce_group<kDeg>(buf, cf, st * (kTcStage / 2) + kg * 4, kg, t, col_side, din2, dfr2);
                // the warp's writes, visible to the tensor core, then one arrival per warp
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(full + b);
            }
            gs += nst;
            if (last_seg) {
                // The item's MMAs have completed: the accumulators (warp w: rows 32 (w % 4) ..,
                // columns 64 (w / 4) ..) go through shared memory (the stage buffers, whose
                // last readers were those MMAs) and out as whole rows of the partial sums.
                const bool fin = mbar_wait_bounded(done, (uint32_t)n_done & 1u, kTcWaitTries);
                tc_fence_after();
                const bool item_ok = __all_sync(0xffffffffu, fin && ok);
                ok = ok && fin;
                const int quarter = warp & 3, half = warp >> 2;
                const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
                float *const srow = scr + (32 * quarter + lane) * kTcScratchStride;
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const int cb = 64 * half + 16 * c4;
                    uint32_t v1[16], v2[16];
                    tmem_ld_32x32b<16>(lane_base + (uint32_t)cb, v1);
                    tmem_ld_32x32b<16>(lane_base + (uint32_t)(kTcTile + cb), v2);
                    tmem_ld_wait();
                    float sv[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        sv[e] = item_ok ? __uint_as_float(v1[e]) + __uint_as_float(v2[e]) : __int_as_float(0x7FC00000);
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        reinterpret_cast<float4 *>(srow + cb)[e] = make_float4(sv[4 * e], sv[4 * e + 1], sv[4 * e + 2], sv[4 * e + 3]);
                }
                // the accumulators are read before the next item's first MMA overwrites them
                // (that MMA waits for every producer warp's arrival on the next stage)
                tc_fence_before();
                producers_sync();
                // warp w writes rows w, w + 8, ..: lane l the columns 4l .. 4l + 3
                const TcScan S = tc_scan(one, many, it);
                const int64_t W = S.W, H = S.H;
                const int64_t ncol = min((int64_t)kTcTile, W - c0);
                const bool vec = (W & 3) == 0 && 4 * lane + 4 <= ncol;
                for (int rr = warp; rr < kTcTile; rr += kGenWarps) {
                    const int64_t r = r0 + rr;
                    if (r >= H) break;
                    const float4 v = reinterpret_cast<const float4 *>(scr + rr * kTcScratchStride)[lane];
                    float *const dst = S.partial + (int64_t)it.row * S.pstride + r * W + c0 + 4 * lane;
                    if (vec) {
                        *reinterpret_cast<float4 *>(dst) = v;
                    } else {
                        if (4 * lane + 0 < ncol) dst[0] = v.x;
                        if (4 * lane + 1 < ncol) dst[1] = v.y;
                        if (4 * lane + 2 < ncol) dst[2] = v.z;
                        if (4 * lane + 3 < ncol) dst[3] = v.w;
                    }
                }
                ++n_done;
            }
            // advance to the next segment; the item record after the next is fetched early
            if (last_seg) {
                q += G;
                it = nxt;
                nxt = items[min(q + G, n_items - 1)];
            }
            s0 = ns0;
        }
    }
    if (!ok) atomicExch(&g_field_tc_timeout, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == kGenWarps) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" :: "r"(tmem) : "memory");
}

}  // namespace ddk
