// dd_surrogate.cu -- kernels of the learned surrogate of the field map (no counterpart
// in the paper): six 3x3 convolutions, NHWC BF16 activations, FP32 accumulation on the
// tensor cores (tcgen05.mma with TMEM accumulators for rows of 128 pixels, mma.sync
// m16n8k16 for other rows and the weight gradient), FP32 master weights with Adam.
//
// Layers: 16 -> 32 -> 32 -> 32 -> 32 -> 32 -> 16 channels (the first layer's input has 4
// real planes padded to 16, the last layer's output 1 real channel padded to 16), ReLU
// after the first five.  Weights are [Cout][tap = ky*3+kx][Cin] BF16; the data gradient
// uses the flipped, transposed copy [Cin][8 - tap][Cout] so that it is the same forward
// kernel.  Every convolution is an implicit GEMM: M = pixels, N = Cout, K = 9 Cin for
// the forward and data gradient; M = Cout, N = 9 Cin, K = pixels for the weight gradient
// (split over CTAs by image rows, partials reduced in a fixed order).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "dd_internal.h"
#include "dd_umma.cuh"

namespace ddk {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t addr, uint32_t &r0, uint32_t &r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];\n"
                 : "=r"(r0), "=r"(r1) : "r"(addr));
}
// D = A (16x16, row) * B (16x8, col) + D, BF16 inputs, FP32 accumulators.
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

enum { kEpiReluBf16 = 0, kEpiLinearF32 = 1, kEpiMaskBf16 = 2 };
constexpr int kTW = 64;   // pixels of one image row per CTA
constexpr int kMaxDil = 32;

// out = conv3x3(in, w) with the epilogue EPI:
//   kEpiReluBf16:  bf16(max(z + bias, 0))                   [B,H,W,CO]
//   kEpiLinearF32: float(z + bias), channel 0 only            [B,H,W]
//   kEpiMaskBf16:  bf16(z * (mask > 0)), mask [B,H,W,CO]      (data gradient through ReLU)
template <int CI, int CO, int EPI>
__global__ void __launch_bounds__(128)
conv3x3_kernel(const bf16 *__restrict__ in, const bf16 *__restrict__ w, const float *__restrict__ bias,
               const bf16 *__restrict__ mask, void *__restrict__ out, int H, int W, int dil) {
    constexpr int CIP = CI + 8;          // padded rows: ldmatrix rows land in distinct banks
    constexpr int KW = 9 * CI + 8;
    // dynamic shared memory: weights [CO][KW], then input rows [3][kTW + 2 dil][CIP]
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 (*s_w)[KW] = reinterpret_cast<bf16 (*)[KW]>(smem_raw);
    bf16 *s_in = reinterpret_cast<bf16 *>(smem_raw + sizeof(bf16) * CO * KW);
    const int cols = kTW + 2 * dil;
    auto IN = [&](int ky, int px) -> bf16 * { return s_in + ((size_t)ky * cols + px) * CIP; };
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_per_row = W / kTW;
    const int x0 = (blockIdx.x % tiles_per_row) * kTW;
    const int row = blockIdx.x / tiles_per_row;          // b * H + y
    const int y = row % H;
    const int64_t img0 = (int64_t)(row - y) * W;         // first pixel of image b

    for (int v = tid; v < CO * 9 * CI / 8; v += 128) {
        const int co = v / (9 * CI / 8), r = v - co * (9 * CI / 8);
        *reinterpret_cast<uint4 *>(&s_w[co][r * 8]) = *reinterpret_cast<const uint4 *>(w + (int64_t)co * 9 * CI + r * 8);
    }
    // tap (ky, kx) of output pixel x reads input (y + (ky-1) dil, x + (kx-1) dil); staged
    // column px holds input x0 - dil + px
    for (int v = tid; v < 3 * cols * (CI / 8); v += 128) {
        const int ky = v / (cols * (CI / 8));
        const int rem = v - ky * cols * (CI / 8);
        const int px = rem / (CI / 8), c8 = rem - px * (CI / 8);
        const int yy = y + (ky - 1) * dil, xx = x0 + px - dil;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (yy >= 0 && yy < H && xx >= 0 && xx < W)
            val = *reinterpret_cast<const uint4 *>(in + (img0 + (int64_t)yy * W + xx) * CI + c8 * 8);
        *reinterpret_cast<uint4 *>(IN(ky, px) + c8 * 8) = val;
    }
    __syncthreads();

    const int m0 = warp * 16;
    float acc[CO / 8][4];
#pragma unroll
    for (int n = 0; n < CO / 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
#pragma unroll
        for (int c0 = 0; c0 < CI; c0 += 16) {
            uint32_t a0, a1, a2, a3;
            ldsm_x4(smem_u32(IN(ky, m0 + (lane & 7) + 8 * ((lane >> 3) & 1) + kx * dil) + c0 + 8 * (lane >> 4)),
                    a0, a1, a2, a3);
#pragma unroll
            for (int n = 0; n < CO / 8; n += 2) {
                uint32_t b0, b1, b2, b3;
                ldsm_x4(smem_u32(&s_w[n * 8 + (lane & 7) + 8 * (lane >> 4)][tap * CI + c0 + 8 * ((lane >> 3) & 1)]),
                        b0, b1, b2, b3);
                mma_bf16(acc[n], a0, a1, a2, a3, b0, b1);
                mma_bf16(acc[n + 1], a0, a1, a2, a3, b2, b3);
            }
        }
    }
    const int g = lane >> 2, t2 = 2 * (lane & 3);
#pragma unroll
    for (int n = 0; n < CO / 8; ++n) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int64_t pix = img0 + (int64_t)y * W + x0 + m0 + g + 8 * half;
            const int ch = n * 8 + t2;
            float v0 = acc[n][2 * half], v1 = acc[n][2 * half + 1];
            if (EPI == kEpiReluBf16) {
                v0 = fmaxf(v0 + bias[ch], 0.f);
                v1 = fmaxf(v1 + bias[ch + 1], 0.f);
                *reinterpret_cast<__nv_bfloat162 *>(static_cast<bf16 *>(out) + pix * CO + ch) = __floats2bfloat162_rn(v0, v1);
            } else if (EPI == kEpiLinearF32) {
                if (ch == 0) static_cast<float *>(out)[pix] = v0 + bias[0];
            } else {
                const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162 *>(mask + pix * CO + ch);
                v0 = __bfloat162float(m.x) > 0.f ? v0 : 0.f;
                v1 = __bfloat162float(m.y) > 0.f ? v1 : 0.f;
                *reinterpret_cast<__nv_bfloat162 *>(static_cast<bf16 *>(out) + pix * CO + ch) = __floats2bfloat162_rn(v0, v1);
            }
        }
    }
}

// ---- the forward / data-gradient convolution on the 5th-generation tensor cores ------
//
// An output row tile is M = 128 pixels x N = Cout, computed with tcgen05.mma (kind::f16,
// BF16 operands, FP32 accumulator in tensor memory): 9 taps x Cin/16 MMAs of K = 16,
// issued by one thread; the accumulator is read back with tcgen05.ld (warp w reads TMEM
// lanes 32w..32w+31, i.e. its 32 pixels) for the epilogue.  Operands are staged in the
// canonical K-major layout without swizzle: "core matrices" of 8 rows x 16 bytes.
//   input row [c8][px][8]: pixel rows 16 bytes apart, so the 128 pixels of any tap
//          (shifted by kx*dil columns) form 16 core matrices 128 bytes apart (SBO), and
//          the next 8 channels sit one channel-group plane further (LBO = cols*16 bytes);
//   weight [tap][c8][co][8]: SBO 128 bytes (next 8 outputs), LBO Cout*16 bytes.
constexpr int kTW5 = 128;
static __device__ int g_tc_timeout;       // set when an MMA completion wait gives up

// 16-byte global -> shared copy that completes asynchronously; src_bytes 0 writes zeros.
__device__ __forceinline__ void cp_async16_zfill(void *smem, const void *gmem, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
                 : "memory");
}

// Persistent CTAs: each stages the weights once and allocates two TMEM accumulators once,
// then walks work items.  An item is a segment of kSeg output rows of one 128-pixel column
// strip, taken with stride dil (rows y0, y0 + dil, ...), so that consecutive rows share two
// of their three input rows: input rows live in a ring of four slots [C8][cols][8], and
// each output row copies in (cp.async) only the row its successor needs while its own
// MMAs run; the MMAs of the next row are issued once this row's epilogue has read the
// other accumulator.
constexpr int kSeg = 8;
template <int CI, int CO, int EPI>
__global__ void __launch_bounds__(128)
conv3x3_tc_kernel(const bf16 *__restrict__ in, const bf16 *__restrict__ w, const float *__restrict__ bias,
                  const bf16 *__restrict__ mask, void *__restrict__ out, int H, int W, int dil, int items_per_strip,
                  int n_items, int withhold_mma) {
    constexpr int C8 = CI / 8;
    static_assert(CI % 16 == 0 && (CO == 16 || CO == 32), "K steps of 16; 16 or 32 accumulator columns");
    // dynamic shared memory: weights [9][C8][CO][8], the ring of 4 input rows
    // [slot][C8][cols][8], two mbarriers, the TMEM address
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 *s_w = reinterpret_cast<bf16 *>(smem_raw);
    const int cols = kTW5 + 2 * dil;
    const int slot_elems = C8 * cols * 8;
    bf16 *s_ring = s_w + 9 * C8 * CO * 8;
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(s_ring + 4 * slot_elems);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(s_bar + 2);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_per_row = W / kTW5;

    // input row yy (zeros outside the image) of image img0, columns x0 - dil .., into slot
    auto stage_row = [&](int64_t img0, int x0, int yy, int slot) {
        bf16 *dst = s_ring + slot * slot_elems;
        const bool row_in = yy >= 0 && yy < H;
        for (int v = tid; v < cols * C8; v += 128) {
            const int c8 = v / cols, px = v - c8 * cols;
            const int xx = x0 + px - dil;
            const bool inside = row_in && xx >= 0 && xx < W;
            const bf16 *src = inside ? in + (img0 + (int64_t)yy * W + xx) * CI + c8 * 8 : in;
            cp_async16_zfill(dst + ((size_t)c8 * cols + px) * 8, src, inside ? 16 : 0);
        }
    };
    // the 9 x Cin/16 MMAs of chain row j (input rows j - 1, j, j + 1 in slots (j + 3) % 4,
    // j % 4, (j + 1) % 4) into accumulator b, committed to barrier b
    auto issue = [&](int j, int b, uint32_t tmem) {
        constexpr uint32_t idesc = umma_idesc_bf16(kTW5, CO);
        int accumulate = 0;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
            const bf16 *row = s_ring + ((j + 3 + ky) & 3) * slot_elems;
#pragma unroll
            for (int c0 = 0; c0 < CI; c0 += 16) {
                const uint32_t a = smem_u32(row + ((size_t)(c0 / 8) * cols + kx * dil) * 8);
                const uint32_t bb = smem_u32(s_w + ((size_t)(tap * C8 + c0 / 8) * CO) * 8);
                umma_bf16(tmem + 32u * b, umma_smem_desc(a, (uint32_t)cols * 16u, 128u),
                          umma_smem_desc(bb, CO * 16u, 128u), idesc, accumulate);
                accumulate = 1;
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(s_bar + b)) : "memory");
    };
    // item q: strip (image, column tile), then the segment within the strip: rows
    // rho + dil * (seg * kSeg + i), i < kSeg, for the residue rho of its chain
    auto decode = [&](int q, int64_t &img0, int &x0, int &rho, int &j0, int &j1) {
        const int strip = q / items_per_strip;
        int r = q - strip * items_per_strip;
        const int bimg = strip / tiles_per_row;
        x0 = (strip - bimg * tiles_per_row) * kTW5;
        img0 = (int64_t)bimg * H * W;
        for (rho = 0; rho < dil; ++rho) {
            const int J = (H - rho + dil - 1) / dil;             // chain rows rho, rho + dil, .. < H
            const int ns = (J + kSeg - 1) / kSeg;
            if (r < ns) { j0 = r * kSeg; j1 = min(J, j0 + kSeg); return; }
            r -= ns;
        }
        j0 = j1 = 0;                                             // not reached for q < n_items
    };

    for (int v = tid; v < CO * 9 * C8; v += 128) {
        const int co = v / (9 * C8), r = v - co * (9 * C8);      // r = tap * C8 + c8
        cp_async16_zfill(s_w + ((size_t)r * CO + co) * 8, w + (int64_t)co * 9 * CI + r * 8, 16);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" :: "r"(smem_u32(s_tmem)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(s_bar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(s_bar + 1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;

    int k = 0;                      // rows done by this CTA: accumulator k & 1, barrier use k >> 1
    bool ok = true;
    for (int q = blockIdx.x; q < n_items && ok; q += gridDim.x) {
        int64_t img0;
        int x0, rho, j0, j1;
        decode(q, img0, x0, rho, j0, j1);
        // the first row's three input rows (chain rows j0 - 1 .. j0 + 1), then its MMAs; every
        // earlier MMA of this CTA has completed (each row's wait precedes its epilogue)
        for (int i = j0 - 1; i <= j0 + 1; ++i) stage_row(img0, x0, rho + i * dil, (i + 4) & 3);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0 && !withhold_mma) issue(j0, k & 1, tmem);
        for (int j = j0; j < j1; ++j, ++k) {
            const int b = k & 1;
            // the input row the next output row adds (chain row j + 2, into the slot of j - 2)
            if (j + 1 < j1) stage_row(img0, x0, rho + (j + 2) * dil, (j + 2) & 3);
            asm volatile("cp.async.commit_group;" ::: "memory");
            // at most 2^18 tries of at most 1 us each (the suspend-time hint): a quarter second
            uint32_t done = 0;
            const uint32_t parity = (uint32_t)(k >> 1) & 1u;
            for (int it = 0; it < (1 << 18) && !done; ++it)
                asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000;\n"
                             " selp.u32 %0, 1, 0, p;\n}\n"
                             : "=r"(done) : "r"(smem_u32(s_bar + b)), "r"(parity) : "memory");
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (done) {
                const int y = rho + j * dil;
                uint32_t v[CO];
                tmem_ld_32x32b<CO>(tmem + 32u * b + ((uint32_t)(32 * warp) << 16), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const int64_t pix = img0 + (int64_t)y * W + x0 + 32 * warp + lane;
                if (EPI == kEpiLinearF32) {
                    static_cast<float *>(out)[pix] = __uint_as_float(v[0]) + bias[0];
                } else {
                    uint4 o[CO / 8];
                    uint4 mk[CO / 8];
                    if (EPI == kEpiMaskBf16) {
#pragma unroll
                        for (int qq = 0; qq < CO / 8; ++qq) mk[qq] = reinterpret_cast<const uint4 *>(mask + pix * CO)[qq];
                    }
#pragma unroll
                    for (int qq = 0; qq < CO / 8; ++qq) {
                        uint32_t packed[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int ch = 8 * qq + 2 * e;
                            float v0 = __uint_as_float(v[ch]), v1 = __uint_as_float(v[ch + 1]);
                            if (EPI == kEpiReluBf16) {
                                v0 = fmaxf(v0 + bias[ch], 0.f);
                                v1 = fmaxf(v1 + bias[ch + 1], 0.f);
                            } else {
                                const uint32_t mw = e == 0 ? mk[qq].x : e == 1 ? mk[qq].y : e == 2 ? mk[qq].z : mk[qq].w;
                                const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162 *>(&mw);
                                v0 = __bfloat162float(m2.x) > 0.f ? v0 : 0.f;
                                v1 = __bfloat162float(m2.y) > 0.f ? v1 : 0.f;
                            }
                            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
                            packed[e] = *reinterpret_cast<const uint32_t *>(&h2);
                        }
                        o[qq] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                    }
#pragma unroll
                    for (int qq = 0; qq < CO / 8; ++qq) reinterpret_cast<uint4 *>(static_cast<bf16 *>(out) + pix * CO)[qq] = o[qq];
                }
            }
            // the next row's input has landed and this row's accumulator has been read
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            const int all_done = __syncthreads_and((int)done);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!all_done) {                    // a wait gave up: report and stop this CTA
                if (tid == 0) atomicExch(&g_tc_timeout, 1);
                ok = false;
                break;
            }
            if (tid == 0 && j + 1 < j1 && !withhold_mma) issue(j + 1, (k + 1) & 1, tmem);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" :: "r"(tmem) : "memory");
}

// Weight gradient partials: CTA c sums rows [c*rows, (c+1)*rows) of the B*H image rows.
//   part[c][co*9*CI + tap*CI + ci] = sum_p dz[p][co] * x[p + offset(tap)][ci]
//   part[c][CO*9*CI + co]          = sum_p dz[p][co]
template <int CI, int CO>
__global__ void __launch_bounds__(128)
conv3x3_wgrad_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ dz, int H, int W, int rows_total,
                     int rows_per_cta, int dil, float *__restrict__ part) {
    constexpr int CIP = CI + 8, COP = CO + 8;
    constexpr int NT = 9 * CI / 8;                 // n-tiles of 8 (tap, ci) columns
    constexpr int MT = CO / 16;                    // m-tiles of 16 output channels
    constexpr int NTW = (NT + 3) / 4;              // n-tiles per warp (round robin)
    __shared__ __align__(16) bf16 s_x[3][kTW + 2 * kMaxDil][CIP];
    __shared__ __align__(16) bf16 s_dz[kTW][COP];
    __shared__ float s_db[CO];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float acc[MT][NTW][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int n = 0; n < NTW; ++n) acc[m][n][0] = acc[m][n][1] = acc[m][n][2] = acc[m][n][3] = 0.f;
    float db = 0.f;
    const int r_begin = blockIdx.x * rows_per_cta;
    const int r_end = min(rows_total, r_begin + rows_per_cta);
    for (int row = r_begin; row < r_end; ++row) {
        const int y = row % H;
        const int64_t img0 = (int64_t)(row - y) * W;
        for (int x0 = 0; x0 < W; x0 += kTW) {
            __syncthreads();
            const int cols = kTW + 2 * dil;
            for (int v = tid; v < 3 * cols * (CI / 8); v += 128) {
                const int ky = v / (cols * (CI / 8));
                const int rem = v - ky * cols * (CI / 8);
                const int px = rem / (CI / 8), c8 = rem - px * (CI / 8);
                const int yy = y + (ky - 1) * dil, xx = x0 + px - dil;
                uint4 val = make_uint4(0, 0, 0, 0);
                if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                    val = *reinterpret_cast<const uint4 *>(x + (img0 + (int64_t)yy * W + xx) * CI + c8 * 8);
                *reinterpret_cast<uint4 *>(&s_x[ky][px][c8 * 8]) = val;
            }
            for (int v = tid; v < kTW * CO / 8; v += 128) {
                const int px = v / (CO / 8), c8 = v - px * (CO / 8);
                *reinterpret_cast<uint4 *>(&s_dz[px][c8 * 8]) =
                    *reinterpret_cast<const uint4 *>(dz + (img0 + (int64_t)y * W + x0 + px) * CO + c8 * 8);
            }
            __syncthreads();
            if (tid < CO)
                for (int px = 0; px < kTW; ++px) db += __bfloat162float(s_dz[px][tid]);
#pragma unroll
            for (int p0 = 0; p0 < kTW; p0 += 16) {
                uint32_t a[MT][4];
#pragma unroll
                for (int m = 0; m < MT; ++m)
                    ldsm_x4_t(smem_u32(&s_dz[p0 + (lane & 7) + 8 * (lane >> 4)][m * 16 + 8 * ((lane >> 3) & 1)]),
                              a[m][0], a[m][1], a[m][2], a[m][3]);
#pragma unroll
                for (int j = 0; j < NTW; ++j) {
                    const int nt = warp + 4 * j;
                    if (nt < NT) {
                        const int tap = (nt * 8) / CI, ci0 = (nt * 8) % CI;
                        const int ky = tap / 3, kx = tap % 3;
                        uint32_t b0, b1;
                        ldsm_x2_t(smem_u32(&s_x[ky][p0 + (lane & 7) + 8 * ((lane >> 3) & 1) + kx * dil][ci0]), b0, b1);
#pragma unroll
                        for (int m = 0; m < MT; ++m) mma_bf16(acc[m][j], a[m][0], a[m][1], a[m][2], a[m][3], b0, b1);
                    }
                }
            }
        }
    }
    float *dst = part + (int64_t)blockIdx.x * (CO * 9 * CI + CO);
    const int g = lane >> 2, t2 = 2 * (lane & 3);
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int j = 0; j < NTW; ++j) {
            const int nt = warp + 4 * j;
            if (nt >= NT) continue;
            const int n = nt * 8 + t2;
            const int co = m * 16 + g;
            dst[co * 9 * CI + n] = acc[m][j][0];
            dst[co * 9 * CI + n + 1] = acc[m][j][1];
            dst[(co + 8) * 9 * CI + n] = acc[m][j][2];
            dst[(co + 8) * 9 * CI + n + 1] = acc[m][j][3];
        }
    if (tid < CO) s_db[tid] = db;
    __syncthreads();
    if (tid < CO) dst[CO * 9 * CI + tid] = s_db[tid];
}

__global__ void reduce_partials_kernel(const float *__restrict__ part, int n_parts, int len, float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    float s = 0.f;
    for (int c = 0; c < n_parts; ++c) s += part[(int64_t)c * len + i];
    out[i] = s;
}

// dz[p][0] = 2 w[p] (pred[p] - target[p]) / n, dz[p][1..15] = 0; per-block sums of
// w[p] (pred[p] - target[p])^2 (w = 1 when weight is NULL).
__global__ void mse_kernel(const float *__restrict__ pred, const float *__restrict__ target,
                           const float *__restrict__ weight, int64_t n, bf16 *__restrict__ dz,
                           double *__restrict__ block_sums) {
    __shared__ double s[256];
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (p < n) {
        const float d = pred[p] - target[p];
        const float wp = weight ? weight[p] : 1.0f;
        e = (double)wp * d * d;
        uint4 z = make_uint4(0, 0, 0, 0);
        __nv_bfloat162 g = __floats2bfloat162_rn(2.0f * wp * d / (float)n, 0.0f);
        z.x = *reinterpret_cast<uint32_t *>(&g);
        uint4 *o = reinterpret_cast<uint4 *>(dz + p * 16);
        o[0] = z;
        o[1] = make_uint4(0, 0, 0, 0);
    }
    s[threadIdx.x] = e;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = s[0];
}

__global__ void sum_doubles_kernel(const double *__restrict__ v, int n, double *__restrict__ out) {
    __shared__ double s[256];
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) a += v[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// Adam on FP32 master weights [co][tap][ci] (+ separate bias array handled the same way),
// writing the BF16 copy and the flipped copy [ci][8 - tap][co] used by the data gradient.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2,
                            bf16 *__restrict__ wb, bf16 *__restrict__ wflip, int ci_n, int co_n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (wb) {
        wb[i] = __float2bfloat16_rn(pi);
        const int ci = i % ci_n, tap = (i / ci_n) % 9, co = i / (9 * ci_n);
        wflip[((int64_t)ci * 9 + (8 - tap)) * co_n + co] = __float2bfloat16_rn(pi);
    }
}

// Input planes [B,H,W,16]: the time map value where visited (its encoding is the caller's), visited mask,
// standardised log D and log dwell; channels 4..15 zero.  tmap < 0 marks unvisited.
__global__ void planes_kernel(const float *__restrict__ tmap, const float *__restrict__ scal, int HW, int64_t n,
                              bf16 *__restrict__ x) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int b = (int)(p / HW);
    const float t = tmap[p];
    __nv_bfloat162 c01 = __floats2bfloat162_rn(t >= 0.f ? t : 0.f, t >= 0.f ? 1.f : 0.f);
    __nv_bfloat162 c23 = __floats2bfloat162_rn(scal[2 * b], scal[2 * b + 1]);
    uint4 z = make_uint4(0, 0, 0, 0);
    z.x = *reinterpret_cast<uint32_t *>(&c01);
    z.y = *reinterpret_cast<uint32_t *>(&c23);
    uint4 *o = reinterpret_cast<uint4 *>(x + p * 16);
    o[0] = z;
    o[1] = make_uint4(0, 0, 0, 0);
}

// The planes of planes_kernel, plus channel 4: each background visit's own term at its
// position (a visit older than k_exact dwells at the end of the scan: ln(w1/w0) of Eq. 3/4,
// w1 = 2 s + 4 kappa age, w0 = 2 s + 4 kappa (age - 1), as the normalised log10 of the
// target), and channel 5: the background mask.  scal3[b] = (standardised log D,
// standardised log dwell, kappa = D dwell / pitch^2).
__global__ void planes_bg_kernel(const float *__restrict__ tmap, const float *__restrict__ scal3, float s_dim,
                                 float k_exact, float mu, float inv_sigma, int HW, int64_t n, bf16 *__restrict__ x) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int b = (int)(p / HW);
    const float t = tmap[p];
    float own = 0.f, bg = 0.f;
    if (t > 0.f) {
        const float age = 1.0f / t;                      // 1 for the last visit
        if (age > k_exact + 0.5f) {
            const float kap = scal3[3 * b + 2];
            const float v = log1pf(4.0f * kap / (2.0f * s_dim + 4.0f * kap * (age - 1.0f)));
            own = (log10f(v) - mu) * inv_sigma;
            bg = 1.f;
        }
    }
    __nv_bfloat162 c01 = __floats2bfloat162_rn(t >= 0.f ? t : 0.f, t >= 0.f ? 1.f : 0.f);
    __nv_bfloat162 c23 = __floats2bfloat162_rn(scal3[3 * b], scal3[3 * b + 1]);
    __nv_bfloat162 c45 = __floats2bfloat162_rn(own, bg);
    uint4 z = make_uint4(0, 0, 0, 0);
    z.x = *reinterpret_cast<uint32_t *>(&c01);
    z.y = *reinterpret_cast<uint32_t *>(&c23);
    z.z = *reinterpret_cast<uint32_t *>(&c45);
    uint4 *o = reinterpret_cast<uint4 *>(x + p * 16);
    o[0] = z;
    o[1] = make_uint4(0, 0, 0, 0);
}

// One CTA per map: peak = max_p psi[m][p] * scale[m], then
// target[m][p] = (log10(max(psi[m][p] * scale[m], peak * 10^floor_rel)) - mu) * inv_sigma
__global__ void targets_kernel(const double *__restrict__ psi, const double *__restrict__ scale, int64_t hw,
                               double floor_rel, float mu, float inv_sigma, float *__restrict__ out) {
    __shared__ double s[256];
    const int64_t m = blockIdx.x;
    const double sc = scale[m];
    double mx = 0.0;
    for (int64_t p = threadIdx.x; p < hw; p += blockDim.x) mx = fmax(mx, psi[m * hw + p] * sc);
    s[threadIdx.x] = mx;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + k]);
        __syncthreads();
    }
    const double lo = fmax(s[0] * pow(10.0, floor_rel), 1e-300);
    for (int64_t p = threadIdx.x; p < hw; p += blockDim.x)
        out[m * hw + p] = (float)((log10(fmax(psi[m * hw + p] * sc, lo)) - (double)mu) * (double)inv_sigma);
}

// Per-pixel loss weights of one map per CTA, from its normalised log targets:
//   f_p = 10^(target_p sigma + mu),  w_p = alpha hw f_p^2 / sum_q f_q^2 + (1 - alpha).
// With alpha = 1 the weighted squared log error sum_p w_p (log10 error_p)^2 / hw is, to
// first order, (relative L2 error of the linear map / ln 10)^2: a pixel weighs as much as
// its share of the map's squared norm; 1 - alpha keeps every pixel in the loss.
__global__ void weights_kernel(const float *__restrict__ target, int64_t hw, float mu, float sigma, float alpha,
                               float *__restrict__ w) {
    __shared__ double s[256];
    const int64_t m = blockIdx.x;
    const float *t = target + m * hw;
    double acc = 0.0;
    for (int64_t p = threadIdx.x; p < hw; p += blockDim.x) {
        const double f = pow(10.0, (double)t[p] * sigma + mu);
        acc += f * f;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    const double norm = s[0] > 0.0 ? (double)alpha * (double)hw / s[0] : 0.0;
    for (int64_t p = threadIdx.x; p < hw; p += blockDim.x) {
        const double f = pow(10.0, (double)t[p] * sigma + mu);
        w[m * hw + p] = (float)(norm * f * f + (1.0 - (double)alpha));
    }
}

// psi[m][p] = 10^(pred[m][p] * sigma + mu) / scale[m]  (back to u/m^2)
__global__ void fields_kernel(const float *__restrict__ pred, const double *__restrict__ scale, int64_t hw,
                              int64_t n, float mu, float sigma, double *__restrict__ psi) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    psi[i] = pow(10.0, (double)pred[i] * sigma + mu) / scale[i / hw];
}

// err[m] = || psi_pred(spots) + add(spots) - exact ||_2 / || exact ||_2 over the k spot
// points of map m (add: an exactly computed part of the field, or NULL)
__global__ void spot_error_kernel(const float *__restrict__ pred, const int32_t *__restrict__ idx,
                                  const double *__restrict__ exact, const double *__restrict__ scale,
                                  const double *__restrict__ add, int hw, int k, float mu, float sigma,
                                  double *__restrict__ err) {
    const int m = blockIdx.x;
    __shared__ double sn[128], sd[128];
    double num = 0.0, den = 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const int p = idx[(int64_t)m * k + j];
        const double e = exact[(int64_t)m * k + j];
        const double v = pow(10.0, (double)pred[(int64_t)m * hw + p] * sigma + mu) / scale[m] +
                         (add ? add[(int64_t)m * hw + p] : 0.0);
        num += (v - e) * (v - e);
        den += e * e;
    }
    sn[threadIdx.x] = num;
    sd[threadIdx.x] = den;
    __syncthreads();
    for (int s = 64; s > 0; s >>= 1) {
        if (threadIdx.x < s) { sn[threadIdx.x] += sn[threadIdx.x + s]; sd[threadIdx.x] += sd[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) err[m] = sd[0] > 0.0 ? sqrt(sn[0] / sd[0]) : (sn[0] > 0.0 ? INFINITY : 0.0);
}

}  // namespace ddk

namespace {

template <int CI, int CO, int EPI>
cudaError_t launch_conv(const void *in, const void *w, const float *bias, const void *mask, void *out, int B,
                        int H, int W, int dil, cudaStream_t st) {
    constexpr int KW = 9 * CI + 8, CIP = CI + 8;
    const size_t smem = sizeof(ddk::bf16) * ((size_t)CO * KW + (size_t)3 * (ddk::kTW + 2 * dil) * CIP);
    static bool configured = false;     // allow the largest dilation's staging area once
    if (!configured) {
        const size_t most = sizeof(ddk::bf16) * ((size_t)CO * KW + (size_t)3 * (ddk::kTW + 2 * ddk::kMaxDil) * CIP);
        cudaError_t err = cudaFuncSetAttribute(ddk::conv3x3_kernel<CI, CO, EPI>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
        if (err != cudaSuccess) return err;
        configured = true;
    }
    const unsigned grid = (unsigned)(B * H * (W / ddk::kTW));
    ddk::conv3x3_kernel<CI, CO, EPI><<<grid, 128, smem, st>>>((const ddk::bf16 *)in, (const ddk::bf16 *)w, bias,
                                                               (const ddk::bf16 *)mask, out, H, W, dil);
    return cudaGetLastError();
}

// The tensor-memory variant (W a multiple of 128): persistent CTAs over segments of
// dilation-strided row chains.  Each CTA holds 64 TMEM columns; its shared-memory request is
// at least 30 KB, so that at most 7 CTAs share an SM (448 of its 512 columns: an
// allocation never waits).
template <int CI, int CO, int EPI>
cudaError_t launch_conv_tc(const void *in, const void *w, const float *bias, const void *mask, void *out, int B,
                           int H, int W, int dil, cudaStream_t st) {
    auto bytes = [](int d) {
        const size_t b = sizeof(ddk::bf16) * ((size_t)9 * CI * CO + (size_t)4 * CI * (ddk::kTW5 + 2 * d)) + 32;
        return std::max<size_t>(b, 30 * 1024);
    };
    static bool configured = false;     // allow the largest dilation's staging area once
    if (!configured) {
        cudaError_t err = cudaFuncSetAttribute(ddk::conv3x3_tc_kernel<CI, CO, EPI>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes(ddk::kMaxDil));
        // the whole L1/shared array as shared memory: without this preference the occupancy
        // query below counts a small shared-memory carveout and allows one CTA (4 warps) per
        // SM, leaving the tensor pipe idle behind each CTA's copy and MMA waits
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(ddk::conv3x3_tc_kernel<CI, CO, EPI>,
                                       cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
        if (err != cudaSuccess) return err;
        configured = true;
    }
    int dev = 0, sms = 0, smem_sm = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (err != cudaSuccess) return err;
    // CTAs that fit one SM's shared memory (each also costs the runtime's 1 KB reserve);
    // the occupancy query was seen to answer 1 here, which left 4 warps per SM
    const int per = (int)((size_t)smem_sm / (bytes(dil) + 1024));
    // items per (image, column tile): the segments of every residue chain rho < dil
    int per_strip = 0;
    for (int rho = 0; rho < dil; ++rho) {
        const int J = (H - rho + dil - 1) / dil;
        per_strip += (J + ddk::kSeg - 1) / ddk::kSeg;
    }
    const int n_items = B * (W / ddk::kTW5) * per_strip;
    const int grid = std::max(1, std::min(n_items, sms * std::min(per, 7)));
    // DD_FAULT=tc_wait (tests): no MMA is issued, so every completion wait runs out and the
    // timeout path (flag, no output, TMEM released) is exercised without a GPU fault
    const int withhold = dd::fault_injected("tc_wait") ? 1 : 0;
    ddk::conv3x3_tc_kernel<CI, CO, EPI><<<grid, 128, bytes(dil), st>>>((const ddk::bf16 *)in, (const ddk::bf16 *)w, bias,
                                                                        (const ddk::bf16 *)mask, out, H, W, dil,
                                                                        per_strip, n_items, withhold);
    return cudaGetLastError();
}

bool conv_shape_ok(int cin, int cout) {
    return (cin == 16 && cout == 32) || (cin == 32 && cout == 32) || (cin == 32 && cout == 16) ||
           (cin == 16 && cout == 16);
}

}  // namespace

extern "C" {

dd_status dd_sur_conv3x3(const void *in, const void *w, const float *bias, const void *mask, void *out,
                         int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t dilation,
                         int32_t epilogue, void *cuda_stream) {
    dd::clear_error();
    if (!in || !w || !out || B < 1 || H < 1 || W < ddk::kTW || W % ddk::kTW)
        return dd::fail(DD_EINVAL, "dd_sur_conv3x3: bad buffers or shape (W must be a multiple of 64)");
    if (!conv_shape_ok(cin, cout)) return dd::fail(DD_EINVAL, "dd_sur_conv3x3: unsupported (cin, cout)");
    if (dilation < 1 || dilation > ddk::kMaxDil) return dd::fail(DD_EINVAL, "dd_sur_conv3x3: dilation must be 1..32");
    if (epilogue < 0 || epilogue > 2 || (epilogue != 2 && !bias) || (epilogue == 2 && !mask))
        return dd::fail(DD_EINVAL, "dd_sur_conv3x3: bad epilogue arguments");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const char *name = epilogue == 2 ? "conv3x3_dgrad" : "conv3x3_fwd";
    dd::ProfScope ps(name, st);
    cudaError_t err = cudaSuccess;
    // rows of 128 pixels: tcgen05 MMA tiles of 128 pixels; otherwise 64-pixel tiles on mma.sync
    const bool tc = W % ddk::kTW5 == 0;
#define DD_CONV(CI, CO)                                                                                   \
    if (cin == CI && cout == CO) {                                                                        \
        if (tc) {                                                                                         \
            if (epilogue == 0) err = launch_conv_tc<CI, CO, ddk::kEpiReluBf16>(in, w, bias, mask, out, B, H, W, dilation, st);  \
            else if (epilogue == 1) err = launch_conv_tc<CI, CO, ddk::kEpiLinearF32>(in, w, bias, mask, out, B, H, W, dilation, st); \
            else err = launch_conv_tc<CI, CO, ddk::kEpiMaskBf16>(in, w, bias, mask, out, B, H, W, dilation, st);  \
        } else {                                                                                          \
            if (epilogue == 0) err = launch_conv<CI, CO, ddk::kEpiReluBf16>(in, w, bias, mask, out, B, H, W, dilation, st);  \
            else if (epilogue == 1) err = launch_conv<CI, CO, ddk::kEpiLinearF32>(in, w, bias, mask, out, B, H, W, dilation, st); \
            else err = launch_conv<CI, CO, ddk::kEpiMaskBf16>(in, w, bias, mask, out, B, H, W, dilation, st);  \
        }                                                                                                 \
    }
    DD_CONV(16, 32)
    DD_CONV(32, 32)
    DD_CONV(32, 16)
    DD_CONV(16, 16)
#undef DD_CONV
    if (err != cudaSuccess) return dd::fail_cuda(err, "dd_sur_conv3x3 launch");
    return DD_OK;
}

dd_status dd_sur_check(void) {
    dd::clear_error();
    DD_CUDA_TRY(cudaDeviceSynchronize());
    int flag = 0;
    DD_CUDA_TRY(cudaMemcpyFromSymbol(&flag, ddk::g_tc_timeout, sizeof(int)));
    if (!flag) return DD_OK;
    const int zero = 0;
    DD_CUDA_TRY(cudaMemcpyToSymbol(ddk::g_tc_timeout, &zero, sizeof(int)));
    return dd::fail(DD_ETIMEOUT, "dd_sur_check: a tensor-core convolution gave up waiting for its MMAs");
}

dd_status dd_sur_wgrad(const void *x, const void *dz, int32_t B, int32_t H, int32_t W, int32_t cin, int32_t cout,
                       int32_t dilation, float *part, int64_t part_floats, float *grad, void *cuda_stream) {
    dd::clear_error();
    if (!x || !dz || !part || !grad || B < 1 || H < 1 || W < ddk::kTW || W % ddk::kTW)
        return dd::fail(DD_EINVAL, "dd_sur_wgrad: bad buffers or shape");
    if (!conv_shape_ok(cin, cout) || cout % 16) return dd::fail(DD_EINVAL, "dd_sur_wgrad: unsupported (cin, cout)");
    if (dilation < 1 || dilation > ddk::kMaxDil) return dd::fail(DD_EINVAL, "dd_sur_wgrad: dilation must be 1..32");
    const int rows_total = B * H;
    const int len = cout * 9 * cin + cout;
    int n_cta = 4 * 152;
    if (n_cta > rows_total) n_cta = rows_total;
    const int rows_per = (rows_total + n_cta - 1) / n_cta;
    n_cta = (rows_total + rows_per - 1) / rows_per;
    if ((int64_t)n_cta * len > part_floats) return dd::fail(DD_EINVAL, "dd_sur_wgrad: partial buffer too small");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    dd::ProfScope ps("conv3x3_wgrad", st);
    const ddk::bf16 *xb = (const ddk::bf16 *)x, *db = (const ddk::bf16 *)dz;
    const int d = dilation;
    if (cin == 16 && cout == 32) ddk::conv3x3_wgrad_kernel<16, 32><<<n_cta, 128, 0, st>>>(xb, db, H, W, rows_total, rows_per, d, part);
    else if (cin == 32 && cout == 32) ddk::conv3x3_wgrad_kernel<32, 32><<<n_cta, 128, 0, st>>>(xb, db, H, W, rows_total, rows_per, d, part);
    else if (cin == 32 && cout == 16) ddk::conv3x3_wgrad_kernel<32, 16><<<n_cta, 128, 0, st>>>(xb, db, H, W, rows_total, rows_per, d, part);
    else ddk::conv3x3_wgrad_kernel<16, 16><<<n_cta, 128, 0, st>>>(xb, db, H, W, rows_total, rows_per, d, part);
    ddk::reduce_partials_kernel<<<(len + 255) / 256, 256, 0, st>>>(part, n_cta, len, grad);
    DD_CUDA_TRY(cudaGetLastError());
    return DD_OK;
}

dd_status dd_sur_mse(const float *pred, const float *target, int64_t n, void *dz, double *block_sums,
                     double *loss_sum, void *cuda_stream) {
    dd::clear_error();
    if (!pred || !target || !dz || !block_sums || !loss_sum || n < 1) return dd::fail(DD_EINVAL, "dd_sur_mse: bad arguments");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nb = (int)((n + 255) / 256);
    ddk::mse_kernel<<<nb, 256, 0, st>>>(pred, target, nullptr, n, (ddk::bf16 *)dz, block_sums);
    ddk::sum_doubles_kernel<<<1, 256, 0, st>>>(block_sums, nb, loss_sum);
    DD_CUDA_TRY(cudaGetLastError());
    return DD_OK;
}

dd_status dd_sur_wmse(const float *pred, const float *target, const float *weight, int64_t n, void *dz,
                      double *block_sums, double *loss_sum, void *cuda_stream) {
    dd::clear_error();
    if (!pred || !target || !weight || !dz || !block_sums || !loss_sum || n < 1)
        return dd::fail(DD_EINVAL, "dd_sur_wmse: bad arguments");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nb = (int)((n + 255) / 256);
    ddk::mse_kernel<<<nb, 256, 0, st>>>(pred, target, weight, n, (ddk::bf16 *)dz, block_sums);
    ddk::sum_doubles_kernel<<<1, 256, 0, st>>>(block_sums, nb, loss_sum);
    DD_CUDA_TRY(cudaGetLastError());
    return DD_OK;
}

dd_status dd_sur_weights(const float *target, int64_t n_maps, int64_t hw, float mu, float sigma, float alpha,
                         float *w, void *cuda_stream) {
    dd::clear_error();
    if (!target || !w || n_maps < 1 || hw < 1 || !(alpha >= 0.f && alpha <= 1.f))
        return dd::fail(DD_EINVAL, "dd_sur_weights: bad arguments");
    ddk::weights_kernel<<<(unsigned)n_maps, 256, 0, (cudaStream_t)cuda_stream>>>(target, hw, mu, sigma, alpha, w);
    DD_CUDA_TRY(cudaGetLastError());
    return DD_OK;
}

dd_status dd_sur_adam(float *param, const float *grad, float *m, float *v, int64_t n, float lr, float beta1,
                      float beta2, float eps, int32_t step, void *w_bf16, void *w_flip_bf16, int32_t cin,
                      int32_t cout, void *cuda_stream) {
    dd::clear_error();
    if (!param || !grad || !m || !v || n < 1 || step < 1) return dd::fail(DD_EINVAL, "dd_sur_adam: bad arguments");
    if (w_bf16 && (!w_flip_bf16 || (int64_t)cin * cout * 9 != n)) return dd::fail(DD_EINVAL, "dd_sur_adam: bad weight shape");
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    ddk::adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(param, grad, m, v, (int)n, lr, beta1, beta2, eps, c1, c2,
                                                                 (ddk::bf16 *)w_bf16, (ddk::bf16 *)w_flip_bf16, cin, cout);
    DD_CUDA_TRY(cudaGetLastError());
    return DD_OK;
}

dd_status dd_sur_planes(const float *tmap, const float *scal, int32_t B, int32_t H, int32_t W, void *x, void *cuda_stream) {
    dd::clear_error();
    if (!tmap || !scal || !x || B < 1 || H < 1 || W < 1) return dd::fail(DD_EINVAL, "dd_sur_planes: bad arguments");
    const int64_t n = (int64_t)B * H * W;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    ddk::planes_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tmap, scal, H * W, n, (ddk::bf16 *)x);
    DD_CUDA_TRY(cudaGetLastError());
    return DD_OK;
}

dd_status dd_sur_planes_bg(const float *tmap, const float *scal3, float s_dim, int32_t k_exact, float mu, float sigma,
                           int32_t B, int32_t H, int32_t W, void *x, void *cuda_stream) {
    dd::clear_error();
    if (!tmap || !scal3 || !x || B < 1 || H < 1 || W < 1 || !(s_dim > 0.f) || k_exact < 0 || !(sigma > 0.f))
        return dd::fail(DD_EINVAL, "dd_sur_planes_bg: bad arguments");
    const int64_t n = (int64_t)B * H * W;
    ddk::planes_bg_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(
        tmap, scal3, s_dim, (float)k_exact, mu, 1.0f / sigma, H * W, n, (ddk::bf16 *)x);
    DD_CUDA_TRY(cudaGetLastError());
    return DD_OK;
}

dd_status dd_sur_targets(const double *psi, const double *scale, int64_t n_maps, int64_t hw, double floor_rel_log10,
                         float mu, float sigma, float *out, void *cuda_stream) {
    dd::clear_error();
    if (!psi || !scale || !out || n_maps < 1 || hw < 1 || !(sigma > 0.f) || !(floor_rel_log10 < 0.0))
        return dd::fail(DD_EINVAL, "dd_sur_targets: bad arguments");
    ddk::targets_kernel<<<(unsigned)n_maps, 256, 0, (cudaStream_t)cuda_stream>>>(psi, scale, hw, floor_rel_log10, mu,
                                                                               1.0f / sigma, out);
    DD_CUDA_TRY(cudaGetLastError());
    return DD_OK;
}

dd_status dd_sur_fields(const float *pred, const double *scale, int64_t n_maps, int64_t hw, float mu, float sigma,
                        double *psi, void *cuda_stream) {
    dd::clear_error();
    if (!pred || !scale || !psi || n_maps < 1 || hw < 1) return dd::fail(DD_EINVAL, "dd_sur_fields: bad arguments");
    const int64_t n = n_maps * hw;
    ddk::fields_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(pred, scale, hw, n, mu,
                                                                                          sigma, psi);
    DD_CUDA_TRY(cudaGetLastError());
    return DD_OK;
}

dd_status dd_sur_spot_error(const float *pred, const int32_t *idx, const double *exact, const double *scale,
                            const double *add, int32_t n_maps, int32_t hw, int32_t k, float mu, float sigma,
                            double *err, void *cuda_stream) {
    dd::clear_error();
    if (!pred || !idx || !exact || !scale || !err || n_maps < 1 || hw < 1 || k < 1)
        return dd::fail(DD_EINVAL, "dd_sur_spot_error: bad arguments");
    ddk::spot_error_kernel<<<n_maps, 128, 0, (cudaStream_t)cuda_stream>>>(pred, idx, exact, scale, add, hw, k, mu,
                                                                          sigma, err);
    DD_CUDA_TRY(cudaGetLastError());
    return DD_OK;
}

}  // extern "C"
