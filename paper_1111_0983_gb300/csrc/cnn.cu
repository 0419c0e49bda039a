// Learned initial guess (no counterpart in the paper): six dilated 3x3
// convolutions, 4 -> 32 -> 32 -> 32 -> 32 -> 32 -> 2 channels, ReLU after the
// first five, BF16 operands with FP32 accumulation on the tcgen05 tensor cores.
//
// Layout.  Images are zero-padded by P (the largest dilation) on every side
// and flattened: pixel q = (b * Hp + i) * Wp + j, Hp = H + 2P, Wp = W + 2P.
// A tensor of C channels is stored channel-group-major, [C/8][npix][8] BF16,
// so each group is an array of 16-byte pixel rows.  That is exactly the
// layout of one column of 8x16-byte core matrices of a K-major (pixels x
// channels) operand, and a tap of the stencil -- a shift of the pixel index
// by di*d*Wp + dj*d -- is a shift of the operand's start address by a whole
// number of 16-byte rows: the implicit GEMM needs no im2col copy.
//
// Convolution (forward, and backward to the input): a CTA owns 128
// consecutive pixels (M = 128), N = output channels, K = input channels in
// slices of 16, summed over the 9 taps; the three input row segments it
// needs (di = -1, 0, 1, each 128 + 2d pixels) are staged in shared memory
// once, the weights too, and one thread issues the 9 * C_in / 16 MMAs into
// a TMEM accumulator.  The epilogue (bias, ReLU, BF16) runs from TMEM.
// Weight gradients: D_t[c_out][c_in] = sum_q dz[q][c_out] x[q + s_t][c_in]
// with the pixels as K, both operands MN-major, one accumulator per tap.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gcmg_cnn.h"

namespace {

constexpr int kLayers = 6;
constexpr int kCin[kLayers] = {4, 32, 32, 32, 32, 32};
constexpr int kCout[kLayers] = {32, 32, 32, 32, 32, 2};
constexpr int kTile = 128;            // pixels per CTA (M)
constexpr int kMaxDil = 96;
constexpr int kSeg = kTile + 2 * kMaxDil;   // staged pixels per row segment
constexpr long kWaitLimit = 1L << 24; // bounded mbarrier polls

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor, no swizzle: start, leading-dimension and
// stride-dimension byte offsets (all >> 4), descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: BF16 A and B, FP32 D, M x N, major-ness
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// polls the barrier's phase with a bound; false if it never completed
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    for (long it = 0; it < kWaitLimit; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int NCOLS>
__device__ __forceinline__ void tmem_alloc(uint32_t slot) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <int NCOLS>
__device__ __forceinline__ void tmem_free(uint32_t taddr) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(NCOLS) : "memory");
}

// 32 lanes x 16 / 32 consecutive FP32 columns of the accumulator
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
    return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

struct Geo {
    int npix, Hp, Wp, H, W, P;
    int gs;        // rows between channel groups (npix plus zero guard rows on both sides)
    __device__ __forceinline__ bool interior(int q, int *b, int *i, int *j) const {
        const int plane = Hp * Wp;
        *b = q / plane;
        const int rem = q - *b * plane;
        *i = rem / Wp;
        *j = rem - *i * Wp;
        return *i >= P && *i < P + H && *j >= P && *j < P + W;
    }
};

// stages the three row segments (di = -1, 0, 1) of G channel groups around
// pixels [q0, q0 + 128): smem[g][s][r] = x[g][q0 + (s-1) d Wp - d + r]
template <int G>
__device__ __forceinline__ void stage_halo(uint4 *sm, const uint4 *__restrict__ x, int npix, int gs, int q0, int Wp,
                                           int dil) {
    const int len = kTile + 2 * dil;
    for (int e = threadIdx.x; e < G * 3 * len; e += blockDim.x) {
        const int g = e / (3 * len);
        const int rem = e - g * 3 * len;
        const int s = rem / len, r = rem - s * len;
        const int q = q0 + (s - 1) * dil * Wp - dil + r;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (q >= 0 && q < npix) v = x[(size_t)g * gs + q];
        sm[(g * 3 + s) * kSeg + r] = v;
    }
}

// ------------------------------------------------------------ convolution
// MODE 0: y = bf16(relu(acc + bias)); 1: out[b][c][i][j] = acc + bias (c < 2);
// 2: y = bf16(acc * (gate > 0)) (backward to the input of the layer below)
struct ConvArgs {
    const uint4 *x;       // [GIN][npix] pixel rows
    const uint4 *w;       // [9][GIN][NOUT] rows of 8 input channels
    const float *bias;    // NOUT
    uint4 *y;             // [NOUT / 8][npix]
    float *out;           // MODE 1: [B][2][H][W]
    const uint4 *gate;    // MODE 2: [NOUT / 8][npix]
    Geo geo;
    int dil;
    int *err;
};

// bulk copy of `bytes` (a multiple of 16) from global to shared memory,
// completing as transaction bytes on `mbar`
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Persistent convolution: a CTA keeps the layer's weights in shared memory
// and walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...  The three
// input row segments of the next tile are brought in by bulk copies into the
// other half of a double buffer while the current tile's MMAs and epilogue
// run.  The activation buffers carry zero guard rows before and after each
// channel group, so every segment lies inside the allocation.
template <int GIN, int NOUT, int MODE>
__global__ void __launch_bounds__(128) k_conv(ConvArgs a, int ntiles) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int HALO = GIN * 3 * kSeg;                          // rows per buffer
    uint4 *sx = reinterpret_cast<uint4 *>(smem);                  // 2 buffers
    uint4 *sw = sx + 2 * HALO;                                    // 9 * GIN * NOUT rows
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sw + 9 * GIN * NOUT);   // full[2], mma
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 3);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int len = kTile + 2 * a.dil;
    const uint32_t seg_bytes = (uint32_t)len * 16;
    const uint32_t full0 = smem_u32(&mbar[0]), full1 = smem_u32(&mbar[1]), mma_bar = smem_u32(&mbar[2]);

    if (warp == 0) tmem_alloc<32>(smem_u32(tslot));
    if (threadIdx.x == 0) {
        mbar_init(full0);
        mbar_init(full1);
        mbar_init(mma_bar);
    }
    for (int e = threadIdx.x; e < 9 * GIN * NOUT; e += blockDim.x) sw[e] = a.w[e];
    fence_async_smem();
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot;

    // the producer: the segments of tile t into buffer b
    auto load_tile = [&](int t, int b) {
        const uint32_t fb = b ? full1 : full0;
        mbar_expect(fb, (uint32_t)(GIN * 3) * seg_bytes);
        const int q0 = t * kTile;
        for (int g = 0; g < GIN; g++)
            for (int sgm = 0; sgm < 3; sgm++) {
                const int q = q0 + (sgm - 1) * a.dil * a.geo.Wp - a.dil;
                bulk_g2s(smem_u32(sx + b * HALO + (g * 3 + sgm) * kSeg), a.x + (size_t)g * a.geo.gs + q, seg_bytes,
                         fb);
            }
    };
    if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) load_tile(blockIdx.x, 0);

    uint32_t ph_full[2] = {0, 0}, ph_mma = 0;
    bool ok = true;
    int k = 0;
#pragma unroll 1
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, k++) {
        const int b = k & 1;
        const bool w1 = mbar_wait(b ? full1 : full0, ph_full[b]);
        ph_full[b] ^= 1;
        ok = ok && w1;
        if (threadIdx.x == 0) {
            constexpr uint32_t idesc = idesc_bf16(kTile, NOUT, 0, 0);
            const uint32_t xa = smem_u32(sx + b * HALO), wa = smem_u32(sw);
            uint32_t acc = 0;
#pragma unroll 1
            for (int tap = 0; tap < 9; tap++) {
                const int sgm = tap / 3, dj = tap % 3 - 1;
                const int r0 = a.dil + dj * a.dil;
#pragma unroll
                for (int gp = 0; gp < GIN / 2; gp++) {
                    const uint64_t ad = sdesc(xa + ((2 * gp * 3 + sgm) * kSeg + r0) * 16, 3 * kSeg * 16, 128);
                    const uint64_t bd = sdesc(wa + ((tap * GIN + 2 * gp) * NOUT) * 16, NOUT * 16, 128);
                    mma_bf16(tmem, ad, bd, idesc, acc);
                    acc = 1;
                }
            }
            mma_commit(mma_bar);
            // the other buffer held the previous tile, whose MMAs completed
            // before its epilogue (below, in the previous iteration)
            if (t + (int)gridDim.x < ntiles) load_tile(t + gridDim.x, b ^ 1);
        }
        __syncwarp();
        const bool w2 = mbar_wait(mma_bar, ph_mma);
        ph_mma ^= 1;
        ok = ok && w2;
        tc_after();

        float v[NOUT];
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        tmem_ld16(lane_addr, v);
        if (NOUT == 32) tmem_ld16(lane_addr + 16, v + 16);

        const int q = t * kTile + warp * 32 + lane;
        int bb, i, j;
        if (q < a.geo.npix) {
            const bool in = a.geo.interior(q, &bb, &i, &j) && ok;
            if (MODE == 1) {
                if (in) {
                    const int H = a.geo.H, W = a.geo.W, P = a.geo.P;
                    for (int c = 0; c < 2; c++)
                        a.out[(((size_t)bb * 2 + c) * H + (i - P)) * W + (j - P)] = v[c] + a.bias[c];
                }
            } else {
#pragma unroll
                for (int g = 0; g < NOUT / 8; g++) {
                    float o[8];
                    if (MODE == 0) {
#pragma unroll
                        for (int e = 0; e < 8; e++) o[e] = in ? fmaxf(v[8 * g + e] + a.bias[8 * g + e], 0.0f) : 0.0f;
                    } else {
                        const uint4 gt = a.gate[(size_t)g * a.geo.gs + q];
                        const uint32_t gw[4] = {gt.x, gt.y, gt.z, gt.w};
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            o[2 * e] = (in && bf16_lo(gw[e]) > 0.0f) ? v[8 * g + 2 * e] : 0.0f;
                            o[2 * e + 1] = (in && bf16_hi(gw[e]) > 0.0f) ? v[8 * g + 2 * e + 1] : 0.0f;
                        }
                    }
                    a.y[(size_t)g * a.geo.gs + q] = make_uint4(pack_bf16(o[0], o[1]), pack_bf16(o[2], o[3]),
                                                               pack_bf16(o[4], o[5]), pack_bf16(o[6], o[7]));
                }
            }
        }
        // the accumulator is read before the next tile's MMAs overwrite it
        tc_before();
        __syncthreads();
        tc_after();
    }
    if (!ok && threadIdx.x == 0) atomicExch(a.err, 1);
    __syncthreads();
    if (warp == 0) {
        tc_after();
        tmem_free<32>(tmem);
    }
}

// --------------------------------------------------------- weight gradient
// D_t[co][ci] += sum over the CTA's pixel tiles of dz[q][co] x[q + s_t][ci];
// rows co >= 8 GA of the M = 128 operand read unrelated shared memory and
// are never stored.
struct DwArgs {
    const uint4 *dz;      // [GA][npix]
    const uint4 *x;       // [GB][npix]
    float *dw;            // [co][ci][9] of this layer (FP32, accumulated)
    int cout, cin;        // real channel counts
    Geo geo;
    int dil;
    int ntiles;
    int *err;
};

constexpr int kDwARows = 16 * kTile;   // 16 m-groups of a 128-pixel tile

template <int GA, int GB>
__global__ void __launch_bounds__(128, 1) k_conv_dw(DwArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint4 *sa = reinterpret_cast<uint4 *>(smem);                  // [16][kTile] rows (first GA filled)
    uint4 *sx = sa + kDwARows;                                    // [GB][3][kSeg]
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sx + GB * 3 * kSeg);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    constexpr int N = 8 * GB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) tmem_alloc<512>(smem_u32(tslot));
    if (threadIdx.x == 0) mbar_init(smem_u32(mbar));
    for (int e = threadIdx.x + GA * kTile; e < kDwARows; e += blockDim.x) sa[e] = make_uint4(0, 0, 0, 0);
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = idesc_bf16(kTile, N, 1, 1);
    uint32_t phase = 0;
    bool ok = true;
    int iter = 0;
#pragma unroll 1
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, iter++) {
        const int q0 = tile * kTile;
        if (iter > 0) {   // the previous tile's MMAs have read shared memory
            const bool w = mbar_wait(smem_u32(mbar), phase);
            ok = ok && w;
            phase ^= 1;
            tc_after();
        }
        for (int e = threadIdx.x; e < GA * kTile; e += blockDim.x) {
            const int g = e / kTile, r = e - g * kTile;
            const int q = q0 + r;
            sa[e] = q < a.geo.npix ? a.dz[(size_t)g * a.geo.gs + q] : make_uint4(0, 0, 0, 0);
        }
        stage_halo<GB>(sx, a.x, a.geo.npix, a.geo.gs, q0, a.geo.Wp, a.dil);
        fence_async_smem();
        tc_before();
        __syncthreads();
        tc_after();
        if (threadIdx.x == 0) {
            const uint32_t aa = smem_u32(sa), xa = smem_u32(sx);
#pragma unroll 1
            for (int kk = 0; kk < kTile / 16; kk++) {
                const uint64_t ad = sdesc(aa + kk * 16 * 16, 128, kTile * 16);
#pragma unroll 1
                for (int t = 0; t < 9; t++) {
                    const int s = t / 3, dj = t % 3 - 1;
                    const int r0 = a.dil + dj * a.dil + 16 * kk;
                    const uint64_t bd = sdesc(xa + (s * kSeg + r0) * 16, 128, 3 * kSeg * 16);
                    mma_bf16(tmem + (uint32_t)(t * N), ad, bd, idesc, (iter > 0 || kk > 0) ? 1u : 0u);
                }
            }
            mma_commit(smem_u32(mbar));
        }
        __syncwarp();
    }
    if (iter > 0) {
        const bool w = mbar_wait(smem_u32(mbar), phase);
        ok = ok && w;
        tc_after();
    }
    if (!ok && threadIdx.x == 0) atomicExch(a.err, 2);
    if (iter > 0 && ok && warp == 0) {
        for (int t = 0; t < 9; t++) {
            for (int c0 = 0; c0 < N; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + (uint32_t)(t * N + c0), v);
                const int co = lane;
                if (co < a.cout)
                    for (int k = 0; k < 16; k++)
                        if (c0 + k < a.cin) atomicAdd(&a.dw[((size_t)co * a.cin + c0 + k) * 9 + t], v[k]);
            }
        }
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        tmem_free<512>(tmem);
    }
}

// ---------------------------------------------------------- small kernels
// input [B][4][H][W] FP32 -> [2][npix] rows (channels 4..15 zero, border zero)
__global__ void k_pack_input(const float *__restrict__ in, uint4 *__restrict__ x, Geo geo) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= geo.npix) return;
    int b, i, j;
    float c[4] = {0, 0, 0, 0};
    if (geo.interior(q, &b, &i, &j)) {
        const size_t plane = (size_t)geo.H * geo.W;
        const size_t off = (size_t)(i - geo.P) * geo.W + (j - geo.P);
        for (int k = 0; k < 4; k++) c[k] = in[((size_t)b * 4 + k) * plane + off];
    }
    x[q] = make_uint4(pack_bf16(c[0], c[1]), pack_bf16(c[2], c[3]), 0, 0);
    x[(size_t)geo.gs + q] = make_uint4(0, 0, 0, 0);
}

// dL/dout [B][2][H][W] FP32 -> [2][npix] rows (channels 2..15 zero)
__global__ void k_pack_dout(const float *__restrict__ d, uint4 *__restrict__ x, Geo geo) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= geo.npix) return;
    int b, i, j;
    float c[2] = {0, 0};
    if (geo.interior(q, &b, &i, &j)) {
        const size_t plane = (size_t)geo.H * geo.W;
        const size_t off = (size_t)(i - geo.P) * geo.W + (j - geo.P);
        for (int k = 0; k < 2; k++) c[k] = d[((size_t)b * 2 + k) * plane + off];
    }
    x[q] = make_uint4(pack_bf16(c[0], c[1]), 0, 0, 0);
    x[(size_t)geo.gs + q] = make_uint4(0, 0, 0, 0);
}

// masked squared error of channel 0 ([B][2][plane] arrays): dout_0 = 2 (out_0 -
// t_0) m_0 / count, dout_1 = 0, loss += sum (out_0 - t_0)^2 m_0 / count
__global__ void k_mse(const float *__restrict__ out, const float *__restrict__ t, const float *__restrict__ m,
                      float *__restrict__ dout, size_t n, size_t plane, float inv_count, double *loss) {
    double s = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const bool ch0 = (e / plane) % 2 == 0;
        const float df = ch0 ? (out[e] - t[e]) * m[e] : 0.0f;
        dout[e] = 2.0f * df * inv_count;
        s += (double)df * df;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += part[w];
        atomicAdd(loss, tot * inv_count);
    }
}

// Residual term of the loss, two passes over [B][H][W]: e = (out_0 - t_0) m_0,
// s = e_N + e_S + e_E + e_W - 4 e where m_1 = 1 (inside the image edge), else
// 0; loss += beta sum s^2 / count; then dout_0 += 2 beta / count *
// (-4 s + s_N + s_S + s_E + s_W) m_0.
__global__ void k_lap_s(const float *__restrict__ out, const float *__restrict__ t, const float *__restrict__ m,
                        float *__restrict__ s, int B, int H, int W, float scale, double *loss) {
    const size_t plane = (size_t)H * W;
    double acc = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)B * plane;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t b = e / plane, p = e - b * plane;
        const int i = (int)(p / W), j = (int)(p - (size_t)i * W);
        const float *o0 = out + b * 2 * plane, *t0 = t + b * 2 * plane, *m0 = m + b * 2 * plane;
        float v = 0.0f;
        if (i > 0 && i < H - 1 && j > 0 && j < W - 1 && m0[plane + p] > 0.0f) {
            auto err = [&](size_t q) { return (o0[q] - t0[q]) * m0[q]; };
            v = err(p - W) + err(p + W) + err(p - 1) + err(p + 1) - 4.0f * err(p);
        }
        s[e] = v;
        acc += (double)v * v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += part[w];
        atomicAdd(loss, tot * scale);
    }
}

__global__ void k_lap_grad(const float *__restrict__ s, const float *__restrict__ m, float *__restrict__ dout, int B,
                           int H, int W, float scale2) {
    const size_t plane = (size_t)H * W;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)B * plane;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t b = e / plane, p = e - b * plane;
        const int i = (int)(p / W), j = (int)(p - (size_t)i * W);
        float g = -4.0f * s[e];
        if (i > 0) g += s[e - W];
        if (i < H - 1) g += s[e + W];
        if (j > 0) g += s[e - 1];
        if (j < W - 1) g += s[e + 1];
        dout[b * 2 * plane + p] += scale2 * g * m[b * 2 * plane + p];
    }
}

// db[c] += sum over pixels of the G-group gradient rows (BF16 values)
__global__ void k_bias_grad(const uint4 *__restrict__ dz, int G, int cout, int npix, int gs, float *db) {
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int g = blockIdx.y;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < npix; q += gridDim.x * blockDim.x) {
        const uint4 v = dz[(size_t)g * gs + q];
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        for (int k = 0; k < 4; k++) {
            acc[2 * k] += bf16_lo(w[k]);
            acc[2 * k + 1] += bf16_hi(w[k]);
        }
    }
    for (int k = 0; k < 8; k++) {
        float s = acc[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0 && 8 * g + k < cout) atomicAdd(&db[8 * g + k], s);
    }
}

// BF16 operand copies of one layer's FP32 weights w[co][ci][9]:
// forward rows  wf[t][g][co][8] = w[co][8g + k][t]            (GIN groups, NOUT rows)
// backward rows wb[t][g][ci][8] = w[8g + k][ci][8 - t]         (GOUT groups, 32 rows)
__global__ void k_prep_weights(const float *__restrict__ w, int cout, int cin, int gin, int nout, int gout,
                               uint16_t *__restrict__ wf, uint16_t *__restrict__ wb) {
    const int nf = 9 * gin * nout * 8, nb = wb ? 9 * gout * 32 * 8 : 0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nf + nb; e += gridDim.x * blockDim.x) {
        float val = 0.0f;
        if (e < nf) {
            const int k = e % 8, co = (e / 8) % nout, g = (e / (8 * nout)) % gin, t = e / (8 * nout * gin);
            const int ci = 8 * g + k;
            if (co < cout && ci < cin) val = w[((size_t)co * cin + ci) * 9 + t];
            wf[e] = __bfloat16_as_ushort(__float2bfloat16_rn(val));
        } else {
            const int f = e - nf;
            const int k = f % 8, ci = (f / 8) % 32, g = (f / 256) % gout, t = f / (256 * gout);
            const int co = 8 * g + k;
            if (co < cout && ci < cin) val = w[((size_t)co * cin + ci) * 9 + (8 - t)];
            wb[f] = __bfloat16_as_ushort(__float2bfloat16_rn(val));
        }
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.0f - b1) * gi;
    const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

// ------------------------------------------------------------------ context
struct gcmg_cnn {
    int batch = 0, H = 0, W = 0, P = 0;
    int dil[kLayers] = {1, 3, 9, 27, 81, 1};
    Geo geo{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int64_t nparams = 0;
    int64_t woff[kLayers] = {}, boff[kLayers] = {};
    float *p = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;   // FP32 master, gradient, Adam moments
    uint16_t *wf[kLayers] = {}, *wb[kLayers] = {};
    uint4 *act[kLayers] = {};    // act[0] = packed input, act[l] = output of layer l (l = 1..5)
    uint4 *dz[2] = {};           // ping-pong gradients
    float *out = nullptr, *dout = nullptr, *lap_s = nullptr;
    double *d_loss = nullptr;
    int *d_err = nullptr;
    int adam_t = 0;
    int sms = 148;
    size_t guard = 0;            // zero rows before and after each channel group
    size_t smem_conv4 = 0, smem_conv2 = 0, smem_dw = 0;
    std::string err;
    std::vector<void *> allocs;
};

namespace {

struct Fail {
    gcmg_status s;
    std::string m;
};

void ck(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Fail{GCMG_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
    }
}

template <typename T>
T *alloc(gcmg_cnn *c, size_t n) {
    void *p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        throw Fail{GCMG_E_OOM, "device allocation failed"};
    }
    c->allocs.push_back(p);
    return static_cast<T *>(p);
}

int groups_in(int l) { return l == 0 ? 2 : 4; }
int nout_of(int l) { return l == kLayers - 1 ? 16 : 32; }

size_t conv_smem(int gin, int nout, size_t slack) {
    const size_t need = (size_t)(2 * gin * 3 * kSeg + 9 * gin * nout) * 16 + 32;
    return std::max(need, slack);
}

#define CNN_GUARD(c, ...)                                             \
    try {                                                             \
        __VA_ARGS__                                                   \
    } catch (const Fail &f) {                                         \
        if (c) (c)->err = f.m;                                        \
        return f.s;                                                   \
    }

void check_err(gcmg_cnn *c) {
    int e = 0;
    ck(cudaMemcpyAsync(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "err");
    ck(cudaStreamSynchronize(c->stream), "sync");
    if (e) throw Fail{GCMG_E_TIMEOUT, "a tensor-core wait ran out (code " + std::to_string(e) + ")"};
}

void prep_weights(gcmg_cnn *c) {
    for (int l = 0; l < kLayers; l++) {
        const int gout = l == kLayers - 1 ? 2 : 4;
        k_prep_weights<<<64, 256, 0, c->stream>>>(c->p + c->woff[l], kCout[l], kCin[l], groups_in(l), nout_of(l),
                                                  gout, c->wf[l], c->wb[l]);
    }
    ck(cudaGetLastError(), "prep weights");
}

template <int GIN, int NOUT, int MODE>
void launch_conv(gcmg_cnn *c, const ConvArgs &a, size_t smem) {
    const int ntiles = (c->geo.npix + kTile - 1) / kTile;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv<GIN, NOUT, MODE>, 128, smem);
    const unsigned grid = (unsigned)std::min(ntiles, std::max(per_sm, 1) * c->sms);
    k_conv<GIN, NOUT, MODE><<<grid, 128, smem, c->stream>>>(a, ntiles);
    ck(cudaGetLastError(), "conv launch");
}

void forward(gcmg_cnn *c, const float *in, float *out) {
    const Geo g = c->geo;
    k_pack_input<<<(g.npix + 255) / 256, 256, 0, c->stream>>>(in, c->act[0], g);
    for (int l = 0; l < kLayers; l++) {
        ConvArgs a{};
        a.x = c->act[l];
        a.w = reinterpret_cast<const uint4 *>(c->wf[l]);
        a.bias = c->p + c->boff[l];
        a.geo = g;
        a.dil = c->dil[l];
        a.err = c->d_err;
        if (l == 0) {
            a.y = c->act[1];
            launch_conv<2, 32, 0>(c, a, c->smem_conv2);
        } else if (l < kLayers - 1) {
            a.y = c->act[l + 1];
            launch_conv<4, 32, 0>(c, a, c->smem_conv4);
        } else {
            a.out = out;
            launch_conv<4, 16, 1>(c, a, c->smem_conv4);
        }
    }
}

// parameter gradients into c->grad for dL/dout = dout (c->dout layout [B][2][H][W])
void backward(gcmg_cnn *c, const float *dout) {
    const Geo g = c->geo;
    ck(cudaMemsetAsync(c->grad, 0, c->nparams * sizeof(float), c->stream), "memset");
    k_pack_dout<<<(g.npix + 255) / 256, 256, 0, c->stream>>>(dout, c->dz[0], g);
    int cur = 0;
    const int ntiles = (g.npix + kTile - 1) / kTile;
    const int sms = c->sms;
    for (int l = kLayers - 1; l >= 0; l--) {
        const int ga = l == kLayers - 1 ? 2 : 4;
        DwArgs d{};
        d.dz = c->dz[cur];
        d.x = c->act[l];
        d.dw = c->grad + c->woff[l];
        d.cout = kCout[l];
        d.cin = kCin[l];
        d.geo = g;
        d.dil = c->dil[l];
        d.ntiles = ntiles;
        d.err = c->d_err;
        const unsigned grid = (unsigned)std::min(ntiles, sms);
        if (ga == 2) k_conv_dw<2, 4><<<grid, 128, c->smem_dw, c->stream>>>(d);
        else if (l == 0) k_conv_dw<4, 2><<<grid, 128, c->smem_dw, c->stream>>>(d);
        else k_conv_dw<4, 4><<<grid, 128, c->smem_dw, c->stream>>>(d);
        ck(cudaGetLastError(), "dw launch");
        k_bias_grad<<<dim3(64, ga), 256, 0, c->stream>>>(c->dz[cur], ga, kCout[l], g.npix, g.gs,
                                                         c->grad + c->boff[l]);
        if (l == 0) break;
        ConvArgs a{};
        a.x = c->dz[cur];
        a.w = reinterpret_cast<const uint4 *>(c->wb[l]);
        a.y = c->dz[cur ^ 1];
        a.gate = c->act[l];
        a.geo = g;
        a.dil = c->dil[l];
        a.err = c->d_err;
        if (ga == 2) launch_conv<2, 32, 2>(c, a, c->smem_conv2);
        else launch_conv<4, 32, 2>(c, a, c->smem_conv4);
        cur ^= 1;
    }
}

}  // namespace

extern "C" {

int64_t gcmg_cnn_num_params(void) {
    int64_t n = 0;
    for (int l = 0; l < kLayers; l++) n += (int64_t)kCout[l] * kCin[l] * 9 + kCout[l];
    return n;
}

gcmg_status gcmg_cnn_create(int batch, int H, int W, const int *dilations, void *stream, gcmg_cnn **out) {
    if (!out) return GCMG_E_ARG;
    *out = nullptr;
    if (batch < 1 || H < 1 || W < 1) return GCMG_E_ARG;
    gcmg_cnn *c = new (std::nothrow) gcmg_cnn;
    if (!c) return GCMG_E_OOM;
    *out = c;
    if (dilations)
        for (int l = 0; l < kLayers; l++) {
            if (dilations[l] < 1 || dilations[l] > kMaxDil) {
                c->err = "dilations must lie in [1, 96]";
                return GCMG_E_ARG;
            }
            c->dil[l] = dilations[l];
        }
    int P = 0;
    for (int l = 0; l < kLayers; l++) P = std::max(P, c->dil[l]);
    const double npix = (double)batch * (H + 2 * P) * (W + 2 * P);
    if (npix >= 2.0e9) {
        c->err = "too many pixels";
        return GCMG_E_ARG;
    }
    c->batch = batch;
    c->H = H;
    c->W = W;
    c->P = P;
    // guard rows: the furthest tap of the last pixel of a tile, on either side
    c->guard = (size_t)P * (W + 2 * P) + P + kTile;
    c->geo = Geo{(int)npix, H + 2 * P, W + 2 * P, H, W, P, (int)((size_t)npix + 2 * c->guard)};
    c->stream = (cudaStream_t)stream;
    CNN_GUARD(c, {
        ck(cudaGetDevice(&c->device), "cudaGetDevice");
        int64_t off = 0;
        for (int l = 0; l < kLayers; l++) {
            c->woff[l] = off;
            off += (int64_t)kCout[l] * kCin[l] * 9;
            c->boff[l] = off;
            off += kCout[l];
        }
        c->nparams = off;
        c->p = alloc<float>(c, off);
        c->grad = alloc<float>(c, off);
        c->m = alloc<float>(c, off);
        c->v = alloc<float>(c, off);
        ck(cudaMemset(c->p, 0, off * sizeof(float)), "memset");
        ck(cudaMemset(c->m, 0, off * sizeof(float)), "memset");
        ck(cudaMemset(c->v, 0, off * sizeof(float)), "memset");
        for (int l = 0; l < kLayers; l++) {
            c->wf[l] = alloc<uint16_t>(c, (size_t)9 * groups_in(l) * nout_of(l) * 8);
            if (l > 0) c->wb[l] = alloc<uint16_t>(c, (size_t)9 * (l == kLayers - 1 ? 2 : 4) * 32 * 8);
        }
        ck(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device), "attr");
        const size_t gs = (size_t)c->geo.gs;
        // each buffer: G groups of gs rows; the pointer skips the first guard
        c->act[0] = alloc<uint4>(c, 2 * gs) + c->guard;
        for (int l = 1; l < kLayers; l++) c->act[l] = alloc<uint4>(c, 4 * gs) + c->guard;
        c->dz[0] = alloc<uint4>(c, 4 * gs) + c->guard;
        c->dz[1] = alloc<uint4>(c, 4 * gs) + c->guard;
        c->out = alloc<float>(c, (size_t)batch * 2 * H * W);
        c->dout = alloc<float>(c, (size_t)batch * 2 * H * W);
        c->lap_s = alloc<float>(c, (size_t)batch * H * W);
        c->d_loss = alloc<double>(c, 1);
        c->d_err = alloc<int>(c, 1);
        ck(cudaMemset(c->d_err, 0, sizeof(int)), "memset");
        // shared memory: the weight-gradient kernel holds 512 TMEM columns, so
        // it asks for enough shared memory to sit alone on an SM
        c->smem_conv4 = conv_smem(4, 32, 0);
        c->smem_conv2 = conv_smem(2, 32, 0);
        c->smem_dw = std::max((size_t)(kDwARows + 4 * 3 * kSeg) * 16 + 16, (size_t)140 * 1024);
        ck(cudaFuncSetAttribute(k_conv<2, 32, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_conv2), "attr");
        ck(cudaFuncSetAttribute(k_conv<4, 32, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_conv4), "attr");
        ck(cudaFuncSetAttribute(k_conv<4, 16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_conv4), "attr");
        ck(cudaFuncSetAttribute(k_conv<2, 32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_conv2), "attr");
        ck(cudaFuncSetAttribute(k_conv<4, 32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_conv4), "attr");
        ck(cudaFuncSetAttribute(k_conv_dw<2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_dw), "attr");
        ck(cudaFuncSetAttribute(k_conv_dw<4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_dw), "attr");
        ck(cudaFuncSetAttribute(k_conv_dw<4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_dw), "attr");
        // zero every activation once: borders and guards stay zero from then on
        for (int l = 0; l < kLayers; l++) ck(cudaMemset(c->act[l] - c->guard, 0, (l ? 4 : 2) * gs * 16), "memset");
        ck(cudaMemset(c->dz[0] - c->guard, 0, 4 * gs * 16), "memset");
        ck(cudaMemset(c->dz[1] - c->guard, 0, 4 * gs * 16), "memset");
        return GCMG_OK;
    })
}

void gcmg_cnn_destroy(gcmg_cnn *c) {
    if (!c) return;
    for (void *p : c->allocs) cudaFree(p);
    delete c;
}

const char *gcmg_cnn_last_error(const gcmg_cnn *c) { return c ? c->err.c_str() : "null network"; }

gcmg_status gcmg_cnn_set_params(gcmg_cnn *c, const float *p_host, int64_t count) {
    if (!c || !p_host || count != c->nparams) return GCMG_E_ARG;
    CNN_GUARD(c, {
        ck(cudaMemcpyAsync(c->p, p_host, count * sizeof(float), cudaMemcpyHostToDevice, c->stream), "params");
        ck(cudaMemsetAsync(c->m, 0, count * sizeof(float), c->stream), "memset");
        ck(cudaMemsetAsync(c->v, 0, count * sizeof(float), c->stream), "memset");
        c->adam_t = 0;
        prep_weights(c);
        ck(cudaStreamSynchronize(c->stream), "sync");
        return GCMG_OK;
    })
}

gcmg_status gcmg_cnn_get_params(gcmg_cnn *c, float *p_host, int64_t count) {
    if (!c || !p_host || count != c->nparams) return GCMG_E_ARG;
    CNN_GUARD(c, {
        ck(cudaMemcpyAsync(p_host, c->p, count * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "params");
        ck(cudaStreamSynchronize(c->stream), "sync");
        return GCMG_OK;
    })
}

gcmg_status gcmg_cnn_forward(gcmg_cnn *c, const float *in_dev, float *out_dev) {
    if (!c || !in_dev || !out_dev) return GCMG_E_ARG;
    CNN_GUARD(c, {
        forward(c, in_dev, out_dev);
        check_err(c);
        return GCMG_OK;
    })
}

gcmg_status gcmg_cnn_activation(gcmg_cnn *c, int layer, float *dst_dev) {
    if (!c || !dst_dev || layer < 0 || layer >= kLayers) return GCMG_E_ARG;
    CNN_GUARD(c, {
        // unpack [G][npix][8] BF16 -> [B][C][H][W] FP32 on the host side of the stream
        const int G = layer == 0 ? 2 : 4, C = layer == 0 ? 4 : 32;
        const size_t np = (size_t)c->geo.npix;
        std::vector<uint16_t> h((size_t)G * np * 8);
        for (int g = 0; g < G; g++)
            ck(cudaMemcpyAsync(h.data() + (size_t)g * np * 8, c->act[layer] + (size_t)g * c->geo.gs, np * 16,
                               cudaMemcpyDeviceToHost, c->stream),
               "act");
        ck(cudaStreamSynchronize(c->stream), "sync");
        std::vector<float> o((size_t)c->batch * C * c->H * c->W);
        for (int b = 0; b < c->batch; b++)
            for (int ch = 0; ch < C; ch++)
                for (int i = 0; i < c->H; i++)
                    for (int j = 0; j < c->W; j++) {
                        const size_t q = ((size_t)b * c->geo.Hp + i + c->P) * c->geo.Wp + j + c->P;
                        const uint32_t bits = (uint32_t)h[((size_t)(ch / 8) * np + q) * 8 + ch % 8] << 16;
                        float f;
                        std::memcpy(&f, &bits, 4);
                        o[(((size_t)b * C + ch) * c->H + i) * c->W + j] = f;
                    }
        ck(cudaMemcpyAsync(dst_dev, o.data(), o.size() * 4, cudaMemcpyHostToDevice, c->stream), "act");
        ck(cudaStreamSynchronize(c->stream), "sync");
        return GCMG_OK;
    })
}

gcmg_status gcmg_cnn_backward(gcmg_cnn *c, const float *dout_dev, float *grad_dev) {
    if (!c || !dout_dev || !grad_dev) return GCMG_E_ARG;
    CNN_GUARD(c, {
        backward(c, dout_dev);
        ck(cudaMemcpyAsync(grad_dev, c->grad, c->nparams * sizeof(float), cudaMemcpyDeviceToDevice, c->stream),
           "grad");
        check_err(c);
        return GCMG_OK;
    })
}

gcmg_status gcmg_cnn_train_step(gcmg_cnn *c, const float *in_dev, const float *target_dev, const float *mask_dev,
                                float mask_count, float lap_weight, float lap_count, float lr, double *loss_host) {
    if (!c || !in_dev || !target_dev || !mask_dev || !(mask_count > 0.0f) || lap_weight < 0.0f ||
        (lap_weight > 0.0f && !(lap_count > 0.0f)))
        return GCMG_E_ARG;
    CNN_GUARD(c, {
        forward(c, in_dev, c->out);
        ck(cudaMemsetAsync(c->d_loss, 0, sizeof(double), c->stream), "memset");
        const size_t n = (size_t)c->batch * 2 * c->H * c->W;
        k_mse<<<256, 256, 0, c->stream>>>(c->out, target_dev, mask_dev, c->dout, n, (size_t)c->H * c->W,
                                          1.0f / mask_count, c->d_loss);
        if (lap_weight > 0.0f) {
            k_lap_s<<<256, 256, 0, c->stream>>>(c->out, target_dev, mask_dev, c->lap_s, c->batch, c->H, c->W,
                                                lap_weight / lap_count, c->d_loss);
            k_lap_grad<<<256, 256, 0, c->stream>>>(c->lap_s, mask_dev, c->dout, c->batch, c->H, c->W,
                                                   2.0f * lap_weight / lap_count);
        }
        backward(c, c->dout);
        c->adam_t++;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.0f - std::pow(b1, (float)c->adam_t), c2 = 1.0f - std::pow(b2, (float)c->adam_t);
        k_adam<<<(unsigned)((c->nparams + 255) / 256), 256, 0, c->stream>>>(c->p, c->grad, c->m, c->v,
                                                                           (int)c->nparams, lr, b1, b2, 1e-8f, c1, c2);
        prep_weights(c);
        double loss = 0.0;
        ck(cudaMemcpyAsync(&loss, c->d_loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "loss");
        check_err(c);
        if (loss_host) *loss_host = loss;
        return GCMG_OK;
    })
}

}  // extern "C"
