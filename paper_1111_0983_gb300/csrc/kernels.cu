// Device kernels of one multigrid level, templated on the precision T and
// the dimension D.  Grids are dense C-ordered n^D arrays (last axis
// contiguous); ghost records are slot-major so that consecutive threads read
// consecutive words.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "gcmg_internal.h"
#include "kernels.h"
#include "kernels_dev.cuh"

namespace gcmg {

std::atomic<long long> g_launches{0};

namespace {

using namespace dev;
constexpr int kThreads = 256;
// lists of at least this many entries (the finest band) take four entries a
// thread in the band and junction-zone sweeps, smaller ones one (measured at
// 513^3: four a thread on every list made a cycle 12 % slower)
constexpr int kListBig = 300000;
constexpr unsigned kNormBlocks = 2048;   // grid cap of the kernels that reduce a max-norm

// Launches with programmatic stream serialization: the kernel may be set up
// while its predecessor in the stream finishes; every kernel of this file
// starts with pdl_wait (griddepcontrol.wait), which returns once the
// predecessor has completed and its writes are visible.
template <typename... P, typename... A>
void pdl_launch(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}



// threads of a launch over a level's nodes (level_node): its active chunks
// where it has them and `chunked` allows, else the whole box
template <typename T>
inline int64_t level_threads(const LevelView<T> &v, bool chunked) {
    return chunked && v.chunks ? v.nchunks * CHUNK : v.nn;
}

inline unsigned blocks_for(int64_t total, int threads = kThreads) {
    int64_t b = (total + threads - 1) / threads;
    return (unsigned)(b > 0 ? b : 1);
}

template <int D>
__device__ __forceinline__ bool decode_colour(int n, int color, int64_t t, int64_t s0, int64_t s1, int64_t &p) {
    // thread t -> node of the given colour (sum of indices even = 0 / odd = 1)
    const int hc = (n + 1) >> 1;
    int i0, i1 = 0, jj;
    if (D == 2) {
        i0 = (int)dev::idx_div(t, hc);
        jj = (int)(t - (int64_t)i0 * hc);
    } else {
        const int64_t rest = dev::idx_div(t, hc);
        jj = (int)(t - rest * hc);
        i0 = (int)dev::idx_div(rest, n);
        i1 = (int)(rest - (int64_t)i0 * n);
    }
    if (i0 >= n) return false;
    const int last = 2 * jj + ((i0 + i1 + color) & 1);
    if (last >= n) return false;
    p = (int64_t)i0 * s0 + (D == 3 ? (int64_t)i1 * s1 : 0) + last;
    return true;
}

// ---------------------------------------------------------------- smoothers
// Gauss-Seidel form of Eq. (jac2d) on the inside nodes of one colour.
template <typename T, int D>
__global__ void k_rb_interior(LevelView<T> v, int color) {
    pdl_wait();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t p;
    if (D == 3 && v.chunks) {
        // over the active chunks: a chunk starts at an even index of its row,
        // bit 7 of its length byte holds the parity of the row's (i0 + i1)
        if (!level_node(v, t, p) || (((v.clen[t >> 5] >> 7) + (int)(t & 31)) & 1) != color) return;
    } else if (!decode_colour<D>(v.n, color, t, v.s0, v.s1, p)) {
        return;
    }
    if ((v.type[p] & NODE_KIND) != NODE_IN) return;
    const T s = mul_rn(v.h2, v.f[p]) + neighbour_sum<T, D>(v.u, p, v.s0, v.s1);   // h^2 f rounded on its own
    v.u[p] = s * (T)(1.0 / (2 * D));
}

// both colours in one pass over the active 2D tiles
template <typename T, int TR, int TC>
__global__ void __launch_bounds__(256) k_rb_fused2d(LevelView<T> v, T *__restrict__ out,
                                                    const int32_t *__restrict__ tiles) {
    pdl_wait();
    rb_fused2d_body<T, TR, TC>(v, out, tiles[blockIdx.x]);
}

// ------------------------------------------------ boundary types from a mask
// Ghost q of a level: the type of its boundary point B is the mask value at
// the fine node nearest B; on a tie (B halfway between two fine nodes along
// an axis) the node on the ghost's side is taken.
__global__ void k_mask_types(int dim, int n, double h, double o0, double o1, double o2, int step, int n_l,
                             const double *__restrict__ B, const int32_t *__restrict__ gnode, int ng,
                             const uint8_t *__restrict__ mask, uint8_t *__restrict__ types) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= ng) return;
    const double org[3] = {o0, o1, o2};
    int gj[3] = {0, 0, 0};
    int64_t rem = gnode[q];
    for (int a = dim - 1; a >= 0; a--) {   // the ghost's index on its own level
        gj[a] = (int)(rem % n_l);
        rem /= n_l;
    }
    int64_t node = 0;
    for (int a = 0; a < dim; a++) {
        const double x = (B[(int64_t)q * dim + a] - org[a]) / h;   // fine index coordinate of B
        const double fl = floor(x), fr = x - fl;
        const int g = gj[a] * step;                                   // the ghost's fine index
        int j = (int)fl + (fr > 0.5 ? 1 : 0);
        if (fr == 0.5) j = (double)g > x ? (int)fl + 1 : (int)fl;
        j = min(max(j, 0), n - 1);
        node = node * n + j;
    }
    types[q] = mask[node] ? 1 : 0;
}

// ------------------------------------------------ 3D fused red-black sweep
// One Gauss-Seidel sweep of Eq. (jac2d) (7-point form) in red-black order,
// both colours in one pass over the grid: a CTA owns a ZM_TY x ZM_TX tile of
// the (axis 1, axis 2) plane and marches along axis 0 over the planes
// [a, b) of its work item.  At step j it computes the red half-sweep on
// plane j over the tile and a 1-node halo (from the old values of planes
// j-1..j+1, staged with a 2-node halo) and the black half-sweep on plane
// j-1 over the tile (from the half-swept planes j-2..j), and stores plane
// j-1 into `out`.  Old u, f and the item's inside-node masks reach shared
// memory through asynchronous copies issued two steps before they are
// needed (u four planes ahead, f and masks three).  Every CTA reads only
// v.u and writes only its own nodes of `out`, so the result does not depend
// on the order of the CTAs; it equals the red sweep followed by the black
// sweep in place.  Sums in the order of the in-place kernels: h^2 f rounded
// on its own, then neighbours along axis 2, axis 0, then axis 1.
constexpr int ZM_THREADS = 512;

template <typename W>
__device__ __forceinline__ void cp_async_zfill(W *smem, const W *gmem, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    const unsigned bytes = valid ? (unsigned)sizeof(W) : 0u;   // 0: the word is zero-filled
    if constexpr (sizeof(W) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(gmem), "r"(bytes) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gmem), "r"(bytes) : "memory");
}
// 16 bytes, both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// waits for all but this thread's two most recent groups of copies
__device__ __forceinline__ void cp_async_wait_but2() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }

constexpr int ZM_UPLANES = 6, ZM_FPLANES = 5;   // ring depths of old u and of f (and the masks)

template <typename T>
constexpr size_t zmarch_smem_bytes() {
    return (size_t)(ZM_UPLANES * (ZM_TY + 4) * (ZM_TX + 4) + (ZM_FPLANES + 3) * (ZM_TY + 2) * (ZM_TX + 2)) *
               sizeof(T) +
           (size_t)ZM_FPLANES * ZM_MPLANE * sizeof(uint32_t);
}

template <typename T>
__global__ void __launch_bounds__(ZM_THREADS, sizeof(T) == 4 ? 3 : 1)
    k_rb_zmarch(LevelView<T> v, T *__restrict__ out, const int2 *__restrict__ items,
                const int32_t *__restrict__ moff, const uint32_t *__restrict__ masks) {
    constexpr int UX = ZM_TX + 4, US = (ZM_TY + 4) * UX;   // old u: 2-node halo
    constexpr int RX = ZM_TX + 2, RS = (ZM_TY + 2) * RX;   // red region: 1-node halo
    static_assert((ZM_UPLANES * US + (ZM_FPLANES + 3) * RS) % 4 == 0, "masks start 16-byte aligned");
    extern __shared__ __align__(16) unsigned char zm_smem[];
    T *su = reinterpret_cast<T *>(zm_smem);                         // ZM_UPLANES planes of old u
    T *sf = su + ZM_UPLANES * US;                                   // ZM_FPLANES planes of f
    T *sh = sf + ZM_FPLANES * RS;                                   // 3 half-swept planes
    uint32_t *sm = reinterpret_cast<uint32_t *>(sh + 3 * RS);       // ZM_FPLANES mask planes
    const int tid = threadIdx.x;
    const int2 item = items[blockIdx.x];
    const int r0 = (item.x >> 16) * ZM_TY, c0 = (item.x & 0xffff) * ZM_TX;
    const int a = item.y >> 16, b = item.y & 0xffff;
    const uint32_t *__restrict__ mg = masks + (int64_t)moff[blockIdx.x] * ZM_MPLANE;   // plane a - 1 first
    const int n = v.n;
    const int64_t s0 = v.s0;
    const T h2 = v.h2, sixth = (T)(1.0 / 6.0);
    const T *__restrict__ ug = v.u;
    const T *__restrict__ fg = v.f;
    auto u_slot = [&](int i) { return su + ((i + ZM_UPLANES) % ZM_UPLANES) * US; };   // i >= -1
    auto f_slot = [&](int i) { return sf + (i % ZM_FPLANES) * RS; };                  // i >= 0
    auto m_slot = [&](int i) { return sm + (i % ZM_FPLANES) * ZM_MPLANE; };
    auto h_slot = [&](int i) { return sh + (i % 3) * RS; };
    auto load_u = [&](int i) {   // plane i of old u (zeros outside the box)
        T *dst = u_slot(i);
        const bool pin = i >= 0 && i < n;
        for (int idx = tid; idx < US; idx += ZM_THREADS) {
            const int ry = idx / UX, gj = r0 - 2 + ry, gk = c0 - 2 + (idx - ry * UX);
            const bool ok = pin && gj >= 0 && gj < n && gk >= 0 && gk < n;
            cp_async_zfill(dst + idx, ok ? ug + (int64_t)i * s0 + (int64_t)gj * n + gk : ug, ok);
        }
    };
    auto load_f = [&](int i) {   // plane i of f over the red region, and its inside-node mask
        T *dst = f_slot(i);
        const bool pin = i >= 0 && i < n;
        for (int idx = tid; idx < RS; idx += ZM_THREADS) {
            const int ry = idx / RX, gj = r0 - 1 + ry, gk = c0 - 1 + (idx - ry * RX);
            const bool ok = pin && gj >= 0 && gj < n && gk >= 0 && gk < n;
            cp_async_zfill(dst + idx, ok ? fg + (int64_t)i * s0 + (int64_t)gj * n + gk : fg, ok);
        }
        if (tid < ZM_MPLANE / 4) cp_async16(m_slot(i) + 4 * tid, mg + (int64_t)(i - a + 1) * ZM_MPLANE + 4 * tid);
    };
    auto inside = [](const uint32_t *m, int ry, int rx) {
        return (m[ry * ZM_MROW + (rx >> 5)] >> (rx & 31)) & 1u;
    };

    pdl_wait();   // u comes from the previous launch
    // groups: {u a-2..a, f a-1}, then the groups of "steps" a-3 and a-2
    load_u(a - 2);
    load_u(a - 1);
    load_u(a);
    load_f(a - 1);
    cp_async_commit();
    load_u(a + 1);
    load_f(a);
    cp_async_commit();
    if (a + 2 <= b + 1) load_u(a + 2);
    if (a + 1 <= b) load_f(a + 1);
    cp_async_commit();
    cp_async_wait_but2();
    __syncthreads();
    for (int j = a - 1; j <= b; j++) {
        if (j + 4 <= b + 1) load_u(j + 4);
        if (j + 3 <= b) load_f(j + 3);
        cp_async_commit();   // possibly empty: one group per step keeps the count
        {   // red half-sweep on plane j, tile + 1-node halo
            const T *um = u_slot(j - 1), *uc = u_slot(j), *up = u_slot(j + 1);
            const T *fj = f_slot(j);
            const uint32_t *mj = m_slot(j);
            T *hj = h_slot(j);
            for (int idx = tid; idx < RS; idx += ZM_THREADS) {
                const int ry = idx / RX, rx = idx - ry * RX;
                const int ui = (ry + 1) * UX + rx + 1;
                T val = uc[ui];
                if (inside(mj, ry, rx) && ((j + ry + rx) & 1) == 0) {   // r0, c0 even
                    const T nb = (((uc[ui - 1] + uc[ui + 1]) + um[ui]) + up[ui]) + (uc[ui - UX] + uc[ui + UX]);
                    val = (mul_rn(h2, fj[idx]) + nb) * sixth;
                }
                hj[idx] = val;
            }
        }
        __syncthreads();
        if (j - 1 >= a) {   // black half-sweep on plane j - 1, the tile; store the plane
            const int i = j - 1;
            const T *hm = h_slot(i - 1), *hc = h_slot(i), *hp = h_slot(i + 1);
            const T *fi = f_slot(i);
            const uint32_t *mi = m_slot(i);
            for (int idx = tid; idx < ZM_TY * ZM_TX; idx += ZM_THREADS) {
                const int oy = idx / ZM_TX, ox = idx - oy * ZM_TX;
                const int gj = r0 + oy, gk = c0 + ox;
                if (gj >= n || gk >= n) continue;
                const int ri = (oy + 1) * RX + ox + 1;
                T val = hc[ri];
                if (inside(mi, oy + 1, ox + 1) && ((i + oy + ox) & 1) == 1) {
                    const T nb = (((hc[ri - 1] + hc[ri + 1]) + hm[ri]) + hp[ri]) + (hc[ri - RX] + hc[ri + RX]);
                    val = (mul_rn(h2, fi[ri]) + nb) * sixth;
                }
                out[(int64_t)i * s0 + (int64_t)gj * n + gk] = val;
            }
        }
        cp_async_wait_but2();
        __syncthreads();
    }
}

// ------------------------------------- 3D fused red-black sweep in registers
// The same sweep as k_rb_zmarch with the planes in registers: a CTA of
// SR_TY + 4 warps owns SR_TY rows (axis 1) x SR_W columns (axis 2); warp w
// holds row r0 - 2 + w, lane l column k0 - 2 + l, and every lane keeps the
// old values of planes j-1, j, j+1 and the half-swept values of planes j-2,
// j-1 of its node while the CTA marches along axis 0.  At step j a lane
// computes the red half-sweep of its node in plane j (rows 1..SR_TY+2,
// lanes 1..30: the tile and a 1-node halo) and the black half-sweep of its
// node in plane j-1 (which needs only plane j's own half-swept value and
// plane j-1's, known from the step before), and stores plane j-1 on the
// tile.  Neighbours along axis 2 come from the adjacent lanes (shuffles),
// along axis 1 from the adjacent warps through shared memory (two rows a
// warp, double buffered: one block barrier a plane).  u, f and node types
// are loaded three planes ahead into registers that are read only when
// their plane comes up (the step is unrolled three times, so no register
// copy waits on a load in flight).  Same sums in the same order as
// k_rb_zmarch: the results are bitwise equal.
template <typename T>
__global__ void __launch_bounds__((SR_TY + 4) * 32, sizeof(T) == 4 ? 3 : 2)
    k_rb_stream3d(LevelView<T> v, T *__restrict__ out, const int2 *__restrict__ items) {
    constexpr int NW = SR_TY + 4;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ T sx[2][2][NW][32];   // [step parity][old u of plane j, half-swept plane j-1][warp][lane]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 item = items[blockIdx.x];
    const int r0 = (item.x >> 16) * SR_TY, k0 = (item.x & 0xffff) * SR_W;
    const int a = item.y >> 16, b = item.y & 0xffff;
    const int n = v.n;
    const int row = r0 - 2 + w, col = k0 - 2 + lane;
    const bool ok = row >= 0 && row < n && col >= 0 && col < n;
    const int64_t off = ok ? (int64_t)row * n + col : 0;
    const int64_t s0 = v.s0;
    const bool red_here = w >= 1 && w <= NW - 2 && lane >= 1 && lane <= 30;
    const bool owner = ok && w >= 2 && w <= NW - 3 && lane >= 2 && lane <= SR_W + 1;
    const int par = (row + col) & 1;   // the node is red in plane i when i + par is even
    const T h2 = v.h2, sixth = (T)(1.0 / 6.0);
    const T *__restrict__ ug = v.u;
    const T *__restrict__ fg = v.f;
    const uint8_t *__restrict__ tg = v.type;
    // unconditional loads from a clamped address: a select on the loaded
    // value would wait for the load at once.  What a lane outside the box or
    // a plane outside [0, n) loads is never used by an update that is stored:
    // inside nodes are never on the box boundary, so all their neighbours are
    // in the box and in planes 1..n-2 (`owner` requires ok, and the node types
    // are masked with ok where they decide an update)
    auto at = [&](int i) { return (int64_t)min(max(i, 0), n - 1) * s0 + off; };
    auto ld_u = [&](int i) -> T { return ug[at(i)]; };
    auto ld_f = [&](int i) -> T { return fg[at(i)]; };
    auto ld_t = [&](int i) -> int { return (int)tg[at(i)]; };
    pdl_wait();   // u comes from the previous launch
    T om = ld_u(a - 2), oc = ld_u(a - 1), op = ld_u(a);   // old u, planes j-1, j, j+1
    T hm = 0, hc = 0;                                     // half-swept, planes j-2, j-1
    T fc = ld_f(a - 1), fm = 0;                           // f, planes j, j-1
    int tc = ld_t(a - 1), tm = 0;                         // node types, planes j, j-1
    T uq0 = ld_u(a + 1), uq1 = ld_u(a + 2), uq2 = ld_u(a + 3);
    T fq0 = ld_f(a), fq1 = ld_f(a + 1), fq2 = ld_f(a + 2);
    int tq0 = ld_t(a), tq1 = ld_t(a + 1), tq2 = ld_t(a + 2);   // (clamped: an item has >= 1 plane)
    auto step = [&](int j, T &uq, T &fq, int &tq) {
        T(*x)[NW][32] = sx[j & 1];
        x[0][w][lane] = oc;
        x[1][w][lane] = hc;
        __syncthreads();
        // red half-sweep on plane j
        const T ozm = __shfl_up_sync(FULL, oc, 1), ozp = __shfl_down_sync(FULL, oc, 1);
        const T oym = w > 0 ? x[0][w - 1][lane] : (T)0, oyp = w < NW - 1 ? x[0][w + 1][lane] : (T)0;
        T hn = oc;
        if (red_here && ok && j >= 0 && (tc & NODE_KIND) == NODE_IN && ((j + par) & 1) == 0)
            hn = (mul_rn(h2, fc) + ((((ozm + ozp) + om) + op) + (oym + oyp))) * sixth;
        // black half-sweep on plane j - 1, stored on the tile
        const T hzm = __shfl_up_sync(FULL, hc, 1), hzp = __shfl_down_sync(FULL, hc, 1);
        const T hym = w > 0 ? x[1][w - 1][lane] : (T)0, hyp = w < NW - 1 ? x[1][w + 1][lane] : (T)0;
        if (owner && j - 1 >= a) {
            T o = hc;
            if ((tm & NODE_KIND) == NODE_IN && ((j - 1 + par) & 1) == 1)
                o = (mul_rn(h2, fm) + ((((hzm + hzp) + hm) + hn) + (hym + hyp))) * sixth;
            out[(int64_t)(j - 1) * s0 + off] = o;
        }
        // advance one plane; the loads issued now are read three steps later
        // (none past the last plane the item reads: predicated, not selected)
        om = oc;
        oc = op;
        op = uq;
        if (j + 5 <= b + 1) uq = ld_u(j + 5);
        hm = hc;
        hc = hn;
        fm = fc;
        fc = fq;
        if (j + 4 <= b) fq = ld_f(j + 4);
        tm = tc;
        tc = tq;
        if (j + 4 <= b) tq = ld_t(j + 4);
    };
    int j = a - 1;
    while (true) {
        step(j, uq0, fq0, tq0);
        if (++j > b) break;
        step(j, uq1, fq1, tq1);
        if (++j > b) break;
        step(j, uq2, fq2, tq2);
        if (++j > b) break;
    }
}

// ------------------------------------- 3D fused red-black sweep on row spans
// The same sweep with a window that follows the domain along the contiguous
// axis: a CTA of SP_NW warps owns SP_J rows (axis 1), warp w holds row
// r0 - 2 + w, and lane l the nodes k0 + l + 32 c (c < C) of it -- a window
// of 32 C nodes along axis 2, of which the first and the last are halo.  The
// lane to the left of node k0 + 32 c is lane 31's column c - 1 and the one
// to the right of lane 31's column c is lane 0's column c + 1 (one shuffle
// each way a column); the outer neighbours of the window, k0 - 1 and
// k0 + 32 C, are loaded by lanes 31 and 0 as an extra column.  Per (plane,
// row) the level's metadata holds the span of the unknowns and of the inside
// nodes (the inside nodes of a row are one interval); a CTA stages the
// metadata of its planes in shared memory before it waits for the previous
// launch, and then reads u only on unknown spans, f only on inside spans and
// writes only unknowns, so the traffic follows the domain at 32-byte sector
// granularity.  Nodes outside the spans read 0; no update that is stored
// uses them (the neighbours of an inside node are unknowns).  The march is
// that of k_rb_stream3d: at step j the red half-sweep of plane j (rows
// 1 .. SP_NW - 2), the black half-sweep of plane j - 1 on the owned rows and
// columns, loads three planes ahead, one block barrier a plane.  Same sums
// in the same order: bitwise equal to red then black in place.
template <int C>
__global__ void __launch_bounds__(SP_NW * 32, 1)
    k_rb_span3d(LevelView<float> v, float *__restrict__ out, const int4 *__restrict__ items,
                const int2 *__restrict__ rows) {
    constexpr int NW = SP_NW, NP = SP_SEG + 4, PL = 2 * NW * C * 32;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char sp_smem[];
    int2 *meta = reinterpret_cast<int2 *>(sp_smem);                            // [NP][NW]
    float *sx = reinterpret_cast<float *>(sp_smem + NP * NW * sizeof(int2));    // [2][old, half][NW][C][32]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 it = items[blockIdx.x];
    const int r0 = it.x * SP_J, k0 = it.y, a = it.z, b = it.w;
    const int n = v.n;
    const int row = r0 - 2 + w;
    const int64_t s0 = v.s0;
    const int64_t rbase = (int64_t)row * n + k0 + lane;   // node (0, row, k0 + lane)
    const bool redrow = w >= 1 && w <= NW - 2, owner = w >= 2 && w <= NW - 3;
    const int par = (row + k0 + lane) & 1;   // a lane's nodes are red in plane i when i + par is even
    const float h2 = v.h2, sixth = (float)(1.0 / 6.0);
    const float *__restrict__ ug = v.u;
    const float *__restrict__ fg = v.f;
    // metadata of planes a - 2 .. b + 1 (set up once: read before the wait)
    const int np = b - a + 4;
    for (int q = threadIdx.x; q < np * NW; q += NW * 32) {
        const int p = a - 2 + q / NW, rr = r0 - 2 + q % NW;
        int2 m = make_int2(0xffff, 0xffff);
        if (p >= 0 && p < n && rr >= 0 && rr < n) m = rows[(int64_t)p * n + rr];
        meta[q] = m;
    }
    __syncthreads();
    auto has = [](int sp, int k) { return k >= (sp & 0xffff) && k <= (int)((unsigned)sp >> 16); };
    auto ld_u = [&](int p, float(&x)[C + 1]) {
        const int sp = meta[(p - a + 2) * NW + w].x;
        const float *src = ug + (int64_t)p * s0 + rbase;
#pragma unroll
        for (int c = 0; c < C; c++) {
            x[c] = 0.f;
            if (has(sp, k0 + lane + 32 * c)) x[c] = src[32 * c];
        }
        const int ke = lane == 31 ? k0 - 1 : k0 + 32 * C;   // the extra column
        x[C] = 0.f;
        if ((lane == 0 || lane == 31) && has(sp, ke)) x[C] = ug[(int64_t)p * s0 + (int64_t)row * n + ke];
    };
    auto ld_f = [&](int p, float(&x)[C]) {
        const int sp = meta[(p - a + 2) * NW + w].y;
        const float *src = fg + (int64_t)p * s0 + rbase;
#pragma unroll
        for (int c = 0; c < C; c++) {
            x[c] = 0.f;
            if (redrow && has(sp, k0 + lane + 32 * c)) x[c] = src[32 * c];
        }
    };
    float om[C], oc[C + 1], op[C + 1], hm[C], hc[C], fm[C], fc[C];
    float uq0[C + 1], uq1[C + 1], uq2[C + 1], fq0[C], fq1[C], fq2[C];
    pdl_wait();   // u comes from the previous launch
    {
        float t[C + 1];
        ld_u(a - 2, t);
#pragma unroll
        for (int c = 0; c < C; c++) om[c] = t[c];
    }
    ld_u(a - 1, oc);
    ld_u(a, op);
#pragma unroll
    for (int c = 0; c <= C; c++) uq0[c] = uq1[c] = uq2[c] = 0.f;
#pragma unroll
    for (int c = 0; c < C; c++) hm[c] = hc[c] = fm[c] = fq0[c] = fq1[c] = fq2[c] = 0.f;
    if (a + 1 <= b + 1) ld_u(a + 1, uq0);
    if (a + 2 <= b + 1) ld_u(a + 2, uq1);
    if (a + 3 <= b + 1) ld_u(a + 3, uq2);
    ld_f(a - 1, fc);
    ld_f(a, fq0);
    if (a + 1 <= b) ld_f(a + 1, fq1);
    if (a + 2 <= b) ld_f(a + 2, fq2);
    auto step = [&](int j, float(&uq)[C + 1], float(&fq)[C]) {
        float *x = sx + (j & 1) * PL;
#pragma unroll
        for (int c = 0; c < C; c++) {
            x[(w * C + c) * 32 + lane] = oc[c];
            x[((NW + w) * C + c) * 32 + lane] = hc[c];
        }
        __syncthreads();
        const int2 mj = meta[(j - a + 2) * NW + w];   // plane j
        const bool red = ((j + par) & 1) == 0;       // red in plane j, black in plane j - 1
        float hn[C];
        // red half-sweep on plane j
#pragma unroll
        for (int c = 0; c < C; c++) {
            const float sl = lane == 31 ? (c == 0 ? oc[C] : oc[c - 1]) : oc[c];
            const float sr = lane == 0 ? (c == C - 1 ? oc[C] : oc[c + 1]) : oc[c];
            const float ozm = __shfl_sync(FULL, sl, (lane + 31) & 31);
            const float ozp = __shfl_sync(FULL, sr, (lane + 1) & 31);
            const float oym = w > 0 ? x[((w - 1) * C + c) * 32 + lane] : 0.f;
            const float oyp = w < NW - 1 ? x[((w + 1) * C + c) * 32 + lane] : 0.f;
            hn[c] = oc[c];
            if (redrow && red && has(mj.y, k0 + lane + 32 * c))
                hn[c] = (mul_rn(h2, fc[c]) + ((((ozm + ozp) + om[c]) + op[c]) + (oym + oyp))) * sixth;
        }
        // black half-sweep on plane j - 1, stored on the owned rows and columns
        if (owner && j - 1 >= a) {
            const int2 mi = meta[(j - 1 - a + 2) * NW + w];
            float *o = out + (int64_t)(j - 1) * s0 + rbase;
#pragma unroll
            for (int c = 0; c < C; c++) {
                const float sl = lane == 31 ? (c == 0 ? 0.f : hc[c - 1]) : hc[c];
                const float sr = lane == 0 ? (c == C - 1 ? 0.f : hc[c + 1]) : hc[c];
                const float hzm = __shfl_sync(FULL, sl, (lane + 31) & 31);
                const float hzp = __shfl_sync(FULL, sr, (lane + 1) & 31);
                const float hym = x[((NW + w - 1) * C + c) * 32 + lane];
                const float hyp = x[((NW + w + 1) * C + c) * 32 + lane];
                const int k = k0 + lane + 32 * c;
                float val = hc[c];
                if (red && has(mi.y, k))
                    val = (mul_rn(h2, fm[c]) + ((((hzm + hzp) + hm[c]) + hn[c]) + (hym + hyp))) * sixth;
                const bool own = !(lane == 0 && c == 0) && !(lane == 31 && c == C - 1);
                if (own && has(mi.x, k)) o[32 * c] = val;
            }
        }
        // advance one plane; the loads issued now are read three steps later
#pragma unroll
        for (int c = 0; c < C; c++) {
            om[c] = oc[c];
            hm[c] = hc[c];
            hc[c] = hn[c];
            fm[c] = fc[c];
            fc[c] = fq[c];
        }
#pragma unroll
        for (int c = 0; c <= C; c++) {
            oc[c] = op[c];
            op[c] = uq[c];
        }
        if (j + 5 <= b + 1) ld_u(j + 5, uq);
        if (j + 4 <= b) ld_f(j + 4, fq);
    };
    int j = a - 1;
    while (true) {
        step(j, uq0, fq0);
        if (++j > b) break;
        step(j, uq1, fq1);
        if (++j > b) break;
        step(j, uq2, fq2);
        if (++j > b) break;
    }
}

// |v| for a max-norm that keeps NaN visible (as +Inf; fmax would drop it)
__device__ __forceinline__ double abs_keep_nan(double v) {
    const double a = fabs(v);
    return a != a ? __longlong_as_double(0x7ff0000000000000ll) : a;
}

// -------------------------------- 3D one-colour sweep over rows, in place
// One colour of the red-black interior sweep (Eq. jac2d, Sec. 2.4) over the
// rows that hold inside nodes, in place (the neighbours of a node are of the
// other colour, which the launch does not write).  The work is a list of
// segments, up to 64 consecutive inside nodes of one row (plane i, row j),
// in plane, row order; a warp takes G segments at once -- lane l the node
// of the colour at k_first + 2 l of each -- and issues the loads of all of
// them before the first update, so that G segments cost about one memory
// round trip; a persistent grid walks the list, prefetching the next group's
// segments.  The warps running together work on neighbouring rows and
// share them in L2; the black launch right after the red one finds much of
// u and f there.  The same sums in the same order as the fused sweeps.
template <typename T, int G>
__global__ void __launch_bounds__(256) k_rb_rows(LevelView<T> v, const int2 *__restrict__ segs, int nseg, int colour) {
    const int lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    int q = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * G;
    int2 nx[G];
#pragma unroll
    for (int g = 0; g < G; g++) nx[g] = q + g < nseg ? segs[q + g] : make_int2(0, 0x0000ffff);   // static
    pdl_wait();
    const int n = v.n;
    const int64_t s0 = v.s0;
    const T h2 = v.h2, sixth = (T)(1.0 / 6.0);
    T *u = v.u;
    const T *__restrict__ f = v.f;
    for (; q < nseg; q += nw * G) {
        int64_t p[G];
        bool on[G];
        T zm[G], zp[G], xm[G], xp[G], ym[G], yp[G], fv[G];
#pragma unroll
        for (int g = 0; g < G; g++) {
            const int2 sg = nx[g];
            const int i = sg.x / n, j = sg.x - (sg.x / n) * n;
            const int k0 = sg.y & 0xffff, k1 = (int)((unsigned)sg.y >> 16);
            const int k = k0 + ((i + j + k0 + colour) & 1) + 2 * lane;
            on[g] = k <= k1;
            p[g] = (int64_t)sg.x * n + k;
            if (on[g]) {
                zm[g] = u[p[g] - 1];
                zp[g] = u[p[g] + 1];
                xm[g] = u[p[g] - s0];
                xp[g] = u[p[g] + s0];
                ym[g] = u[p[g] - n];
                yp[g] = u[p[g] + n];
                fv[g] = f[p[g]];
            }
        }
        const int qn = q + nw * G;
#pragma unroll
        for (int g = 0; g < G; g++) nx[g] = qn + g < nseg ? segs[qn + g] : make_int2(0, 0x0000ffff);
#pragma unroll
        for (int g = 0; g < G; g++)
            if (on[g]) u[p[g]] = (mul_rn(h2, fv[g]) + ((((zm[g] + zp[g]) + xm[g]) + xp[g]) + (ym[g] + yp[g]))) * sixth;
    }
}

// The defect f + Lap_h u (TGCS step 3) at every inside node of a 3D level
// into r, over the row segments: a warp takes G segments at once, lane l the
// nodes k0 + l and k0 + l + 32 of each, all loads issued before the first
// store; with norm, its max-norm.  MIXED (the FP64 finest level of the mixed
// form): also f32 = the defect rounded to FP32 and e32 = 0 at those nodes.
// The expression of defect_node.
template <typename T, int G, bool MIXED>
__global__ void __launch_bounds__(256) k_defect_rows(LevelView<T> v, unsigned long long *norm, float *__restrict__ f32,
                                                    float *__restrict__ e32) {
    if (MIXED) pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const int n = v.n, nseg = v.nsegs;
    const int2 *__restrict__ segs = v.segs;
    pdl_wait();
    // the max-norm on the bit patterns of |d| (integer compares; the order of
    // non-negative doubles, NaN above +Inf, which reduce_norm maps to +Inf)
    unsigned long long mb = 0;
    for (int q = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * G; q < nseg; q += nw * G) {
        T d[2 * G];
        int64_t p[2 * G];
        bool on[2 * G];
#pragma unroll
        for (int g = 0; g < G; g++) {
            const int2 sg = q + g < nseg ? segs[q + g] : make_int2(0, 0x0000ffff);
            const int k0 = sg.y & 0xffff, k1 = (int)((unsigned)sg.y >> 16);
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int k = k0 + lane + 32 * h;
                on[2 * g + h] = k <= k1;
                p[2 * g + h] = (int64_t)sg.x * n + k;
                if (on[2 * g + h]) d[2 * g + h] = inside_defect<T, 3>(v, p[2 * g + h]);
            }
        }
#pragma unroll
        for (int e = 0; e < 2 * G; e++)
            if (on[e]) {
                v.r[p[e]] = d[e];
                if (MIXED) {
                    f32[p[e]] = (float)d[e];
                    e32[p[e]] = 0.0f;
                }
                const unsigned long long b = (unsigned long long)__double_as_longlong((double)d[e]) & 0x7fffffffffffffffull;
                mb = b > mb ? b : mb;
            }
    }
    reduce_norm(norm, __longlong_as_double((long long)mb));
}

// The interpolation of the coarse correction added at every unknown of a 3D
// level (Sec. 2.6; the sums of prolong_node_early): the inside nodes over
// the row segments, G at once, lane l the nodes k0 + l and k0 + l + 32 of
// each, every parent's type and value loaded before the first sum; past
// them the ghosts, a thread each.
template <typename T, int G>
__global__ void __launch_bounds__(256) k_prolong_rows(LevelView<T> F, LevelView<T> C, const T *__restrict__ e,
                                                      T *__restrict__ out) {
    if (sizeof(T) == 4) pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const int n = F.n, nseg = F.nsegs;
    pdl_wait();
    for (int q = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * G; q < nseg; q += nw * G) {
        T ev[2 * G][8], old[2 * G];
        bool use[2 * G][8], on[2 * G];
        int64_t pp[2 * G];
        int cnt[2 * G];
#pragma unroll
        for (int g = 0; g < G; g++) {
            const int2 sg = q + g < nseg ? F.segs[q + g] : make_int2(0, 0x0000ffff);
            const int i = sg.x / n, j = sg.x - (sg.x / n) * n;
            const int k0 = sg.y & 0xffff, k1 = (int)((unsigned)sg.y >> 16);
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int e_ = 2 * g + h, k = k0 + lane + 32 * h;
                on[e_] = k <= k1;
                pp[e_] = (int64_t)sg.x * n + k;
                const int n1 = (i & 1) ? 2 : 1, n2 = (j & 1) ? 2 : 1, n3 = (k & 1) ? 2 : 1;
                cnt[e_] = n1 * n2 * n3;
                const int64_t X0 = (int64_t)(i / 2) * C.s0 + (int64_t)(j / 2) * C.s1 + k / 2;
#pragma unroll
                for (int s8 = 0; s8 < 8; s8++) {
                    const int a = s8 >> 2, b = (s8 >> 1) & 1, c = s8 & 1;
                    const int64_t X = X0 + a * C.s0 + b * C.s1 + c;
                    use[e_][s8] = false;
                    if (on[e_] && a < n1 && b < n2 && c < n3) {
                        const uint8_t kc = C.type[X] & NODE_KIND;
                        use[e_][s8] = kc == NODE_IN || kc == NODE_GHOST;   // parents in Omega_2h u Gamma_2h
                    }
                    ev[e_][s8] = use[e_][s8] ? e[X] : (T)0;
                }
                old[e_] = on[e_] ? out[pp[e_]] : (T)0;
            }
        }
#pragma unroll
        for (int e_ = 0; e_ < 2 * G; e_++) {
            if (!on[e_]) continue;
            T num = 0, den = 0;
            const T w = (T)1 / (T)cnt[e_];   // a power of two: exact
#pragma unroll
            for (int s8 = 0; s8 < 8; s8++)
                if (use[e_][s8]) {
                    num += w * ev[e_][s8];
                    den += w;
                }
            const T val = den > (T)0 ? num / den : (T)0;
            out[pp[e_]] = old[e_] + val;
        }
    }
    for (int qg = (int)(blockIdx.x * blockDim.x + threadIdx.x); qg < F.ng; qg += (int)(gridDim.x * blockDim.x))
        prolong_node<T, 3>(F, C, e, out, true, F.gnode[qg]);
}

// u64 += e32 at the inside nodes over the row segments (G at once) and, past
// them, at the ghosts
template <int G>
__global__ void __launch_bounds__(256) k_add_rows(LevelView<double> v, double *__restrict__ u64,
                                                  const float *__restrict__ e32) {
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const int n = v.n, nseg = v.nsegs;
    const int2 *__restrict__ segs = v.segs;
    pdl_wait();
    for (int q = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * G; q < nseg; q += nw * G) {
        double a[2 * G];
        float b[2 * G];
        int64_t p[2 * G];
        bool on[2 * G];
#pragma unroll
        for (int g = 0; g < G; g++) {
            const int2 sg = q + g < nseg ? segs[q + g] : make_int2(0, 0x0000ffff);
            const int k0 = sg.y & 0xffff, k1 = (int)((unsigned)sg.y >> 16);
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int k = k0 + lane + 32 * h;
                on[2 * g + h] = k <= k1;
                p[2 * g + h] = (int64_t)sg.x * n + k;
                if (on[2 * g + h]) {
                    a[2 * g + h] = u64[p[2 * g + h]];
                    b[2 * g + h] = e32[p[2 * g + h]];
                }
            }
        }
#pragma unroll
        for (int e = 0; e < 2 * G; e++)
            if (on[e]) u64[p[e]] = a[e] + (double)b[e];
    }
    for (int q = (int)(blockIdx.x * blockDim.x + threadIdx.x); q < v.ng; q += (int)(gridDim.x * blockDim.x)) {
        const int64_t g = v.gnode[q];
        u64[g] += (double)e32[g];
    }
}

template <typename K>
static unsigned resident_blocks(K kernel) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, 0);
    return (unsigned)std::max(1, sms * std::max(per, 1));
}

// a persistent grid over a level's row segments, G a warp at once
template <typename K>
static unsigned segment_blocks(K kernel, int nseg, int G, unsigned &resident) {
    if (resident == 0) resident = resident_blocks(kernel);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)(nseg + G - 1) / G * 32 + 255) / 256, resident));
}

// ------------------------------------------- 3D boundary phase in one launch
// Grid-wide barrier for k_boundary3d, whose CTAs are all resident at once
// (the grid is sized by the kernel's occupancy and the launch does not
// overlap another kernel of the stream).  bar[0] counts arrivals, bar[1] is
// the generation.  A wait gives up after `spin` polls: it sets *err (reported
// as GCMG_E_TIMEOUT) and returns, and once *err is set no later barrier
// waits, so the launch always ends.  Writes before the barrier are visible
// to every CTA after it (fences on both sides; u is read with L2-coherent
// loads, see ldu).
__device__ __forceinline__ void grid_barrier(unsigned *bar, unsigned nbar, int *err, unsigned spin) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        volatile int *verr = err;
        const unsigned g = atomicAdd(bar + 1, 0u);
        __threadfence();
        if (atomicAdd(bar, 1u) == nbar - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned it = 0;
            while (*gen == g && !*verr) {
                if (++it > spin) {
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// u is written by other CTAs between the phases of one launch: read it
// through L2 (ld.global.cg), never from a possibly stale L1 line
template <typename T>
__device__ __forceinline__ T ldu(const T *p) { return __ldcg(p); }

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The phases of one 3D boundary relaxation; between two phases a grid-wide
// barrier (CLUSTER = false: every CTA of the launch, grid_barrier) or the
// hardware barrier of a thread-block cluster (CLUSTER = true: the launch is
// one cluster)
template <typename T, bool CLUSTER>
__device__ __forceinline__ void boundary3d_body(LevelView<T> &v, const BoundaryProgram3 &P) {
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
    T *__restrict__ u = v.u;
    auto band = [&](const int32_t *__restrict__ list, int cnt) {   // Gauss-Seidel form of Eq. (jac2d), 7 points
        for (int64_t i = t0; i < cnt; i += st) {
            const int64_t p = list[i];
            T nb = ldu(u + p - 1) + ldu(u + p + 1) + ldu(u + p - v.s0) + ldu(u + p + v.s0);
            nb += ldu(u + p - v.s1) + ldu(u + p + v.s1);
            u[p] = (mul_rn(v.h2, v.f[p]) + nb) * (T)(1.0 / 6.0);
        }
    };
    auto ghost_new = [&](const int32_t *__restrict__ list, int cnt) {   // Eqs. (dir2d)/(neu2d), Jacobi
        for (int64_t i = t0; i < cnt; i += st) {
            const int q = list ? list[i] : (int)i;
            T s = 0;
#pragma unroll
            for (int k = 0; k < 27; k++) s += v.gw[(int64_t)k * v.ng + q] * ldu(u + v.gstn[(int64_t)k * v.ng + q]);
            v.gtmp[q] = ldu(u + v.gnode[q]) + v.gc[q] * (v.gg[q] - s);
        }
    };
    auto ghost_store = [&](const int32_t *__restrict__ list, int cnt) {
        for (int64_t i = t0; i < cnt; i += st) {
            const int q = list ? list[i] : (int)i;
            u[v.gnode[q]] = __ldcg(v.gtmp + q);
        }
    };
    auto sync = [&]() {
        if (CLUSTER) cluster_sync_all();
        else grid_barrier(P.bar, P.nbar, P.err, P.spin);
    };
    pdl_wait();
    bool first = true;
    auto phase_sync = [&]() {   // a barrier before every phase but the first
        if (!first) sync();
        first = false;
    };
    if (P.lead) {
        phase_sync(); ghost_new(nullptr, v.ng);
        phase_sync(); ghost_store(nullptr, v.ng);
    }
    for (int k = 0; k < P.lambda; k++) {
        phase_sync(); band(P.red, P.nred);
        phase_sync(); band(P.black, P.nblack);
        phase_sync(); ghost_new(nullptr, v.ng);
        phase_sync(); ghost_store(nullptr, v.ng);
    }
    for (int k = 0; k < P.mu; k++) {
        phase_sync(); band(P.zred, P.nzred);
        phase_sync(); band(P.zblack, P.nzblack);
        phase_sync(); ghost_new(P.zghost, P.nzghost);
        phase_sync(); ghost_store(P.zghost, P.nzghost);
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_boundary3d(LevelView<T> v, BoundaryProgram3 P) {
    boundary3d_body<T, false>(v, P);
}

// the same as one thread-block cluster of BC_SIZE CTAs (small levels and the
// junction zone: a few thousand entries a phase)
constexpr int BC_SIZE = 16, BC_THREADS = 1024;
template <typename T>
__global__ void __launch_bounds__(BC_THREADS) k_boundary3d_cluster(LevelView<T> v, BoundaryProgram3 P) {
    boundary3d_body<T, true>(v, P);
}

// Same update over a compact list of band nodes of one colour (Sec. 3.2).
template <typename T, int D, int LIST_M>
__global__ void k_rb_list(LevelView<T> v, const int32_t *__restrict__ list, int cnt) {
    // entries i0 + m * (threads of the launch), m < LIST_M: the loads of all
    // of a thread's entries are issued before its first update; the list is
    // fixed and read before the wait for the previous launch, and the next
    // launch may start reading its own fixed data meanwhile
    pdl_trigger();
    const int nt = (int)(gridDim.x * blockDim.x), i0 = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    int64_t p[LIST_M];
    T sum[LIST_M];
#pragma unroll
    for (int m = 0; m < LIST_M; m++) p[m] = i0 + m * nt < cnt ? list[i0 + m * nt] : -1;
    pdl_wait();
#pragma unroll
    for (int m = 0; m < LIST_M; m++)
        if (p[m] >= 0) sum[m] = mul_rn(v.h2, v.f[p[m]]) + neighbour_sum<T, D>(v.u, p[m], v.s0, v.s1);   // h^2 f rounded on its own
#pragma unroll
    for (int m = 0; m < LIST_M; m++)
        if (p[m] >= 0) v.u[p[m]] = sum[m] * (T)(1.0 / (2 * D));
}

// The red half of a 3D band or junction-zone sweep merged with the store of
// the ghosts' new values: threads below cnt update the list's red nodes,
// reading each axis neighbour from src (slot major: the node, or -1 - q for
// ghost q, whose new value is still in gtmp), threads past cnt store gtmp
// into u for the ghosts of glist (null: every ghost).  Nothing the updates
// read is written in the launch (their neighbours are black nodes and
// ghosts).  The sum of k_rb_list in the same order.
template <typename T, int LIST_M>
__global__ void k_rb_list_store(LevelView<T> v, const int32_t *__restrict__ list, const int32_t *__restrict__ src,
                                int cnt, const int32_t *__restrict__ glist, int gcnt) {
    // items i0 + m * (threads of the launch), m < LIST_M, loads first (as
    // k_rb_list); the lists, sources and ghost nodes are fixed and read
    // before the wait for the previous launch
    pdl_trigger();
    const int nt = (int)(gridDim.x * blockDim.x), i0 = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    T x[LIST_M][6], fv[LIST_M], gv[LIST_M];
    int64_t p[LIST_M];
    int kind[LIST_M];   // 0 none, 1 red entry, 2 ghost store
    int sk[LIST_M][6], gq[LIST_M];
#pragma unroll
    for (int m = 0; m < LIST_M; m++) {
        const int i = i0 + m * nt;
        kind[m] = i < cnt ? 1 : i - cnt < gcnt ? 2 : 0;
        p[m] = 0;
        gq[m] = 0;
        if (kind[m] == 1) {
            p[m] = list[i];
#pragma unroll
            for (int k = 0; k < 6; k++) sk[m][k] = src[(int64_t)k * cnt + i];
        } else if (kind[m] == 2) {
            gq[m] = glist ? glist[i - cnt] : i - cnt;
            p[m] = v.gnode[gq[m]];
        }
    }
    pdl_wait();
#pragma unroll
    for (int m = 0; m < LIST_M; m++) {
        if (kind[m] == 1) {
#pragma unroll
            for (int k = 0; k < 6; k++) x[m][k] = sk[m][k] >= 0 ? v.u[sk[m][k]] : v.gtmp[-1 - sk[m][k]];
            fv[m] = v.f[p[m]];
        } else if (kind[m] == 2) {
            gv[m] = v.gtmp[gq[m]];
        }
    }
#pragma unroll
    for (int m = 0; m < LIST_M; m++) {
        if (kind[m] == 1) {
            T nb = x[m][0] + x[m][1] + x[m][2] + x[m][3];
            nb += x[m][4] + x[m][5];
            const T s = mul_rn(v.h2, fv[m]) + nb;   // h^2 f rounded on its own
            v.u[p[m]] = s * (T)(1.0 / 6.0);
        } else if (kind[m] == 2) {
            v.u[p[m]] = gv[m];
        }
    }
}

// Ghost relaxation, Eqs. (dir2d)/(neu2d): new value from the current values.
// The ghost's stencil, weights, coefficient and node are fixed while a
// solve runs: they are read before the wait for the previous launch, the
// values of u and g after it (one round trip instead of three).
template <typename T, int K>
__device__ __forceinline__ void ghost_new_early(const LevelView<T> &v, int q, bool on) {
    int32_t st[K], gn = 0;
    T w[K], gc = 0;
    if (on) {
        gc = v.gc[q];
        gn = v.gnode[q];
        const unsigned code = K == 27 && v.gcode ? v.gcode[q] : 0u;
        if (code) {
            // a box stencil: the nodes from slot 0 and the axis directions;
            // an 8-slot box pads with the ghost itself and zero weights
            const int m = (int)(code & 3u);
            const int64_t b0 = v.gbase[q], D0 = (code & 4u) ? -v.s0 : v.s0, D1 = (code & 8u) ? -v.s1 : v.s1;
            const int64_t D2 = (code & 16u) ? -1 : 1;
#pragma unroll
            for (int k = 0; k < K; k++) {
                if (m == 3) st[k] = (int32_t)(b0 + (k / 9) * D0 + ((k / 3) % 3) * D1 + (k % 3) * D2);
                else st[k] = k < 8 ? (int32_t)(b0 + (k / 4) * D0 + ((k / 2) % 2) * D1 + (k % 2) * D2) : gn;
                w[k] = (m == 2 && k >= 8) ? (T)0 : v.gw[(int64_t)k * v.ng + q];
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; k++) {
                st[k] = v.gstn[(int64_t)k * v.ng + q];
                w[k] = v.gw[(int64_t)k * v.ng + q];
            }
        }
    }
    pdl_wait();
    if (!on) return;
    T s = 0;
#pragma unroll
    for (int k = 0; k < K; k++) s += w[k] * v.u[st[k]];
    v.gtmp[q] = v.u[gn] + gc * (v.gg[q] - s);
}

template <typename T, int K>
__global__ void k_ghost_new(LevelView<T> v) {
    pdl_trigger();   // the next launch reads its fixed data while this one runs
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    ghost_new_early<T, K>(v, q, q < v.ng);
}

// same update restricted to a list of ghost numbers
template <typename T, int K>
__global__ void k_ghost_new_list(LevelView<T> v, const int32_t *__restrict__ list, int cnt) {
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    ghost_new_early<T, K>(v, i < cnt ? list[i] : 0, i < cnt);
}

template <typename T>
__global__ void k_ghost_store_list(LevelView<T> v, const int32_t *__restrict__ list, int cnt) {
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int q = 0;
    int32_t gn = 0;
    if (i < cnt) {   // fixed: read before the wait
        q = list[i];
        gn = v.gnode[q];
    }
    pdl_wait();
    if (i >= cnt) return;
    v.u[gn] = v.gtmp[q];
}

template <typename T>
__global__ void k_ghost_store(LevelView<T> v) {
    pdl_trigger();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t gn = q < v.ng ? v.gnode[q] : 0;   // fixed: read before the wait
    pdl_wait();
    if (q >= v.ng) return;
    v.u[gn] = v.gtmp[q];
}

// shared-memory programs (junction zones, 2D boundary blocks), one CTA per
// component; two CTAs per SM for the FP32 2D programs (64 registers, no
// spills), the FP64 and 3D ones need more registers than that
template <typename T, int D>
__global__ void __launch_bounds__(LOCAL_THREADS, sizeof(T) == 4 && D == 2 ? 2 : 1)
    k_local(LocalView<T> J, int lead_ghost, int reps) {
    pdl_wait();
    local_body<T, D>(J, J.u, J.wb ? J.wb : J.u, blockIdx.x, lead_ghost, reps);
}

// ------------------------------------------------------------------ defect
// grid-stride over the level's nodes: a capped grid keeps the number of
// atomic updates of the norm word small
template <typename T, int D>
__global__ void k_defect_interior(LevelView<T> v, bool zero_rest, unsigned long long *norm) {
    pdl_wait();
    if (zero_rest) v.chunks = nullptr;   // every node of r is written: the whole box
    const int64_t nt = v.chunks ? v.nchunks * CHUNK : v.nn;
    double m = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t p;
        if (level_node(v, t, p)) m = fmax(m, abs_keep_nan(defect_node<T, D>(v, p, zero_rest)));
    }
    reduce_norm(norm, m);
}

template <typename T, int K>
__global__ void k_defect_ghost(LevelView<T> v, unsigned long long *norm) {
    pdl_wait();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const double val = q < v.ng ? defect_ghost_item<T, K>(v, q) : 0.0;
    reduce_norm(norm, val);
}

// ---------------------------------------------------------------- extension
// One wavefront of the defect extension (Sec. 2.6).
template <typename T>
__global__ void k_extend(T *__restrict__ r, const int32_t *__restrict__ node, const uint8_t *__restrict__ cnt,
                         const int32_t *__restrict__ src, const T *__restrict__ w, int ne, int begin, int end) {
    pdl_wait();
    const int i = begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= end) return;
    T s = 0;
    const int c = cnt[i];
    for (int k = 0; k < c; k++) s += w[(int64_t)k * ne + i] * r[src[(int64_t)k * ne + i]];
    r[node[i]] = s;
}

// ------------------------------------------------------------- restriction
template <typename T, int D>
__global__ void k_restrict_interior(LevelView<T> F, LevelView<T> C, T *__restrict__ fc) {
    pdl_wait();
    const int64_t X = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (X < C.nn) restrict_node<T, D>(F, C, X, fc);
}

template <typename T, int D, bool FROM_R>
__global__ void k_descend(LevelView<T> F, LevelView<T> C, T *__restrict__ fc, T *__restrict__ gc,
                          T *__restrict__ uc, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                          const T *__restrict__ val, bool split) {
    // FP32 instances let their dependents start now; FP64 ones do not (their
    // dependents are large FP64 launches whose early CTAs measured slower)
    if (sizeof(T) == 4) pdl_trigger();
    if (D == 3) {
        // 3D: the coarse nodes of the coarse level's active chunks, a thread
        // each (every unknown is in one; the other nodes keep u = 0 and an f
        // that nothing reads); the coarse ghost rows are summed by k_ghost_rows
        // (split: the coarse nodes whose neighbourhood is partly outside are
        // left to k_descend_partial)
        int64_t i;
        const bool has = level_node(C, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, i);
        pdl_wait();
        if (has) descend_node<T, D, FROM_R>(F, C, fc, uc, i, split);
        return;
    }
    if (sizeof(T) == 8) {
        // the thread-per-index form: in FP64 the terms are plain reads of r
        pdl_wait();
        descend_item<T, D, FROM_R>(F, C, fc, gc, uc, ptr, col, val, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
        return;
    }
    // 2D: the first 32 C.ng threads take the coarse ghost rows, a warp each;
    // the rest the coarse nodes, a thread each; both read their static data
    // before waiting for the previous launch
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nw = 32 * (int64_t)C.ng;
    if (t < nw) descend_ghost_row_warp_early<T, D, FROM_R>(F, gc, ptr, col, val, (int)(t >> 5));   // uniform over the warp
    else if (t - nw < C.nn) descend_node_early<T, D, FROM_R>(F, C, fc, uc, t - nw);
}

// 3D descent at the coarse inside nodes whose fine neighbourhood is partly
// outside Omega_h (the box search of the partial transfer), a thread each:
// kept out of k_descend so that its warps all take full weighting
// The weights (w, 27 per node, slot major) come from the host, computed with
// the device's operations in its order; the sum is that of partial_transfer_of.
template <typename T>
__global__ void k_descend_partial(LevelView<T> F, LevelView<T> C, T *__restrict__ fc,
                                  const int32_t *__restrict__ list, const T *__restrict__ w, int cnt) {
    if (sizeof(T) == 4) pdl_trigger();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = 0, p = 0;
    T wc[27];
    if (t < cnt) {   // set up once: read before the wait
        i = list[t];
        p = fine_image<3>(i, C.s0, C.s1, F.s0, F.s1);
#pragma unroll
        for (int c = 0; c < 27; c++) wc[c] = w[(int64_t)c * cnt + t];
    }
    pdl_wait();
    if (t >= cnt) return;
    T val[27];
#pragma unroll
    for (int c = 0; c < 27; c++)
        val[c] = wc[c] != (T)0 ? F.r[p + (c / 9 - 1) * F.s0 + ((c / 3) % 3 - 1) * F.s1 + (c % 3 - 1)] : (T)0;
    T acc = 0;
#pragma unroll
    for (int c = 0; c < 27; c++)
        if (wc[c] != (T)0) acc += wc[c] * val[c];
    fc[i] = acc;
}

// 3D descent, coarse ghost rows (extension + partial transfer at coarse ghost
// q as one sparse row over the fine ghost defects): a warp per row, the lanes
// over every 32nd term, then a butterfly sum.  The fine ghost defects come
// from rg[column] (FP32: computed once by k_ghost_defects) or, with GATHER,
// from rg[gnode[column]] (FP64: the defect grid).
template <typename T, bool GATHER>
__global__ void k_ghost_rows(const T *__restrict__ rg, const int32_t *__restrict__ gnode, T *__restrict__ gc,
                             const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                             const T *__restrict__ val, int nrows) {
    if (sizeof(T) == 4) pdl_trigger();
    pdl_wait();
    const int q = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (q >= nrows) return;   // uniform over the warp
    T s = 0;
    const int end = ptr[q + 1];
    for (int j = ptr[q] + lane; j < end; j += 32) s = fma(val[j], rg[GATHER ? gnode[col[j]] : col[j]], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) gc[q] = s;
}

// g - L_G u at every ghost of a level into v.gtmp (free between
// relaxations), for the 3D FP32 descent
template <typename T, int K>
__global__ void k_ghost_defects(LevelView<T> v) {
    pdl_trigger();
    pdl_wait();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < v.ng) v.gtmp[q] = ghost_defect<T, K>(v, q);
}

template <typename T, int D>
__global__ void k_restrict_ghost(LevelView<T> F, LevelView<T> C, T *__restrict__ gc) {
    pdl_wait();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < C.ng) restrict_ghost_item<T, D>(F, C, q, gc);
}

template <typename T>
__global__ void k_ghost_transfer(const T *__restrict__ rf, const int32_t *__restrict__ fgnode,
                                 const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                 const T *__restrict__ val, T *__restrict__ gc, int ngc) {
    pdl_wait();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < ngc) ghost_transfer_row<T>(rf, fgnode, ptr, col, val, gc, q);
}

// ------------------------------------------------------------ interpolation
template <typename T, int D>
__global__ void k_prolong(LevelView<T> F, LevelView<T> C, const T *__restrict__ e, T *__restrict__ out, bool add) {
    if (sizeof(T) == 4) pdl_trigger();
    if (!add) F.chunks = nullptr;   // every node of out is written: the whole box
    int64_t p;
    if (level_node(F, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, p))
        prolong_node_early<T, D>(F, C, e, out, add, p);   // waits after reading the types
    else
        pdl_wait();
}

// --------------------------------------------------------------- coarsest
template <typename T>
__global__ void k_coarse_solve(LevelView<T> v, const int32_t *__restrict__ unk_node,
                               const int32_t *__restrict__ unk_ghost, const T *__restrict__ Ainv, int m) {
    if (sizeof(T) == 4) pdl_trigger();
    pdl_wait();
    coarse_rows<T>(v, unk_node, unk_ghost, Ainv, m, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------- mixed precision
// FP64 defect of the finest level (r, its norm) that also sets up the next
// FP32 correction problem: right-hand side = the defect rounded to FP32 at
// inside nodes, 0 elsewhere; initial correction e32 = 0 everywhere
template <int D>
__global__ void k_defect_interior_mixed(LevelView<double> v, unsigned long long *norm, float *__restrict__ f32,
                                        float *__restrict__ e32) {
    pdl_trigger();
    pdl_wait();
    const int64_t nt = v.chunks ? v.nchunks * CHUNK : v.nn;
    double m = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t p;
        if (!level_node(v, t, p)) continue;   // nodes off the chunks stay 0
        const double val = defect_node<double, D>(v, p, false);   // 0 off Omega_h
        f32[p] = (float)val;
        e32[p] = 0.0f;
        m = fmax(m, abs_keep_nan(val));
    }
    reduce_norm(norm, m);
}

// ... and its ghost rows: the ghost defects rounded to FP32
// (e32: when not null, also e32 = 0 at the ghosts)
template <int K>
__global__ void k_defect_ghost_mixed(LevelView<double> v, unsigned long long *norm, float *__restrict__ g32,
                                     float *__restrict__ e32) {
    pdl_trigger();
    pdl_wait();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    double val = 0.0;
    if (q < v.ng) {
        val = defect_ghost_item<double, K>(v, q);
        g32[q] = (float)val;
        if (e32) e32[v.gnode[q]] = 0.0f;
    }
    reduce_norm(norm, val);
}

// u64 += e32 on Omega_h u Gamma_h
__global__ void k_add_correction(LevelView<double> v, double *__restrict__ u64, const float *__restrict__ e32) {
    pdl_trigger();
    pdl_wait();
    const uint8_t *__restrict__ type = v.type;
    int64_t p;
    if (!level_node(v, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, p)) return;
    const uint8_t k = type[p] & NODE_KIND;
    if (k == NODE_IN || k == NODE_GHOST) u64[p] += (double)e32[p];
}

// keep u = 0 off Omega_h u Gamma_h
template <typename T>
__global__ void k_mask_unknowns(const uint8_t *__restrict__ type, T *__restrict__ u, int64_t nn) {
    pdl_wait();
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nn) return;
    const uint8_t k = type[p] & NODE_KIND;
    if (k != NODE_IN && k != NODE_GHOST) u[p] = 0;
}

}  // namespace

// ------------------------------------------------------------- launchers
template <typename T>
void launch_rb(const LevelView<T> &v, int dim, int color, cudaStream_t s) {
    const int hc = (v.n + 1) / 2;
    g_launches++;
    if (dim == 2) pdl_launch(k_rb_interior<T, 2>, dim3(blocks_for((int64_t)v.n * hc)), dim3(kThreads), 0, s, v, color);
    else if (v.chunks) pdl_launch(k_rb_interior<T, 3>, dim3(blocks_for(v.nchunks * CHUNK)), dim3(kThreads), 0, s, v, color);
    else pdl_launch(k_rb_interior<T, 3>, dim3(blocks_for((int64_t)v.n * v.n * hc)), dim3(kThreads), 0, s, v, color);
}

// One FP32 2D relaxation in one launch: the first nsc CTAs sweep the strips
// (one a warp) and store the inside nodes outside the band; the others run
// the boundary blocks from the same grid v.u -- each block first takes the
// interior sweep over what it reads, then the ghost sweep and the band
// sweeps -- and store their band nodes and ghosts.  Every CTA reads only
// v.u and the stored node sets are disjoint, so nothing is written twice and
// no CTA reads a value another one writes.
// EPT: inside entries per thread and colour the boundary blocks need
template <int SR, int EPT>
__global__ void __launch_bounds__(LOCAL_THREADS, 2)
    k_relax2d(LevelView<float> v, float *__restrict__ out, const int32_t *__restrict__ strips, int ns, int nsc,
              LocalView<float> J, int lambda) {
    pdl_trigger();
    if ((int)blockIdx.x < nsc) {
        const int s = blockIdx.x * (LOCAL_THREADS / 32) + (threadIdx.x >> 5);
        const int32_t st = s < ns ? strips[s] : 0;   // static: read before the wait
        pdl_wait();
        if (s < ns) rb_strip<float, SR, true>(v, out, st);   // uniform over the warp
        return;
    }
    // the block copies its index lists before waiting for the previous launch
    local_body<float, 2, EPT>(J, v.u, out, (int)blockIdx.x - nsc, 1, lambda, true, true);
}

template <int SR, int EPT>
void launch_relax2d_as(dim3 grid, size_t smem, cudaStream_t s, const LevelView<float> &v, float *out,
                       const DevGeom &g, int nsc, const LocalView<float> &J, int lambda) {
    static size_t opted = 0;   // dynamic shared memory opted in for this instance
    if (smem > opted) {
        cudaFuncSetAttribute(k_relax2d<SR, EPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        opted = smem;
    }
    pdl_launch(k_relax2d<SR, EPT>, grid, dim3(LOCAL_THREADS), smem, s, v, out, g.strips, g.nstrips, nsc, J, lambda);
}

void launch_relax2d(const LevelView<float> &v, float *out, const DevGeom &g, const LocalView<float> &J, int lambda,
                    cudaStream_t s) {
    g_launches++;
    const int per = LOCAL_THREADS / 32;
    const int nsc = (g.nstrips + per - 1) / per;
    const size_t smem = local_smem_bytes(J, 2, true);
    const dim3 grid((unsigned)(nsc + J.ncomp));
    if (J.max_colour <= LOCAL_THREADS) {
        if (g.strip_rows == 32) launch_relax2d_as<32, 1>(grid, smem, s, v, out, g, nsc, J, lambda);
        else if (g.strip_rows == 16) launch_relax2d_as<16, 1>(grid, smem, s, v, out, g, nsc, J, lambda);
        else launch_relax2d_as<8, 1>(grid, smem, s, v, out, g, nsc, J, lambda);
    } else {
        if (g.strip_rows == 32) launch_relax2d_as<32, LOCAL_EPT>(grid, smem, s, v, out, g, nsc, J, lambda);
        else if (g.strip_rows == 16) launch_relax2d_as<16, LOCAL_EPT>(grid, smem, s, v, out, g, nsc, J, lambda);
        else launch_relax2d_as<8, LOCAL_EPT>(grid, smem, s, v, out, g, nsc, J, lambda);
    }
}

// both colours in one pass over the active 2D strips: 4 warps a CTA, one strip a warp
// (INTERIOR_ONLY: the boundary blocks, launched beside, store the band and ghosts)
template <typename T, int SR, bool INTERIOR_ONLY = false>
__global__ void __launch_bounds__(128) k_rb_strip(LevelView<T> v, T *__restrict__ out,
                                                  const int32_t *__restrict__ strips, int ns) {
    pdl_wait();
    const int s = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (s < ns) rb_strip<T, SR, INTERIOR_ONLY>(v, out, strips[s]);   // uniform over the warp
}

template <int SR>
static void launch_strips_interior(const LevelView<float> &v, float *out, const DevGeom &g, cudaStream_t s) {
    pdl_launch(k_rb_strip<float, SR, true>, dim3((unsigned)((g.nstrips + 3) / 4)), dim3(128), 0, s, v, out, g.strips,
               g.nstrips);
}

void launch_relax2d_split(const LevelView<float> &v, float *out, const DevGeom &g, const LocalView<float> &J,
                          int lambda, cudaStream_t s, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join) {
    // the boundary blocks (k_relax2d without strips) on the side stream, the
    // strips (interior nodes off the band) on the main one: both read v.u and
    // store disjoint nodes of out, as the merged launch does
    g_launches += 2;
    cudaEventRecord(fork, s);
    cudaStreamWaitEvent(side, fork, 0);
    const size_t smem = local_smem_bytes(J, 2, true);
    const dim3 grid((unsigned)J.ncomp);
    if (J.max_colour <= LOCAL_THREADS) {
        if (g.strip_rows == 32) launch_relax2d_as<32, 1>(grid, smem, side, v, out, g, 0, J, lambda);
        else if (g.strip_rows == 16) launch_relax2d_as<16, 1>(grid, smem, side, v, out, g, 0, J, lambda);
        else launch_relax2d_as<8, 1>(grid, smem, side, v, out, g, 0, J, lambda);
    } else {
        if (g.strip_rows == 32) launch_relax2d_as<32, LOCAL_EPT>(grid, smem, side, v, out, g, 0, J, lambda);
        else if (g.strip_rows == 16) launch_relax2d_as<16, LOCAL_EPT>(grid, smem, side, v, out, g, 0, J, lambda);
        else launch_relax2d_as<8, LOCAL_EPT>(grid, smem, side, v, out, g, 0, J, lambda);
    }
    if (g.strip_rows == 32) launch_strips_interior<32>(v, out, g, s);
    else if (g.strip_rows == 16) launch_strips_interior<16>(v, out, g, s);
    else launch_strips_interior<8>(v, out, g, s);
    cudaEventRecord(join, side);
    cudaStreamWaitEvent(s, join, 0);
}

template <typename T>
void launch_rb_strip(const LevelView<T> &v, T *out, const DevGeom &g, cudaStream_t s) {
    if (g.nstrips <= 0) return;
    g_launches++;
    const dim3 grid((unsigned)((g.nstrips + 3) / 4));
    if (g.strip_rows == 32) pdl_launch(k_rb_strip<T, 32>, grid, dim3(128), 0, s, v, out, g.strips, g.nstrips);
    else if (g.strip_rows == 16) pdl_launch(k_rb_strip<T, 16>, grid, dim3(128), 0, s, v, out, g.strips, g.nstrips);
    else pdl_launch(k_rb_strip<T, 8>, grid, dim3(128), 0, s, v, out, g.strips, g.nstrips);
}

template <typename T>
void launch_rb_fused2d(const LevelView<T> &v, T *out, const int32_t *tiles, int ntiles, cudaStream_t s) {
    if (ntiles <= 0) return;
    g_launches++;
    pdl_launch(k_rb_fused2d<T, TILE_R, TILE_C>, dim3(ntiles), dim3(256), 0, s, v, out, tiles);
}

void launch_mask_types(int dim, int n, double h, const double *origin, int step, int n_l, const double *B,
                       const int32_t *gnode, int ng, const uint8_t *mask, uint8_t *types, cudaStream_t s) {
    if (ng <= 0) return;
    g_launches++;
    k_mask_types<<<blocks_for(ng), kThreads, 0, s>>>(dim, n, h, origin[0], origin[1], origin[2], step, n_l, B, gnode,
                                                     ng, mask, types);
}

template <typename T>
bool launch_boundary3d(const LevelView<T> &v, BoundaryProgram3 P, int phantom, cudaStream_t s) {
    // CTAs resident at once (per device; the first launch asks the runtime)
    static int dev_seen = -1, resident = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (dev != dev_seen) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_boundary3d<T>, kThreads, 0) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        resident = per_sm * sms;
        dev_seen = dev;
    }
    if (resident <= 0) return false;
    // enough CTAs for the largest phase at four entries a thread, at most
    // one wave: fewer CTAs make each barrier cheaper
    const int64_t work = std::max<int64_t>({(int64_t)v.ng, P.nred, P.nblack, P.nzred, P.nzblack, 1});
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(resident, (work + 4 * kThreads - 1) /
                                                                                       (4 * kThreads)));
    P.nbar = nb + (unsigned)std::max(phantom, 0);
    g_launches++;
    // a plain launch: it starts after the previous kernel of the stream has
    // finished and no CTA of another kernel of this stream runs beside it
    k_boundary3d<T><<<nb, kThreads, 0, s>>>(v, P);
    return true;
}

template <typename T>
bool launch_boundary3d_cluster(const LevelView<T> &v, const BoundaryProgram3 &P, cudaStream_t s) {
    static int opted_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (dev != opted_dev) {   // cluster size 16 is beyond the portable 8
        if (cudaFuncSetAttribute(k_boundary3d_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        opted_dev = dev;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(BC_SIZE);
    cfg.blockDim = dim3(BC_THREADS);
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = BC_SIZE;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    if (cudaLaunchKernelEx(&cfg, k_boundary3d_cluster<T>, v, P) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    g_launches++;
    return true;
}

template <typename T>
void launch_rb_stream3d(const LevelView<T> &v, T *out, const DevGeom &g, cudaStream_t s) {
    if (g.nsr <= 0) return;
    g_launches++;
    pdl_launch(k_rb_stream3d<T>, dim3((unsigned)g.nsr), dim3((SR_TY + 4) * 32), 0, s, v, out,
               reinterpret_cast<const int2 *>(g.sr));
}

template <int C>
static void launch_span3d(const LevelView<float> &v, float *out, const DevGeom &g, cudaStream_t s) {
    constexpr size_t smem = (size_t)(SP_SEG + 4) * SP_NW * sizeof(int2) + (size_t)4 * SP_NW * C * 32 * sizeof(float);
    static bool opted = false;
    if (!opted) {
        cudaFuncSetAttribute(k_rb_span3d<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        opted = true;
    }
    pdl_launch(k_rb_span3d<C>, dim3((unsigned)g.nsp), dim3(SP_NW * 32), smem, s, v, out,
               reinterpret_cast<const int4 *>(g.sp), reinterpret_cast<const int2 *>(g.sp_rows));
}

bool launch_rb_span3d(const LevelView<float> &v, float *out, const DevGeom &g, cudaStream_t s) {
    if (g.nsp <= 0) return false;
    switch (g.sp_cols) {
    case 2: launch_span3d<2>(v, out, g, s); break;
    case 3: launch_span3d<3>(v, out, g, s); break;
    case 4: launch_span3d<4>(v, out, g, s); break;
    case 5: launch_span3d<5>(v, out, g, s); break;
    default: return false;
    }
    g_launches++;
    return true;
}

template <typename T>
bool launch_rb_rows(const LevelView<T> &v, const DevGeom &g, cudaStream_t s) {
    if (g.nspl <= 0) return false;
    constexpr int G = 8;   // segments a warp at once (measured at 513^3: 4 -> 60.7 us a sweep, 8 -> 58.5 us)
    static int resident = 0;   // the persistent grid: CTAs resident on the device
    if (resident == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rb_rows<T, G>, 256, 0);
        resident = std::max(1, sms * std::max(per, 1));
    }
    const int64_t need = ((int64_t)(g.nspl + G - 1) / G * 32 + 255) / 256;
    const unsigned blocks = (unsigned)std::min<int64_t>(need, resident);
    const int2 *segs = reinterpret_cast<const int2 *>(g.sp_list);
    for (int colour = 0; colour < 2; colour++)
        pdl_launch(k_rb_rows<T, G>, dim3(blocks), dim3(256), 0, s, v, segs, g.nspl, colour);
    g_launches += 2;
    return true;
}

template <typename T>
void launch_rb_zmarch(const LevelView<T> &v, T *out, const DevGeom &g, cudaStream_t s) {
    if (g.nzm <= 0) return;
    constexpr size_t smem = zmarch_smem_bytes<T>();
    static bool opted = false;
    if (!opted) {
        cudaFuncSetAttribute(k_rb_zmarch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        opted = true;
    }
    g_launches++;
    pdl_launch(k_rb_zmarch<T>, dim3((unsigned)g.nzm), dim3(ZM_THREADS), smem, s, v, out,
               reinterpret_cast<const int2 *>(g.zm), (const int32_t *)g.zm_moff, (const uint32_t *)g.zm_mask);
}

template <typename T>
void launch_rb_list(const LevelView<T> &v, int dim, const int32_t *list, int cnt, cudaStream_t s) {
    if (cnt <= 0) return;
    g_launches++;
    if (cnt >= kListBig) {
        const unsigned nb = blocks_for(((int64_t)cnt + 3) / 4);
        if (dim == 2) pdl_launch(k_rb_list<T, 2, 4>, dim3(nb), dim3(kThreads), 0, s, v, list, cnt);
        else pdl_launch(k_rb_list<T, 3, 4>, dim3(nb), dim3(kThreads), 0, s, v, list, cnt);
    } else {
        if (dim == 2) pdl_launch(k_rb_list<T, 2, 1>, dim3(blocks_for(cnt)), dim3(kThreads), 0, s, v, list, cnt);
        else pdl_launch(k_rb_list<T, 3, 1>, dim3(blocks_for(cnt)), dim3(kThreads), 0, s, v, list, cnt);
    }
}

template <typename T>
void launch_ghost_relax(const LevelView<T> &v, int dim, cudaStream_t s) {
    if (v.ng <= 0) return;
    g_launches += 2;
    if (dim == 2) pdl_launch(k_ghost_new<T, 9>, dim3(blocks_for(v.ng)), dim3(kThreads), 0, s, v);
    else pdl_launch(k_ghost_new<T, 27>, dim3(blocks_for(v.ng)), dim3(kThreads), 0, s, v);
    pdl_launch(k_ghost_store<T>, dim3(blocks_for(v.ng)), dim3(kThreads), 0, s, v);
}

template <typename T>
void launch_rb_list_store(const LevelView<T> &v, const int32_t *list, const int32_t *src, int cnt,
                          const int32_t *glist, int gcnt, cudaStream_t s) {
    if (cnt + gcnt <= 0) return;
    g_launches++;
    if ((int64_t)cnt + gcnt >= kListBig)
        pdl_launch(k_rb_list_store<T, 4>, dim3(blocks_for(((int64_t)cnt + gcnt + 3) / 4)), dim3(kThreads), 0, s, v,
                   list, src, cnt, glist, gcnt);
    else
        pdl_launch(k_rb_list_store<T, 1>, dim3(blocks_for((int64_t)cnt + gcnt)), dim3(kThreads), 0, s, v, list, src,
                   cnt, glist, gcnt);
}

// the two halves of a Jacobi ghost sweep as separate launches (3D: the store
// merged into the next red sweep, see k_rb_list_store)
template <typename T>
void launch_ghost_new(const LevelView<T> &v, const int32_t *list, int cnt, cudaStream_t s) {
    if (cnt <= 0) return;
    g_launches++;
    if (list) pdl_launch(k_ghost_new_list<T, 27>, dim3(blocks_for(cnt)), dim3(kThreads), 0, s, v, list, cnt);
    else pdl_launch(k_ghost_new<T, 27>, dim3(blocks_for(cnt)), dim3(kThreads), 0, s, v);
}

template <typename T>
void launch_ghost_store(const LevelView<T> &v, const int32_t *list, int cnt, cudaStream_t s) {
    if (cnt <= 0) return;
    g_launches++;
    if (list) pdl_launch(k_ghost_store_list<T>, dim3(blocks_for(cnt)), dim3(kThreads), 0, s, v, list, cnt);
    else pdl_launch(k_ghost_store<T>, dim3(blocks_for(cnt)), dim3(kThreads), 0, s, v);
}

template <typename T>
void launch_ghost_relax_list(const LevelView<T> &v, int dim, const int32_t *list, int cnt, cudaStream_t s) {
    if (cnt <= 0) return;
    g_launches += 2;
    if (dim == 2) pdl_launch(k_ghost_new_list<T, 9>, dim3(blocks_for(cnt)), dim3(kThreads), 0, s, v, list, cnt);
    else pdl_launch(k_ghost_new_list<T, 27>, dim3(blocks_for(cnt)), dim3(kThreads), 0, s, v, list, cnt);
    pdl_launch(k_ghost_store_list<T>, dim3(blocks_for(cnt)), dim3(kThreads), 0, s, v, list, cnt);
}

template <typename T>
void launch_defect(const LevelView<T> &v, int dim, bool zero_rest, unsigned long long *norm, cudaStream_t s) {
    g_launches += v.ng > 0 ? 2 : 1;
    const unsigned nb = std::min(blocks_for(level_threads(v, !zero_rest)), kNormBlocks);
    if (dim == 3 && !zero_rest && v.nsegs > 0) {   // inside nodes over the row segments
        constexpr int G = 4;
        static unsigned resident = 0;
        pdl_launch(k_defect_rows<T, G, false>, dim3(segment_blocks(k_defect_rows<T, G, false>, v.nsegs, G, resident)),
                   dim3(256), 0, s, v, norm, (float *)nullptr, (float *)nullptr);
    } else if (dim == 2) pdl_launch(k_defect_interior<T, 2>, dim3(nb), dim3(kThreads), 0, s, v, zero_rest, norm);
    else pdl_launch(k_defect_interior<T, 3>, dim3(nb), dim3(kThreads), 0, s, v, zero_rest, norm);
    if (v.ng > 0) {
        if (dim == 2) pdl_launch(k_defect_ghost<T, 9>, dim3(blocks_for(v.ng)), dim3(kThreads), 0, s, v, norm);
        else pdl_launch(k_defect_ghost<T, 27>, dim3(blocks_for(v.ng)), dim3(kThreads), 0, s, v, norm);
    }
}

template <typename T>
void launch_extend(T *r, const DevGeom &g, const T *ew, cudaStream_t s) {
    for (size_t w = 1; w < g.wave.size(); w++) {
        const int b = g.wave[w - 1], e = g.wave[w];
        if (e > b) g_launches++;
        if (e > b) pdl_launch(k_extend<T>, dim3(blocks_for(e - b)), dim3(kThreads), 0, s, r, g.enode, g.ecnt, g.esrc, ew, g.ne, b, e);
    }
}

template <typename T>
void launch_restrict_interior(const LevelView<T> &F, const LevelView<T> &C, int dim, T *fc, cudaStream_t s) {
    g_launches++;
    if (dim == 2) pdl_launch(k_restrict_interior<T, 2>, dim3(blocks_for(C.nn)), dim3(kThreads), 0, s, F, C, fc);
    else pdl_launch(k_restrict_interior<T, 3>, dim3(blocks_for(C.nn)), dim3(kThreads), 0, s, F, C, fc);
}

template <typename T>
void launch_restrict(const LevelView<T> &F, const LevelView<T> &C, int dim, T *fc, T *gc, cudaStream_t s) {
    g_launches += C.ng > 0 ? 2 : 1;
    if (dim == 2) {
        pdl_launch(k_restrict_interior<T, 2>, dim3(blocks_for(C.nn)), dim3(kThreads), 0, s, F, C, fc);
        if (C.ng > 0) pdl_launch(k_restrict_ghost<T, 2>, dim3(blocks_for(C.ng)), dim3(kThreads), 0, s, F, C, gc);
    } else {
        pdl_launch(k_restrict_interior<T, 3>, dim3(blocks_for(C.nn)), dim3(kThreads), 0, s, F, C, fc);
        if (C.ng > 0) pdl_launch(k_restrict_ghost<T, 3>, dim3(blocks_for(C.ng)), dim3(kThreads), 0, s, F, C, gc);
    }
}

template <typename T>
void launch_descend(const LevelView<T> &F, const LevelView<T> &C, const DevGeom &gf, const T *gt_val, T *fc, T *gc,
                    T *uc, cudaStream_t s, const T *pt_w) {
    const bool warp_rows = sizeof(T) == 4 && gf.dim == 2;   // 2D FP32: a warp per coarse ghost row
    const int64_t n = gf.dim == 3 ? level_threads(C, true) : warp_rows ? C.nn + 32 * (int64_t)C.ng
                                                                      : std::max<int64_t>(C.nn, C.ng);
    if (gf.dim == 3 && F.nsegs > 0) {
        // 3D with row segments: one defect pass first (inside nodes over the
        // segments, then the ghosts), so that each fine defect is computed
        // once rather than once per coarse node whose 27-node neighbourhood
        // holds it (27/8 times on average); the same values as on the spot
        constexpr int G = 4;
        static unsigned resident = 0;
        const unsigned blocks = segment_blocks(k_defect_rows<T, G, false>, F.nsegs, G, resident);
        g_launches++;
        pdl_launch(k_defect_rows<T, G, false>, dim3(blocks), dim3(256), 0, s, F, (unsigned long long *)nullptr,
                   (float *)nullptr, (float *)nullptr);
        if (F.ng > 0) {
            g_launches++;
            pdl_launch(k_defect_ghost<T, 27>, dim3(blocks_for(F.ng)), dim3(kThreads), 0, s, F,
                       (unsigned long long *)nullptr);
        }
        if (C.ng > 0) {
            g_launches++;
            pdl_launch(k_ghost_rows<T, true>, dim3(blocks_for(32 * (int64_t)C.ng)), dim3(kThreads), 0, s,
                       (const T *)F.r, F.gnode, gc, gf.gt_ptr, gf.gt_col, gt_val, C.ng);
        }
        // the coarse nodes of full weighting first, then those whose fine
        // neighbourhood is partly outside
        g_launches++;
        pdl_launch(k_descend<T, 3, true>, dim3(blocks_for(n)), dim3(kThreads), 0, s, F, C, fc, gc, uc, gf.gt_ptr,
                   gf.gt_col, gt_val, gf.npartial > 0 && pt_w != nullptr);
        if (gf.npartial > 0 && pt_w) {
            g_launches++;
            pdl_launch(k_descend_partial<T>, dim3(blocks_for(gf.npartial)), dim3(kThreads), 0, s, F, C, fc,
                       (const int32_t *)gf.partial_coarse, pt_w, gf.npartial);
        }
        return;
    }
    constexpr bool from_r = sizeof(T) == 8;   // FP64: one defect pass first (see descend_item)
    if (from_r) launch_defect<T>(F, gf.dim, false, nullptr, s);
    if (gf.dim == 3 && C.ng > 0) {
        // 3D: the fine ghost defects once (FP32: into F.gtmp; FP64: the
        // defect pass above), then the coarse ghost rows a warp each
        if (!from_r && F.ng > 0) {
            g_launches++;
            pdl_launch(k_ghost_defects<T, 27>, dim3(blocks_for(F.ng)), dim3(kThreads), 0, s, F);
        }
        g_launches++;
        pdl_launch(k_ghost_rows<T, from_r>, dim3(blocks_for(32 * (int64_t)C.ng)), dim3(kThreads), 0, s,
                   (const T *)(from_r ? F.r : F.gtmp), F.gnode, gc, gf.gt_ptr, gf.gt_col, gt_val, C.ng);
    }
    g_launches++;
    if (gf.dim == 2)
        pdl_launch(k_descend<T, 2, from_r>, dim3(blocks_for(n)), dim3(kThreads), 0, s, F, C, fc, gc, uc, gf.gt_ptr, gf.gt_col, gt_val,
                   false);
    else
        pdl_launch(k_descend<T, 3, from_r>, dim3(blocks_for(n)), dim3(kThreads), 0, s, F, C, fc, gc, uc, gf.gt_ptr, gf.gt_col, gt_val,
                   false);
}

template <typename T>
void launch_ghost_transfer(const T *rf, const int32_t *fgnode, const int32_t *ptr, const int32_t *col, const T *val,
                           T *gc, int ngc, cudaStream_t s) {
    if (ngc <= 0) return;
    g_launches++;
    pdl_launch(k_ghost_transfer<T>, dim3(blocks_for(ngc)), dim3(kThreads), 0, s, rf, fgnode, ptr, col, val, gc, ngc);
}

template <typename T>
void launch_prolong(const LevelView<T> &F, const LevelView<T> &C, int dim, const T *e, T *out, bool add,
                    cudaStream_t s) {
    g_launches++;
    if (dim == 3 && add && F.nsegs > 0) {   // inside nodes over the row segments, then the ghosts
        constexpr int G = 1;
        static unsigned resident = 0;
        pdl_launch(k_prolong_rows<T, G>, dim3(segment_blocks(k_prolong_rows<T, G>, F.nsegs, G, resident)), dim3(256),
                   0, s, F, C, e, out);
        return;
    }
    const int64_t nt = level_threads(F, add);
    if (dim == 2) pdl_launch(k_prolong<T, 2>, dim3(blocks_for(nt)), dim3(kThreads), 0, s, F, C, e, out, add);
    else pdl_launch(k_prolong<T, 3>, dim3(blocks_for(nt)), dim3(kThreads), 0, s, F, C, e, out, add);
}

template <typename T>
void launch_coarse_solve(const LevelView<T> &v, const DevGeom &g, const T *Ainv, cudaStream_t s) {
    const int m = g.nunk;
    if (m <= 0) return;
    g_launches++;
    const int threads = 512;
    const unsigned blocks = (unsigned)std::min(1024, (m + 15) / 16);
    pdl_launch(k_coarse_solve<T>, dim3(blocks), dim3(threads), (size_t)m * sizeof(T), s, v, g.unk_node, g.unk_ghost, Ainv, m);
}

// defects of the junction-solve rows; with a pending boundary-block
// write-back (J.wb set) the same launch also copies the write-back nodes into
// u, the defects reading those nodes from the write-back grid
template <typename T, int D, bool WB>
__global__ void __launch_bounds__(kThreads) k_js_defect(LevelView<T> v, const int32_t *__restrict__ node,
                                                        const int32_t *__restrict__ ghost,
                                                        const int32_t *__restrict__ rpos, T *__restrict__ r, int n,
                                                        LocalView<T> J) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (WB) {
        pdl_wait();
        local_copyback<T>(J, v.u, k);
        if (k < n) r[rpos[k]] = dev::js_defect<T, D, WB>(v, node[k], ghost[k], J.wb);
        return;
    }
    // the row's static data (node, ghost stencil and weights) is read before
    // waiting for the relaxation, u, f and g after it
    if (sizeof(T) == 4) pdl_trigger();
    if (k >= n) return;
    const int32_t p = node[k], q = ghost[k], rp = rpos[k];
    if (q >= 0) {
        constexpr int K = D == 2 ? 9 : 27;
        int32_t st[K];
        T w[K];
#pragma unroll
        for (int a = 0; a < K; a++) {
            st[a] = v.gstn[(int64_t)a * v.ng + q];
            w[a] = v.gw[(int64_t)a * v.ng + q];
        }
        pdl_wait();
        T s = 0;
#pragma unroll
        for (int a = 0; a < K; a++) s += w[a] * v.u[st[a]];   // as js_defect
        r[rp] = v.gg[q] - s;
    } else {
        pdl_wait();
        r[rp] = dev::js_defect<T, D, false>(v, p, -1);
    }
}

// R rows a warp, 8 warps a CTA: R = 4 amortises the per-CTA address chain
// over 4 rows once the launch fills the GPU several times over; a small
// launch (a single domain: about a thousand rows a level) keeps one row a
// warp so that it spreads over more SMs
template <typename T, int R>
__global__ void __launch_bounds__(256)
    k_js_apply(T *__restrict__ u, const int32_t *__restrict__ node, const int32_t *__restrict__ comp,
               const int32_t *__restrict__ off, const int64_t *__restrict__ aoff, const int32_t *__restrict__ roff,
               const T *__restrict__ inv, const T *__restrict__ r, int n) {
    if (sizeof(T) == 4) pdl_trigger();
    const int k0 = blockIdx.x * 8 * R + (threadIdx.x >> 5) * R;
    if (R == 1) {   // one row a warp: its part of the inverse is loaded before the wait
        if (k0 < n) dev::js_apply_row_early<T, 8>(u, node, comp, off, aoff, roff, inv, r, k0, threadIdx.x & 31);
        else pdl_wait();
        return;
    }
    pdl_wait();
    dev::js_apply_span<T, R>(u, node, comp, off, aoff, roff, inv, r, k0, min(k0 + R, n), threadIdx.x & 31);
}

// SMs of the current device (queried once)
int num_sms() {
    static int count = 0;
    if (count <= 0) {
        int d = 0, m = 0;
        if (cudaGetDevice(&d) == cudaSuccess && cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, d) ==
                                                     cudaSuccess)
            count = m;
    }
    return count > 0 ? count : 1;
}

template <typename T>
void launch_junction_solve(const LevelView<T> &v, const DevGeom &g, const T *inv, T *r, cudaStream_t s,
                           const LocalView<T> *pending) {
    const int n = g.js_n;
    if (n <= 0) {
        if (pending) launch_local_copyback<T>(*pending, s);
        return;
    }
    g_launches += 2;
    if (pending)   // 2D boundary blocks only
        pdl_launch(k_js_defect<T, 2, true>, dim3(blocks_for(std::max(n, pending->nwb))), dim3(kThreads), 0, s, v,
                   g.js_node, g.js_ghost, g.js_rpos, r, n, *pending);
    else if (g.dim == 2)
        pdl_launch(k_js_defect<T, 2, false>, dim3(blocks_for(n)), dim3(kThreads), 0, s, v, g.js_node, g.js_ghost,
                   g.js_rpos, r, n, LocalView<T>{});
    else
        pdl_launch(k_js_defect<T, 3, false>, dim3(blocks_for(n)), dim3(kThreads), 0, s, v, g.js_node, g.js_ghost,
                   g.js_rpos, r, n, LocalView<T>{});
    if (n >= 8 * 4 * 4 * num_sms())   // at least four CTAs of 4-row warps an SM
        pdl_launch(k_js_apply<T, 4>, dim3((unsigned)((n + 31) / 32)), dim3(256), 0, s, v.u, g.js_node, g.js_comp,
                   g.js_off, g.js_aoff, g.js_roff, inv, r, n);
    else
        pdl_launch(k_js_apply<T, 1>, dim3((unsigned)((n + 7) / 8)), dim3(256), 0, s, v.u, g.js_node, g.js_comp,
                   g.js_off, g.js_aoff, g.js_roff, inv, r, n);
}

template <typename T>
size_t local_smem_bytes(const LocalView<T> &J, int dim, bool pre) {
    const int K = dim == 2 ? 9 : 27;
    size_t b = sizeof(T) * ((size_t)J.max_nodes + (size_t)(K + 3) * J.max_gh + J.max_int) +
               sizeof(int) * ((size_t)(K + 2) * J.max_gh + J.max_nodes + J.max_int);
    if (pre) b = (b + sizeof(T) - 1) / sizeof(T) * sizeof(T) + (sizeof(T) + sizeof(int) * (2 + 2 * dim)) * (size_t)J.max_pre;
    return b;
}

bool local_fits_registers(int max_int_per_colour) { return max_int_per_colour <= LOCAL_THREADS * LOCAL_EPT; }

template <typename T>
__global__ void __launch_bounds__(256) k_local_copyback(LocalView<T> J) {
    pdl_wait();
    local_copyback<T>(J, J.u, blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
void launch_local_copyback(const LocalView<T> &J, cudaStream_t s) {
    if (!J.wb || J.nwb <= 0) return;
    g_launches++;
    pdl_launch(k_local_copyback<T>, dim3(blocks_for(J.nwb)), dim3(256), 0, s, J);
}

template <typename T>
void launch_local(const LocalView<T> &J, int dim, int lead_ghost, int reps, cudaStream_t s) {
    if (J.ncomp <= 0 || (reps <= 0 && !lead_ghost)) return;
    g_launches++;
    const size_t smem = local_smem_bytes(J, dim);
    if (dim == 2) pdl_launch(k_local<T, 2>, dim3(J.ncomp), dim3(LOCAL_THREADS), smem, s, J, lead_ghost, reps);
    else pdl_launch(k_local<T, 3>, dim3(J.ncomp), dim3(LOCAL_THREADS), smem, s, J, lead_ghost, reps);
}

template <typename T>
void local_prepare(int dim, size_t smem) {
    // opt in to large dynamic shared memory once per precision / dimension
    if (dim == 2) cudaFuncSetAttribute(k_local<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else cudaFuncSetAttribute(k_local<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T>
void launch_mask_unknowns(const uint8_t *type, T *u, int64_t nn, cudaStream_t s) {
    g_launches++;
    pdl_launch(k_mask_unknowns<T>, dim3(blocks_for(nn)), dim3(kThreads), 0, s, type, u, nn);
}

void launch_defect_mixed(const LevelView<double> &v, int dim, unsigned long long *norm, float *f32, float *g32,
                         float *e32, cudaStream_t s) {
    g_launches += v.ng > 0 ? 2 : 1;
    const unsigned nb = std::min(blocks_for(level_threads(v, true)), kNormBlocks);
    // 3D with row segments: the inside nodes over the segments, e32 = 0 at
    // the ghosts by the ghost launch; the other nodes of f32 and e32 are 0
    // from the start and nothing writes them
    const bool rows = dim == 3 && v.nsegs > 0;
    if (rows) {
        constexpr int G = 2;
        static unsigned resident = 0;
        pdl_launch(k_defect_rows<double, G, true>,
                   dim3(segment_blocks(k_defect_rows<double, G, true>, v.nsegs, G, resident)), dim3(256), 0, s, v,
                   norm, f32, e32);
    } else if (dim == 2) pdl_launch(k_defect_interior_mixed<2>, dim3(nb), dim3(kThreads), 0, s, v, norm, f32, e32);
    else pdl_launch(k_defect_interior_mixed<3>, dim3(nb), dim3(kThreads), 0, s, v, norm, f32, e32);
    float *ge = rows ? e32 : nullptr;
    if (v.ng > 0) {
        if (dim == 2) pdl_launch(k_defect_ghost_mixed<9>, dim3(blocks_for(v.ng)), dim3(kThreads), 0, s, v, norm, g32, ge);
        else pdl_launch(k_defect_ghost_mixed<27>, dim3(blocks_for(v.ng)), dim3(kThreads), 0, s, v, norm, g32, ge);
    }
}

void launch_add_correction(const DevGeom &g, double *u64, const float *e32, cudaStream_t s) {
    g_launches++;
    LevelView<double> v{};
    v.n = g.n;
    v.nn = g.nn;
    v.type = g.type;
    v.chunks = g.chunks;
    v.clen = g.chunk_len;
    v.nchunks = g.nchunks;
    if (g.dim == 3 && g.nspl > 0) {   // inside nodes over the row segments, then the ghosts
        constexpr int G = 4;
        static unsigned resident = 0;
        v.segs = reinterpret_cast<const int2 *>(g.sp_list);
        v.nsegs = g.nspl;
        v.ng = g.ng;
        v.gnode = g.gnode;
        pdl_launch(k_add_rows<G>, dim3(segment_blocks(k_add_rows<G>, v.nsegs, G, resident)), dim3(256), 0, s, v, u64,
                   e32);
        return;
    }
    pdl_launch(k_add_correction, dim3(blocks_for(level_threads(v, true))), dim3(kThreads), 0, s, v, u64, e32);
}

#define GCMG_INSTANTIATE(T)                                                                              \
    template void launch_rb<T>(const LevelView<T> &, int, int, cudaStream_t);                            \
    template void launch_rb_list<T>(const LevelView<T> &, int, const int32_t *, int, cudaStream_t);     \
    template void launch_rb_fused2d<T>(const LevelView<T> &, T *, const int32_t *, int, cudaStream_t);  \
    template void launch_rb_strip<T>(const LevelView<T> &, T *, const DevGeom &, cudaStream_t);           \
    template void launch_ghost_relax<T>(const LevelView<T> &, int, cudaStream_t);                         \
    template void launch_ghost_relax_list<T>(const LevelView<T> &, int, const int32_t *, int, cudaStream_t); \
    template void launch_rb_list_store<T>(const LevelView<T> &, const int32_t *, const int32_t *, int,      \
                                          const int32_t *, int, cudaStream_t);                               \
    template void launch_ghost_new<T>(const LevelView<T> &, const int32_t *, int, cudaStream_t);          \
    template void launch_ghost_store<T>(const LevelView<T> &, const int32_t *, int, cudaStream_t);        \
    template void launch_defect<T>(const LevelView<T> &, int, bool, unsigned long long *, cudaStream_t); \
    template void launch_extend<T>(T *, const DevGeom &, const T *, cudaStream_t);                        \
    template void launch_restrict<T>(const LevelView<T> &, const LevelView<T> &, int, T *, T *, cudaStream_t); \
    template void launch_restrict_interior<T>(const LevelView<T> &, const LevelView<T> &, int, T *, cudaStream_t); \
    template void launch_ghost_transfer<T>(const T *, const int32_t *, const int32_t *, const int32_t *, const T *, \
                                           T *, int, cudaStream_t);                                              \
    template void launch_prolong<T>(const LevelView<T> &, const LevelView<T> &, int, const T *, T *, bool,  \
                                    cudaStream_t);                                                       \
    template void launch_coarse_solve<T>(const LevelView<T> &, const DevGeom &, const T *, cudaStream_t); \
    template void launch_junction_solve<T>(const LevelView<T> &, const DevGeom &, const T *, T *, cudaStream_t, \
                                           const LocalView<T> *);                                                \
    template void launch_descend<T>(const LevelView<T> &, const LevelView<T> &, const DevGeom &, const T *, T *, T *, \
                                    T *, cudaStream_t, const T *);                                                 \
    template void launch_mask_unknowns<T>(const uint8_t *, T *, int64_t, cudaStream_t);            \
    template void launch_rb_zmarch<T>(const LevelView<T> &, T *, const DevGeom &, cudaStream_t);    \
    template void launch_rb_stream3d<T>(const LevelView<T> &, T *, const DevGeom &, cudaStream_t);  \
    template bool launch_rb_rows<T>(const LevelView<T> &, const DevGeom &, cudaStream_t);           \
    template bool launch_boundary3d<T>(const LevelView<T> &, BoundaryProgram3, int, cudaStream_t);  \
    template bool launch_boundary3d_cluster<T>(const LevelView<T> &, const BoundaryProgram3 &, cudaStream_t); \
    template size_t local_smem_bytes<T>(const LocalView<T> &, int, bool);                                 \
    template void launch_local<T>(const LocalView<T> &, int, int, int, cudaStream_t);               \
    template void launch_local_copyback<T>(const LocalView<T> &, cudaStream_t);                      \
    template void local_prepare<T>(int, size_t);

GCMG_INSTANTIATE(float)
GCMG_INSTANTIATE(double)

}  // namespace gcmg
