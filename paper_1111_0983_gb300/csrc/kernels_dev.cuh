// Device-side bodies of the per-level kernels, shared by the single-domain
// kernels (kernels.cu) and the batched multi-domain kernels (batch.cu).  Each
// body does the work of one thread (or one CTA) for one item -- a node, a
// ghost, a tile or a program component -- given that level's view.
#pragma once

#include <cuda_runtime.h>

#include "exact_lap.h"
#include "gcmg_internal.h"

namespace gcmg {
namespace dev {

constexpr int LOCAL_THREADS = 512;
constexpr int LOCAL_EPT = 4;     // inside entries per thread and colour in local programs (at most)

// max-norm reduction on the bit pattern of a non-negative double (monotone
// for non-negative IEEE values); NaN is folded into +Inf so that it is seen.
// waits for the preceding kernel of the stream (programmatic dependent launch;
// a no-op when the kernel was launched without it).  No kernel triggers its
// dependents early: measured, a 1025^2 solve went from 4.84 to 5.13 ms when
// every kernel did, the waiting CTAs taking SM slots from the running grid.
// asynchronous global -> shared copy of one word (4 or 8 bytes): no register
// holds it and the issuing thread does not wait for it
template <typename W>
__device__ __forceinline__ void cp_async(W *smem, const W *gmem) {
    static_assert(sizeof(W) == 4 || sizeof(W) == 8, "4- or 8-byte words");
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(W) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem) : "memory");
}
// waits until this thread's asynchronous copies have landed (and are visible to it)
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// start of the pre-sweep lists in a local program's shared memory: the end
// of the other lists rounded up to a word of T
template <typename T>
__device__ __forceinline__ void *local_pre_base(int *end) {
    return (void *)(((uintptr_t)end + sizeof(T) - 1) & ~(uintptr_t)(sizeof(T) - 1));
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// lets the launch that depends on this grid start its CTAs now: they run
// whatever precedes their pdl_wait (reads of data no launch writes) while
// this grid works
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void atomic_max_abs(unsigned long long *bits, double v) {
    v = fabs(v);
    if (v != v) v = __longlong_as_double(0x7ff0000000000000ll);
    atomicMax(bits, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// block-wide max of |v| (every thread of the block must call), one atomic per block
__device__ __forceinline__ void reduce_norm(unsigned long long *bits, double v) {
    if (!bits) return;
    __shared__ double wmax[32];
    double a = fabs(v);
    if (a != a) a = __longlong_as_double(0x7ff0000000000000ll);
    a = warp_max(a);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) wmax[w] = a;
    __syncthreads();
    if (w == 0) {
        a = (int)threadIdx.x < nw ? wmax[threadIdx.x] : 0.0;
        a = warp_max(a);
        if (threadIdx.x == 0 && a > 0.0) atomic_max_abs(bits, a);
    }
}

// Node of thread t of a launch over a level: over its active chunks where
// the level has them (3D; CHUNK = 32 threads a chunk), else over the whole
// box.  False: the thread has no node.
template <typename T>
__device__ __forceinline__ bool level_node(const LevelView<T> &v, int64_t t, int64_t &p) {
    if (v.chunks) {
        const int64_t c = t >> 5;
        if (c >= v.nchunks || (int)(t & 31) >= (v.clen[c] & 63)) return false;
        p = (int64_t)v.chunks[c] + (t & 31);
        return true;
    }
    if (t >= v.nn) return false;
    p = t;
    return true;
}

template <typename T, int D>
__device__ __forceinline__ T neighbour_sum(const T *__restrict__ u, int64_t p, int64_t s0, int64_t s1) {
    T s = u[p - 1] + u[p + 1] + u[p - s0] + u[p + s0];
    if (D == 3) s += u[p - s1] + u[p + s1];
    return s;
}

// ------------------------------------------------------------ fused sweep
// Both colours of the Gauss-Seidel form of Eq. (jac2d) in one pass over one
// 2D tile (TR x TC nodes, axis 1 contiguous; tile = row tile << 16 | column
// tile): u staged with a 2-node halo, f and node types with a 1-node halo;
// red nodes updated on the tile and its 1-node halo (the values the
// neighbouring tiles compute for their own nodes), then black nodes on the
// tile; the tile's inside nodes are stored (into a second buffer).  Equal to
// a red half-sweep followed by a black half-sweep over the whole grid.
// FP64 form: one flat index over the staged region, f read at inside nodes
// only (the FP64 pipe, not instruction issue, bounds this form)
template <typename T, int TR, int TC>
__device__ __forceinline__ void rb_fused2d_flat(const LevelView<T> &v, T *__restrict__ out, int tile) {
    constexpr int UR = TR + 4, UC = TC + 4, FR = TR + 2, FC = TC + 2;
    __shared__ T su[UR][UC];
    __shared__ T sf[FR][FC];
    __shared__ uint8_t sk[FR][FC];
    const int i0 = (tile >> 16) * TR, j0 = (tile & 0xffff) * TC;
    const int n = v.n;
    for (int idx = threadIdx.x; idx < UR * UC; idx += blockDim.x) {
        const int r = idx / UC, cc = idx - r * UC;
        const int gi = i0 - 2 + r, gj = j0 - 2 + cc;
        su[r][cc] = (gi >= 0 && gi < n && gj >= 0 && gj < n) ? v.u[(int64_t)gi * v.s0 + gj] : (T)0;
    }
    for (int idx = threadIdx.x; idx < FR * FC; idx += blockDim.x) {
        const int r = idx / FC, cc = idx - r * FC;
        const int gi = i0 - 1 + r, gj = j0 - 1 + cc;
        const bool in = gi >= 0 && gi < n && gj >= 0 && gj < n;
        const int64_t p = (int64_t)gi * v.s0 + gj;
        const uint8_t k = in ? (uint8_t)(v.type[p] & NODE_KIND) : (uint8_t)NODE_OUT;
        sk[r][cc] = k;
        sf[r][cc] = (k == NODE_IN) ? v.h2 * v.f[p] : (T)0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < FR * FC; idx += blockDim.x) {
        const int r = idx / FC, cc = idx - r * FC;
        if (sk[r][cc] != NODE_IN || (((i0 - 1 + r) + (j0 - 1 + cc)) & 1)) continue;
        const int ur = r + 1, uc = cc + 1;
        su[ur][uc] = (sf[r][cc] + su[ur - 1][uc] + su[ur + 1][uc] + su[ur][uc - 1] + su[ur][uc + 1]) * (T)0.25;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TR * TC; idx += blockDim.x) {
        const int r = idx / TC, cc = idx - r * TC;
        if (sk[r + 1][cc + 1] != NODE_IN || (((i0 + r) + (j0 + cc)) & 1) == 0) continue;
        const int ur = r + 2, uc = cc + 2;
        su[ur][uc] = (sf[r + 1][cc + 1] + su[ur - 1][uc] + su[ur + 1][uc] + su[ur][uc - 1] + su[ur][uc + 1]) * (T)0.25;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TR * TC; idx += blockDim.x) {
        const int r = idx / TC, cc = idx - r * TC;
        if (sk[r + 1][cc + 1] == NODE_OUT) continue;   // inside: new value; ghost: carried over
        out[(int64_t)(i0 + r) * v.s0 + (j0 + cc)] = su[r + 2][cc + 2];
    }
}

template <typename T, int TR, int TC>
__device__ __forceinline__ void rb_fused2d_cols(const LevelView<T> &v, T *__restrict__ out, int tile) {
    // FP32 form: 256 threads as TY rows x TC columns: a thread owns a column (and the
    // halo columns TC + tx for the first few tx) and steps through rows, so
    // no index is divided and addresses advance by a constant stride
    static_assert(256 % TC == 0 && TC >= 4, "tile width");
    constexpr int TY = 256 / TC;
    constexpr int UR = TR + 4, UC = TC + 4, FR = TR + 2, FC = TC + 2;
    __shared__ T su[UR][UC];
    __shared__ T sf[FR][FC];
    __shared__ uint8_t sk[FR][FC];
    const int i0 = (tile >> 16) * TR, j0 = (tile & 0xffff) * TC;
    const int n = v.n;
    const int tx = threadIdx.x % TC, ty = threadIdx.x / TC;
    // u with a 2-node halo; f and node types with a 1-node halo (f is read
    // whatever the node type: only inside nodes use it); all loads independent
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int cc = tx + k * TC;
        if (k == 1 && tx >= 4) break;
        const int gj = j0 - 2 + cc;
        const bool jok = gj >= 0 && gj < n;
#pragma unroll 4
        for (int r = ty; r < UR; r += TY) {
            const int gi = i0 - 2 + r;
            su[r][cc] = (jok && gi >= 0 && gi < n) ? v.u[(int64_t)gi * v.s0 + gj] : (T)0;
        }
    }
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int cc = tx + k * TC;
        if (k == 1 && tx >= 2) break;
        const int gj = j0 - 1 + cc;
        const bool jok = gj >= 0 && gj < n;
#pragma unroll 4
        for (int r = ty; r < FR; r += TY) {
            const int gi = i0 - 1 + r;
            const bool in = jok && gi >= 0 && gi < n;
            const int64_t p = in ? (int64_t)gi * v.s0 + gj : 0;
            const uint8_t kk = v.type[p];
            const T f = v.f[p];
            sk[r][cc] = in ? (uint8_t)(kk & NODE_KIND) : (uint8_t)NODE_OUT;
            sf[r][cc] = v.h2 * f;
        }
    }
    __syncthreads();
    // red nodes of the tile and its 1-node halo
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int cc = tx + k * TC;
        if (k == 1 && tx >= 2) break;
#pragma unroll 4
        for (int r = ty; r < FR; r += TY) {
            if (sk[r][cc] != NODE_IN || (((i0 - 1 + r) + (j0 - 1 + cc)) & 1)) continue;
            const int ur = r + 1, uc = cc + 1;
            su[ur][uc] = (sf[r][cc] + su[ur - 1][uc] + su[ur + 1][uc] + su[ur][uc - 1] + su[ur][uc + 1]) * (T)0.25;
        }
    }
    __syncthreads();
    // black nodes of the tile
#pragma unroll 4
    for (int r = ty; r < TR; r += TY) {
        if (sk[r + 1][tx + 1] != NODE_IN || (((i0 + r) + (j0 + tx)) & 1) == 0) continue;
        const int ur = r + 2, uc = tx + 2;
        su[ur][uc] = (sf[r + 1][tx + 1] + su[ur - 1][uc] + su[ur + 1][uc] + su[ur][uc - 1] + su[ur][uc + 1]) * (T)0.25;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = ty; r < TR; r += TY) {
        if (sk[r + 1][tx + 1] == NODE_OUT) continue;   // inside: new value; ghost: carried over
        out[(int64_t)(i0 + r) * v.s0 + (j0 + tx)] = su[r + 2][tx + 2];
    }
}

// ------------------------------------------------------------- strip sweep
// Both colours of the Gauss-Seidel form of Eq. (jac2d) over one strip, by one
// warp, without shared memory: lane l holds columns j0 + 2l and j0 + 2l + 1 of
// the strip's 64 (lanes 1-30 own theirs, lanes 0 and 31 are the strip's
// halo) and the warp walks down the strip's rows, keeping three rows of old u
// and of red-updated values in registers (horizontal neighbours by warp
// shuffles) and loading STRIP_PD rows ahead.  Per node, R = the red update at
// red inside nodes, else the old value; the result = the black update (from
// R) at black inside nodes, else R; inside nodes and ghosts are stored into
// `out`.  The sums are those of rb_fused2d_* in the same order, so the values
// are the same.  Loads are clamped to the grid: the setup keeps inside nodes
// and ghosts off the box boundary, so clamped values only reach outside nodes,
// which are not stored.  strip = row block << 16 | column block.
constexpr int STRIP_PD = 3;    // rows loaded ahead

// h^2 f rounded on its own (never contracted into the sum that follows)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// INTERIOR_ONLY: store only the inside nodes outside the boundary band (the
// boundary blocks of the same launch store the band nodes and the ghosts)
template <typename T, int SR, bool INTERIOR_ONLY = false>
__device__ __forceinline__ void rb_strip(const LevelView<T> &v, T *__restrict__ out, int strip) {
    constexpr int PD = STRIP_PD;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int n = v.n;
    const int64_t s0 = v.s0;
    const int i0 = (strip >> 16) * SR, j0 = (strip & 0xffff) * STRIP_W - 2;
    const int c0 = j0 + 2 * lane, c1 = c0 + 1;
    const int q0 = min(max(c0, 0), n - 1), q1 = min(max(c1, 0), n - 1);
    const bool own = lane >= 1 && lane <= 30;
    const T h2 = v.h2;
    const T *__restrict__ u = v.u;
    const T *__restrict__ f = v.f;
    const uint8_t *__restrict__ ty = v.type;
    // row offsets in 32 bits: every grid the solver accepts has fewer than 2^31 nodes
    const int pitch = (int)s0;
    auto rowb = [&](int x) -> int { return min(max(x, 0), n - 1) * pitch; };
    // at row x: ua/ub/uc = u rows x-1, x, x+1; qu[k] = u row x+2+k;
    // fc/kc = f, type of row x; fq/kq[k] = row x+1+k
    T ua0, ua1, ub0, ub1, uc0, uc1, qu0[PD], qu1[PD], fc0, fc1, fq0[PD], fq1[PD];
    uint8_t kc0, kc1, kq0[PD], kq1[PD];
    {
        int b = rowb(i0 - 2);
        ua0 = u[b + q0];
        ua1 = u[b + q1];
        b = rowb(i0 - 1);
        ub0 = u[b + q0];
        ub1 = u[b + q1];
        fc0 = f[b + q0];
        fc1 = f[b + q1];
        kc0 = ty[b + q0];
        kc1 = ty[b + q1];
        b = rowb(i0);
        uc0 = u[b + q0];
        uc1 = u[b + q1];
#pragma unroll
        for (int k = 0; k < PD; k++) {
            const int bu = rowb(i0 + 1 + k), bf = rowb(i0 + k);
            qu0[k] = u[bu + q0];
            qu1[k] = u[bu + q1];
            fq0[k] = f[bf + q0];
            fq1[k] = f[bf + q1];
            kq0[k] = ty[bf + q0];
            kq1[k] = ty[bf + q1];
        }
    }
    T ra0 = 0, ra1 = 0, rb0 = 0, rb1 = 0, fp0 = 0, fp1 = 0;   // R rows x-2, x-1; f of row x-1
    uint8_t kp0 = NODE_OUT, kp1 = NODE_OUT;                     // types of row x-1
#pragma unroll   // SR + 2 rows: the load ring becomes register renaming
    for (int x = i0 - 1; x <= i0 + SR; x++) {
        const T uL = __shfl_up_sync(FULL, ub1, 1), uR = __shfl_down_sync(FULL, ub0, 1);
        const bool red0 = ((x + c0) & 1) == 0;   // c1 has the other colour
        T r0 = ub0, r1 = ub1;
        if ((kc0 & NODE_KIND) == NODE_IN && red0) r0 = (mul_rn(h2, fc0) + ua0 + uc0 + uL + ub1) * (T)0.25;
        if ((kc1 & NODE_KIND) == NODE_IN && !red0) r1 = (mul_rn(h2, fc1) + ua1 + uc1 + ub0 + uR) * (T)0.25;
        if (x > i0) {   // row o = x - 1 of the strip is complete (warp-uniform)
            const int o = x - 1;
            const T RL = __shfl_up_sync(FULL, rb1, 1), RR = __shfl_down_sync(FULL, rb0, 1);
            // a column's colour flips from row to row: c0 is black in row o when it is red in row x
            T o0 = rb0, o1 = rb1;
            if ((kp0 & NODE_KIND) == NODE_IN && red0) o0 = (mul_rn(h2, fp0) + ra0 + r0 + RL + rb1) * (T)0.25;
            if ((kp1 & NODE_KIND) == NODE_IN && !red0) o1 = (mul_rn(h2, fp1) + ra1 + r1 + rb0 + RR) * (T)0.25;
            if (own && o < n) {
                const int b = o * pitch;
                auto stored = [](uint8_t k) {
                    return INTERIOR_ONLY ? (k & (NODE_KIND | NODE_BAND)) == NODE_IN : (k & NODE_KIND) != NODE_OUT;
                };
                if (stored(kp0) && c0 < n) out[b + c0] = o0;
                if (stored(kp1) && c1 < n) out[b + c1] = o1;
            }
        }
        ra0 = rb0;
        ra1 = rb1;
        rb0 = r0;
        rb1 = r1;
        fp0 = fc0;
        fp1 = fc1;
        kp0 = kc0;
        kp1 = kc1;
        fc0 = fq0[0];
        fc1 = fq1[0];
        kc0 = kq0[0];
        kc1 = kq1[0];
        ua0 = ub0;
        ua1 = ub1;
        ub0 = uc0;
        ub1 = uc1;
        uc0 = qu0[0];
        uc1 = qu1[0];
#pragma unroll
        for (int k = 0; k + 1 < PD; k++) {
            qu0[k] = qu0[k + 1];
            qu1[k] = qu1[k + 1];
            fq0[k] = fq0[k + 1];
            fq1[k] = fq1[k + 1];
            kq0[k] = kq0[k + 1];
            kq1[k] = kq1[k + 1];
        }
        const int bu = rowb(x + 3 + PD - 1), bf = rowb(x + 2 + PD - 1);
        qu0[PD - 1] = u[bu + q0];
        qu1[PD - 1] = u[bu + q1];
        fq0[PD - 1] = f[bf + q0];
        fq1[PD - 1] = f[bf + q1];
        kq0[PD - 1] = ty[bf + q0];
        kq1[PD - 1] = ty[bf + q1];
    }
}

// Reads v.u and writes into out (another buffer): every tile stages the values
// before the sweep whatever order the tiles run in.  Ghosts of the tile are
// copied unchanged; tiles cover every inside node and ghost.
template <typename T, int TR, int TC>
__device__ __forceinline__ void rb_fused2d_body(const LevelView<T> &v, T *__restrict__ out, int tile) {
    if constexpr (sizeof(T) == 8) rb_fused2d_flat<T, TR, TC>(v, out, tile);
    else rb_fused2d_cols<T, TR, TC>(v, out, tile);
}

// ------------------------------------------------------- local programs
// One component of a LocalProgram relaxed in shared memory by one CTA of
// LOCAL_THREADS threads: node values, ghost weights, stencil slots, g and
// mu dt staged in shared memory, each thread's inside entries (slot,
// neighbour slots, h^2 f) in registers; an optional ghost sweep, then reps x
// (red, black, Jacobi ghosts); the write-back nodes are stored.  Junction
// zones are components closed under their reads; 2D boundary blocks carry a
// halo covering the dependency cone of the sweeps, so the written values
// equal those of the global sweeps.  The component is staged from grid
// `src` and its write-back nodes are stored into `dst` (the same grid for
// junction zones; for boundary blocks, whose halos overlap, a separate grid
// that local_copyback copies into u once every block has staged its halo, so
// the result does not depend on the order in which the blocks run).  The
// grids are arguments rather than fields of J so that J stays a reference to
// kernel-parameter or global memory instead of a copy held in registers.
// The prologue is two waves of asynchronous copies: the index lists, then
// the gathers through them (each thread gathers through the entries it copied
// itself), so a component costs two memory round trips to stage whatever its
// size.
// wait_lists: the caller has not waited for the launches it depends on yet;
// the index lists (static) are copied first, then it waits.
// pre: also stage the pre-sweep's nodes and run its red then black interior
// update first (the relaxation's interior sweep over what the component
// reads, from `src` holding the grid before that sweep; the same sums as the
// sweep kernels: h^2 f rounded on its own, neighbours in axis order)
template <typename T, int D, int EPT = LOCAL_EPT>
__device__ __forceinline__ void local_body(const LocalView<T> &J, const T *src, T *dst, int c, int lead_ghost,
                                           int reps, bool pre = false, bool wait_lists = false) {
    constexpr int K = D == 2 ? 9 : 27;
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    const int n0 = J.node_off[c], nl = pre ? J.node_off[c + 1] - n0 : J.node_base[c];
    const int i0 = J.int_off[c], ni = J.int_off[c + 1] - i0, nred = J.red_cnt[c];
    const int g0 = J.gh_off[c], ngh = J.gh_off[c + 1] - g0;
    T *val = reinterpret_cast<T *>(smem_dyn);
    T *gw = val + J.max_nodes;       // K per ghost
    T *gv = gw + (size_t)K * J.max_gh;
    T *gcv = gv + J.max_gh;
    T *gt = gcv + J.max_gh;
    T *sf = gt + J.max_gh;                                // f of the inside entries
    int *gst = reinterpret_cast<int *>(sf + J.max_int);   // K per ghost
    int *gme = gst + (size_t)K * J.max_gh;
    int *sln = gme + J.max_gh;                            // staged global nodes
    int *sgq = sln + J.max_nodes;                         // ghost numbers
    int *sig = sgq + J.max_gh;                            // inside entries' global nodes
    T *pf = reinterpret_cast<T *>(local_pre_base<T>(sig + J.max_int));   // pre-sweep: f, slot, node, neighbours
    int *pme = reinterpret_cast<int *>(pf + J.max_pre);
    int *pgl = pme + J.max_pre;
    int *pnb = pgl + J.max_pre;
    const int p0 = pre ? J.pre_off[c] : 0, np = pre ? J.pre_off[c + 1] - p0 : 0;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < nl; i += nt) cp_async(&sln[i], &J.lnode[n0 + i]);
    for (int e = tid; e < ngh; e += nt) {
        cp_async(&sgq[e], &J.gh_q[g0 + e]);
        cp_async(&gme[e], &J.gh_me[g0 + e]);
    }
    for (int i = tid; i < ngh * K; i += nt) cp_async(&gst[i], &J.gh_stn[(size_t)g0 * K + i]);
    for (int i = tid; i < ni; i += nt) cp_async(&sig[i], &J.int_glob[i0 + i]);
    for (int i = tid; i < np; i += nt) {
        cp_async(&pme[i], &J.pre_me[p0 + i]);
        cp_async(&pgl[i], &J.pre_glob[p0 + i]);
    }
    for (int i = tid; i < np * 2 * D; i += nt) cp_async(&pnb[i], &J.pre_nb[(size_t)p0 * 2 * D + i]);
    int rme[EPT], rnb[EPT][2 * D], bme[EPT], bnb[EPT][2 * D];
    T rf[EPT], bf[EPT];
#pragma unroll
    for (int e = 0; e < EPT; e++) {
        const int ir = tid + e * nt, ib = nred + tid + e * nt;
        rme[e] = -1;
        bme[e] = -1;
        if (ir < nred) {
            rme[e] = J.int_me[i0 + ir];
#pragma unroll
            for (int a = 0; a < 2 * D; a++) rnb[e][a] = J.int_nb[(size_t)(i0 + ir) * (2 * D) + a];
        }
        if (ib < ni) {
            bme[e] = J.int_me[i0 + ib];
#pragma unroll
            for (int a = 0; a < 2 * D; a++) bnb[e][a] = J.int_nb[(size_t)(i0 + ib) * (2 * D) + a];
        }
    }
    cp_async_wait_all();
    if (wait_lists) pdl_wait();   // the gathers read what earlier launches wrote
    for (int i = tid; i < nl; i += nt) cp_async(&val[i], &src[sln[i]]);
    for (int e = tid; e < ngh; e += nt) {
        const int q = sgq[e];
        cp_async(&gv[e], &J.gg[q]);
        cp_async(&gcv[e], &J.gc[q]);
        for (int k = 0; k < K; k++) cp_async(&gw[e * K + k], &J.gw[(int64_t)k * J.ng + q]);
    }
    for (int i = tid; i < ni; i += nt) cp_async(&sf[i], &J.f[sig[i]]);
    for (int i = tid; i < np; i += nt) cp_async(&pf[i], &J.f[pgl[i]]);
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int e = 0; e < EPT; e++) {
        const int ir = tid + e * nt, ib = nred + tid + e * nt;
        if (ir < nred) rf[e] = D == 3 ? mul_rn(J.h2, sf[ir]) : J.h2 * sf[ir];
        if (ib < ni) bf[e] = D == 3 ? mul_rn(J.h2, sf[ib]) : J.h2 * sf[ib];
    }
    // 3D: the sum of the global list sweeps (neighbour_sum: axis 2, axis 0,
    // then axis 1; the slots are ordered axis 0, 1, 2), so that a program
    // gives bitwise the values of the launches over the union lists
    auto inside_sum = [&](T h2f, const int *nb) -> T {
        if (D == 3) {
            T s = val[nb[4]] + val[nb[5]] + val[nb[0]] + val[nb[1]];
            s += val[nb[2]] + val[nb[3]];
            return h2f + s;
        }
        T s = h2f;
#pragma unroll
        for (int a = 0; a < 2 * D; a++) s += val[nb[a]];
        return s;
    };
    const T inv = (T)(1.0 / (2 * D));
    if (pre) {
        const int npr = J.pre_red_cnt[c];
        auto update = [&](int e) {
            T s = mul_rn(J.h2, pf[e]);
#pragma unroll
            for (int a = 0; a < 2 * D; a++) s += val[pnb[e * 2 * D + a]];
            val[pme[e]] = s * inv;
        };
        for (int e = threadIdx.x; e < npr; e += blockDim.x) update(e);
        __syncthreads();
        for (int e = npr + threadIdx.x; e < np; e += blockDim.x) update(e);
        __syncthreads();
    }
    auto ghost_sweep = [&]() {
        for (int e = threadIdx.x; e < ngh; e += blockDim.x) {
            T s = 0;
#pragma unroll
            for (int k = 0; k < K; k++) s += gw[e * K + k] * val[gst[e * K + k]];
            gt[e] = val[gme[e]] + gcv[e] * (gv[e] - s);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < ngh; e += blockDim.x) val[gme[e]] = gt[e];
        __syncthreads();
    };
    if (lead_ghost) ghost_sweep();
    for (int it = 0; it < reps; it++) {
#pragma unroll
        for (int e = 0; e < EPT; e++)
            if (rme[e] >= 0) val[rme[e]] = inside_sum(rf[e], rnb[e]) * inv;
        __syncthreads();
#pragma unroll
        for (int e = 0; e < EPT; e++)
            if (bme[e] >= 0) val[bme[e]] = inside_sum(bf[e], bnb[e]) * inv;
        __syncthreads();
        ghost_sweep();
    }
    const int nw = J.wb_cnt[c];
    for (int i = tid; i < nw; i += nt) dst[sln[i]] = val[i];
}

// write-back node i of the flat list: u = wb
template <typename T>
__device__ __forceinline__ void local_copyback(const LocalView<T> &J, T *u, int i) {
    if (i < J.nwb) {
        const int32_t p = J.wb_list[i];
        u[p] = J.wb[p];
    }
}

// ------------------------------------------------------------------ defect
// r = f + Lap_h u at inside node p (TGCS step 3), as a sum of differences so
// that the O(u / h^2) terms do not cancel; with zero_rest, 0 at outside nodes.
// The numerator sum_k u_k - 2d u_p of the 5/7-point Laplacian at inside node
// p (neighbours in the order x-1, x+1, then the two slower axes).  FP32: the
// sum of differences.  FP64: the exact integer sum of exact_lap.h rounded
// once (no FP64-pipe work but the conversion), the sum of differences only
// for non-finite or tiny values.
template <typename T, int D>
__device__ __forceinline__ T lap_numerator(const LevelView<T> &v, int64_t p, T up) {
    T nb[2 * D];
    nb[0] = v.u[p - 1];
    nb[1] = v.u[p + 1];
    nb[2] = v.u[p - v.s0];
    nb[3] = v.u[p + v.s0];
    if (D == 3) {
        nb[2 * D - 2] = v.u[p - v.s1];
        nb[2 * D - 1] = v.u[p + v.s1];
    }
    if constexpr (sizeof(T) == 8) {
        double s;
        if (exl::lap_sum_exact<2 * D>(up, nb, &s)) return s;
    }
    T lap = (nb[0] - up) + (nb[1] - up) + (nb[2] - up) + (nb[3] - up);
    if (D == 3) lap += (nb[2 * D - 2] - up) + (nb[2 * D - 1] - up);
    return lap;
}

// Returns the defect (0 off Omega_h) for the norm.
template <typename T, int D>
__device__ __forceinline__ double defect_node(const LevelView<T> &v, int64_t p, bool zero_rest) {
    const uint8_t k = v.type[p] & NODE_KIND;
    if (k == NODE_IN) {
        const T up = v.u[p];
        const T lap = lap_numerator<T, D>(v, p, up);
        const T r = v.f[p] + lap * v.inv_h2;
        v.r[p] = r;
        return (double)r;
    }
    if (zero_rest && k == NODE_OUT) v.r[p] = 0;
    return 0.0;
}

// r = g - L_G u at ghost q
template <typename T, int K>
__device__ __forceinline__ double defect_ghost_item(const LevelView<T> &v, int q) {
    T s = 0;
#pragma unroll
    for (int k = 0; k < K; k++) s += v.gw[(int64_t)k * v.ng + q] * v.u[v.gstn[(int64_t)k * v.ng + q]];
    const T r = v.gg[q] - s;
    v.r[v.gnode[q]] = r;
    return (double)r;
}

// ------------------------------------------------------------- restriction
// Partial transfer (Sec. 2.5) at a coarse node whose fine image is p: boxes
// prod_a [al_a, be_a] inside the member set, largest ones averaged, weights
// the tensor products of (1,2,1)/4, (2,2,0)/4, (0,2,2)/4, (0,4,0)/4.
template <int D>
__device__ __forceinline__ unsigned box_mask(int b) {
    // bit c of the 3^D neighbourhood (axis 0 slowest, offsets -1,0,1) inside box b;
    // interval code per axis: 0 [-1,1], 1 [-1,0], 2 [0,1], 3 [0,0].  The mask is
    // the AND of one mask per axis: the offsets an interval holds (bits 0..2 of
    // s = 7, 3, 6, 2) spread over the cells with that axis digit.
    auto offs = [](int iv) { return iv == 0 ? 7u : iv == 1 ? 3u : iv == 2 ? 6u : 2u; };
    auto triple = [](unsigned t, unsigned unit, int shift) {   // unit << (shift * digit) for each digit in t
        return ((t & 1u) ? unit : 0u) | ((t & 2u) ? unit << shift : 0u) | ((t & 4u) ? unit << (2 * shift) : 0u);
    };
    if (D == 2) {
        const unsigned m0 = triple(offs(b & 3), 0x7u, 3);              // axis 0: rows of 3 cells
        const unsigned m1 = offs((b >> 2) & 3) * 0x49u;               // axis 1: every 3rd cell
        return m0 & m1;
    }
    const unsigned m0 = triple(offs(b & 3), 0x1FFu, 9);                // axis 0: planes of 9 cells
    const unsigned m1 = triple(offs((b >> 2) & 3), 0x7u, 3) * 0x40201u; // axis 1: rows of 3 in each plane
    const unsigned m2 = offs((b >> 4) & 3) * 0x1249249u;              // axis 2: every 3rd cell
    return m0 & m1 & m2;
}

// 1D factor of the box weights (exact in any binary precision)
template <typename T>
__device__ __forceinline__ T w1d(int iv, int o) {
    switch (iv) {
        case 0: return o == 0 ? (T)0.5 : (T)0.25;
        case 1: return o == 1 ? (T)0 : (T)0.5;
        case 2: return o == -1 ? (T)0 : (T)0.5;
        default: return o == 0 ? (T)1 : (T)0;
    }
}

// a / b for non-negative grid indexes: 32-bit division where a fits (every
// grid the solver accepts), the 64-bit one otherwise
__device__ __forceinline__ int64_t idx_div(int64_t a, int64_t b) {
    if (a <= 0x7fffffffll && b <= 0x7fffffffll) return (int64_t)((uint32_t)a / (uint32_t)b);
    return a / b;
}

template <int D>
__device__ __forceinline__ int64_t fine_image(int64_t X, int64_t cs0, int64_t cs1, int64_t fs0, int64_t fs1) {
    int64_t rem = X;
    if (D == 2) {
        const int64_t j0 = idx_div(rem, cs0), j1 = rem - j0 * cs0;
        return 2 * j0 * fs0 + 2 * j1;
    }
    const int64_t j0 = idx_div(rem, cs0);
    rem -= j0 * cs0;
    const int64_t j1 = idx_div(rem, cs1), j2 = rem - j1 * cs1;
    return 2 * j0 * fs0 + 2 * j1 * fs1 + 2 * j2;
}

// wait: call pdl_wait once the node types are read, before any value (the
// types are fixed while a solve runs; the values come from earlier launches)
// skipped: when not null, a neighbourhood that is not all members is not
// searched: *skipped is set and 0 returned (the caller handles those nodes
// in another launch)
template <typename T, int D, typename Get>
__device__ T partial_transfer_of(const LevelView<T> &F, int64_t p, bool interior, Get value, bool wait = false,
                                 bool *skipped = nullptr) {
    const int cube = D == 2 ? 9 : 27;
    const unsigned full = (1u << cube) - 1u;
    unsigned member = 0;
#pragma unroll
    for (int c = 0; c < cube; c++) {   // the 3^D types are loaded together
        int rem = c;
        int64_t q = p;
        for (int a = D - 1; a >= 0; a--) {
            const int o = rem % 3 - 1;
            rem /= 3;
            q += o * (a == D - 1 ? (int64_t)1 : (a == 0 ? F.s0 : F.s1));
        }
        const uint8_t k = F.type[q] & NODE_KIND;
        if (interior ? (k == NODE_IN) : (k != NODE_IN)) member |= 1u << c;
    }
    const int nbox = D == 2 ? 16 : 64;
    int best = 0, count = 0;
    unsigned long long bestset = 0;   // the boxes of the largest size inside the set
    if (member == full) {
        best = 1;  // full weighting fast path
    } else if (skipped) {
        *skipped = true;
        if (wait) pdl_wait();
        return (T)0;
    } else {
        for (int b = 0; b < nbox; b++) {
            const unsigned m = box_mask<D>(b);
            if (m & ~member) continue;
            const int sz = __popc(m);
            if (sz > best) { best = sz; count = 1; bestset = 1ull << b; }
            else if (sz == best) { count++; bestset |= 1ull << b; }
        }
    }
    if (wait) pdl_wait();
    if (member == full) {
        // full weighting: every value loaded before the first product (one
        // round trip, not 3^D), then the same sum in the same order as below
        T val[cube];
#pragma unroll
        for (int c = 0; c < cube; c++) {
            int rem = c;
            int64_t q = p;
            for (int a = D - 1; a >= 0; a--) {
                q += (rem % 3 - 1) * (a == D - 1 ? (int64_t)1 : (a == 0 ? F.s0 : F.s1));
                rem /= 3;
            }
            val[c] = value(q);
        }
        T acc = 0;
#pragma unroll
        for (int c = 0; c < cube; c++) {
            int rem = c;
            T w = 1;
            int o[3] = {0, 0, 0};
            for (int a = D - 1; a >= 0; a--) {
                o[a] = rem % 3 - 1;
                rem /= 3;
            }
            for (int a = 0; a < D; a++) w *= w1d<T>(0, o[a]);
            acc += w * val[c];
        }
        return acc;
    }
    if (count == 0) return (T)0;   // no box inside the set
    // the members' values loaded together first, then weights and sum in T:
    // the weights are dyadic or 1/count, an FP32 cycle keeps its arithmetic
    // on the FP32 pipe
    T val[cube];
#pragma unroll
    for (int c = 0; c < cube; c++) {
        int rem = c;
        int64_t q = p;
        for (int a = D - 1; a >= 0; a--) {
            q += (rem % 3 - 1) * (a == D - 1 ? (int64_t)1 : (a == 0 ? F.s0 : F.s1));
            rem /= 3;
        }
        val[c] = ((member >> c) & 1u) ? value(q) : (T)0;
    }
    T acc = 0;
#pragma unroll
    for (int c = 0; c < cube; c++) {
        if (!((member >> c) & 1u)) continue;
        int rem = c;
        int o[3] = {0, 0, 0};
        for (int a = D - 1; a >= 0; a--) {
            o[a] = rem % 3 - 1;
            rem /= 3;
        }
        // the largest boxes in increasing order (as a scan of all boxes would)
        T w = 0;
        for (unsigned long long bs = bestset; bs; bs &= bs - 1) {
            const int b = __ffsll((long long)bs) - 1;
            T wb = 1;
            for (int a = 0; a < D; a++) wb *= w1d<T>((b >> (2 * a)) & 3, o[a]);
            w += wb;
        }
        w /= (T)count;
        if (w != (T)0) acc += w * val[c];
    }
    return acc;
}

template <typename T, int D>
__device__ T partial_transfer(const LevelView<T> &F, int64_t p, bool interior) {
    return partial_transfer_of<T, D>(F, p, interior, [&](int64_t q) { return F.r[q]; });
}

// the defect f + Lap_h u at inside node p (the expression of defect_node)
template <typename T, int D>
__device__ __forceinline__ T inside_defect(const LevelView<T> &v, int64_t p) {
    const T up = v.u[p];
    return v.f[p] + lap_numerator<T, D>(v, p, up) * v.inv_h2;
}

// the defect g - L_G u at ghost q (the expression of defect_ghost_item)
template <typename T, int K>
__device__ __forceinline__ T ghost_defect(const LevelView<T> &v, int q) {
    T s = 0;
#pragma unroll
    for (int k = 0; k < K; k++) s += v.gw[(int64_t)k * v.ng + q] * v.u[v.gstn[(int64_t)k * v.ng + q]];
    return v.gg[q] - s;
}

// One descent of the cycle at coarse index i (TGCS steps 3-5 up to the
// coarse solve): the restricted defect at coarse inside node i (the fine
// defects it needs computed on the spot), the transferred defect at coarse
// ghost i (extension + partial transfer of the fine ghost defects), and a
// zero coarse correction.
// FROM_R: the fine defects are read from F.r (written by a defect pass)
// instead of being computed here: where arithmetic rather than latency is
// the bound (FP64), each fine defect is then computed once instead of once
// per coarse node whose 3^d neighbourhood holds it (9/4 times on average in
// 2D).
// full_only: nodes whose neighbourhood is not all inside are left to another
// launch (their fc is not written)
template <typename T, int D, bool FROM_R>
__device__ __forceinline__ void descend_node(const LevelView<T> &F, const LevelView<T> &C, T *__restrict__ fc,
                                             T *__restrict__ uc, int64_t i, bool full_only = false) {
    uc[i] = 0;
    if ((C.type[i] & NODE_KIND) != NODE_IN) {
        fc[i] = (T)0;
        return;
    }
    bool skipped = false;
    const T v = partial_transfer_of<T, D>(F, fine_image<D>(i, C.s0, C.s1, F.s0, F.s1), true,
                                          [&](int64_t q) { return FROM_R ? F.r[q] : inside_defect<T, D>(F, q); },
                                          false, full_only ? &skipped : nullptr);
    if (!skipped) fc[i] = v;
}

// the fine ghost defect that entry col of a ghost-transfer row weighs
template <typename T, int D, bool FROM_R>
__device__ __forceinline__ T transfer_term(const LevelView<T> &F, int col) {
    return FROM_R ? F.r[F.gnode[col]] : ghost_defect<T, D == 2 ? 9 : 27>(F, col);
}

// descend_node in a launch that starts before its predecessor ends: the
// node types are read first, then pdl_wait, then the defects
template <typename T, int D, bool FROM_R>
__device__ __forceinline__ void descend_node_early(const LevelView<T> &F, const LevelView<T> &C,
                                                   T *__restrict__ fc, T *__restrict__ uc, int64_t i) {
    T v = 0;
    if ((C.type[i] & NODE_KIND) == NODE_IN)
        v = partial_transfer_of<T, D>(F, fine_image<D>(i, C.s0, C.s1, F.s0, F.s1), true,
                                      [&](int64_t q) { return FROM_R ? F.r[q] : inside_defect<T, D>(F, q); }, true);
    else
        pdl_wait();
    uc[i] = 0;
    fc[i] = v;
}

// both parts at index i, the ghost row summed by one thread
template <typename T, int D, bool FROM_R = false>
__device__ __forceinline__ void descend_item(const LevelView<T> &F, const LevelView<T> &C, T *__restrict__ fc,
                                             T *__restrict__ gc, T *__restrict__ uc, const int32_t *__restrict__ ptr,
                                             const int32_t *__restrict__ col, const T *__restrict__ val, int64_t i) {
    if (i < C.nn) descend_node<T, D, FROM_R>(F, C, fc, uc, i);
    if (i < C.ng) {
        T s = 0;
        for (int j = ptr[i]; j < ptr[i + 1]; j++) s = fma(val[j], transfer_term<T, D, FROM_R>(F, col[j]), s);
        gc[i] = s;
    }
}

// Coarse ghost row q of the descent by one warp: the lanes fetch the row's
// terms at once (each a chain of dependent loads), then every lane sums them
// in the row's order, as descend_item does.
template <typename T, int D, bool FROM_R>
__device__ __forceinline__ void descend_ghost_row_warp(const LevelView<T> &F, T *__restrict__ gc,
                                                       const int32_t *__restrict__ ptr,
                                                       const int32_t *__restrict__ col, const T *__restrict__ val,
                                                       int q) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, j0 = ptr[q], len = ptr[q + 1] - j0;
    T s = 0;
    for (int base = 0; base < len; base += 32) {
        T w = 0, x = 0;
        if (base + lane < len) {
            w = val[j0 + base + lane];
            x = transfer_term<T, D, FROM_R>(F, col[j0 + base + lane]);
        }
        const int cnt = min(32, len - base);
        for (int k = 0; k < cnt; k++) s = fma(__shfl_sync(FULL, w, k), __shfl_sync(FULL, x, k), s);
    }
    if (lane == 0) gc[q] = s;
}

// descend_ghost_row_warp in a launch that starts before its predecessor
// ends: the first 32 terms' static data (entry, weight, the fine ghost's
// stencil nodes and weights) is read, then pdl_wait, then u and g.  The
// same sums as ghost_defect and descend_item.
template <typename T, int D, bool FROM_R>
__device__ __forceinline__ void descend_ghost_row_warp_early(const LevelView<T> &F, T *__restrict__ gc,
                                                             const int32_t *__restrict__ ptr,
                                                             const int32_t *__restrict__ col,
                                                             const T *__restrict__ val, int q) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int K = D == 2 ? 9 : 27;
    const int lane = threadIdx.x & 31, j0 = ptr[q], len = ptr[q + 1] - j0;
    T w = 0, x = 0;
    int cl = 0, gn = 0, st[K];
    T gw[K];
    if (lane < len) {
        w = val[j0 + lane];
        cl = col[j0 + lane];
        if (FROM_R) {
            gn = F.gnode[cl];
        } else {
#pragma unroll
            for (int k = 0; k < K; k++) {
                st[k] = F.gstn[(int64_t)k * F.ng + cl];
                gw[k] = F.gw[(int64_t)k * F.ng + cl];
            }
        }
    }
    pdl_wait();
    if (lane < len) {
        if (FROM_R) {
            x = F.r[gn];
        } else {
            T t = 0;
#pragma unroll
            for (int k = 0; k < K; k++) t += gw[k] * F.u[st[k]];
            x = F.gg[cl] - t;
        }
    }
    T s = 0;
    const int cnt = min(32, len);
    for (int k = 0; k < cnt; k++) s = fma(__shfl_sync(FULL, w, k), __shfl_sync(FULL, x, k), s);
    for (int base = 32; base < len; base += 32) {   // rows longer than a warp
        T w2 = 0, x2 = 0;
        if (base + lane < len) {
            w2 = val[j0 + base + lane];
            x2 = transfer_term<T, D, FROM_R>(F, col[j0 + base + lane]);
        }
        const int c2 = min(32, len - base);
        for (int k = 0; k < c2; k++) s = fma(__shfl_sync(FULL, w2, k), __shfl_sync(FULL, x2, k), s);
    }
    if (lane == 0) gc[q] = s;
}


// coarse node X: transfer over Omega_h at coarse inside nodes, 0 elsewhere
template <typename T, int D>
__device__ __forceinline__ void restrict_node(const LevelView<T> &F, const LevelView<T> &C, int64_t X, T *fc) {
    if ((C.type[X] & NODE_KIND) != NODE_IN) { fc[X] = 0; return; }
    fc[X] = partial_transfer<T, D>(F, fine_image<D>(X, C.s0, C.s1, F.s0, F.s1), true);
}

// coarse ghost q: transfer over D_h - Omega_h (used by the single-step API)
template <typename T, int D>
__device__ __forceinline__ void restrict_ghost_item(const LevelView<T> &F, const LevelView<T> &C, int q, T *gc) {
    gc[q] = partial_transfer<T, D>(F, fine_image<D>(C.gnode[q], C.s0, C.s1, F.s0, F.s1), false);
}

// extension + partial transfer at coarse ghost q as one sparse row over the
// fine ghost defects (read from the fine defect grid)
template <typename T>
__device__ __forceinline__ void ghost_transfer_row(const T *__restrict__ rf, const int32_t *__restrict__ fgnode,
                                                   const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                                   const T *__restrict__ val, T *__restrict__ gc, int q) {
    T s = 0;
    for (int j = ptr[q]; j < ptr[q + 1]; j++) s += val[j] * rf[fgnode[col[j]]];
    gc[q] = s;
}

// ------------------------------------------------------------ interpolation
// Bilinear / trilinear interpolation onto Omega_h u Gamma_h at fine node p
// (Sec. 2.6), weights renormalised over the parents in Omega_2h u Gamma_2h.
template <typename T, int D>
__device__ __forceinline__ void prolong_node(const LevelView<T> &F, const LevelView<T> &C, const T *__restrict__ e,
                                             T *__restrict__ out, bool add, int64_t p) {
    const uint8_t k = F.type[p] & NODE_KIND;
    if (k != NODE_IN && k != NODE_GHOST) {
        if (!add) out[p] = 0;
        return;
    }
    int j[3] = {0, 0, 0};
    int64_t rem = p;
    j[0] = (int)idx_div(rem, F.s0);
    rem -= (int64_t)j[0] * F.s0;
    if (D == 2) {
        j[1] = (int)rem;
    } else {
        j[1] = (int)idx_div(rem, F.s1);
        j[2] = (int)(rem - (int64_t)j[1] * F.s1);
    }
    T num = 0, den = 0;
    const int n1 = (j[0] & 1) ? 2 : 1, n2 = (j[1] & 1) ? 2 : 1, n3 = (D == 3 && (j[2] & 1)) ? 2 : 1;
    for (int a = 0; a < n1; a++)
        for (int b = 0; b < n2; b++)
            for (int c = 0; c < n3; c++) {
                const int64_t X = (int64_t)(j[0] / 2 + a) * C.s0 +
                                  (D == 2 ? (int64_t)(j[1] / 2 + b) : (int64_t)(j[1] / 2 + b) * C.s1 + (j[2] / 2 + c));
                const uint8_t kc = C.type[X] & NODE_KIND;
                if (kc != NODE_IN && kc != NODE_GHOST) continue;
                const T w = (T)1 / (T)(n1 * n2 * n3);   // a power of two: exact
                num += w * e[X];
                den += w;
            }
    const T val = den > (T)0 ? num / den : (T)0;
    if (add) out[p] += val;
    else out[p] = val;
}

// prolong_node in a launch that starts before its predecessor ends: the
// node's and its parents' types are read first, then pdl_wait, then e and
// out.  The same sums as prolong_node.
template <typename T, int D>
__device__ __forceinline__ void prolong_node_early(const LevelView<T> &F, const LevelView<T> &C,
                                                   const T *__restrict__ e, T *__restrict__ out, bool add, int64_t p) {
    const uint8_t k = F.type[p] & NODE_KIND;
    const bool on = k == NODE_IN || k == NODE_GHOST;
    int j[3] = {0, 0, 0};
    int64_t rem = p;
    j[0] = (int)idx_div(rem, F.s0);
    rem -= (int64_t)j[0] * F.s0;
    if (D == 2) {
        j[1] = (int)rem;
    } else {
        j[1] = (int)idx_div(rem, F.s1);
        j[2] = (int)(rem - (int64_t)j[1] * F.s1);
    }
    const int n1 = (j[0] & 1) ? 2 : 1, n2 = (j[1] & 1) ? 2 : 1, n3 = (D == 3 && (j[2] & 1)) ? 2 : 1;
    // up to 2^D parents in fixed slots (a, b, c), every load of a phase issued
    // before the first use
    constexpr int NS = D == 3 ? 8 : 4;
    int64_t X[NS];
    bool use[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) {
        const int a = D == 3 ? s >> 2 : s >> 1, b = D == 3 ? (s >> 1) & 1 : s & 1, c = D == 3 ? s & 1 : 0;
        X[s] = (int64_t)(j[0] / 2 + a) * C.s0 +
               (D == 2 ? (int64_t)(j[1] / 2 + b) : (int64_t)(j[1] / 2 + b) * C.s1 + (j[2] / 2 + c));
        use[s] = false;
        if (on && a < n1 && b < n2 && c < n3) {
            const uint8_t kc = C.type[X[s]] & NODE_KIND;
            use[s] = kc == NODE_IN || kc == NODE_GHOST;   // parents in Omega_2h u Gamma_2h
        }
    }
    pdl_wait();
    if (!on) {
        if (!add) out[p] = 0;
        return;
    }
    T ev[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) ev[s] = use[s] ? e[X[s]] : (T)0;
    T num = 0, den = 0;
    const T w = (T)1 / (T)(n1 * n2 * n3);   // a power of two: exact
#pragma unroll
    for (int s = 0; s < NS; s++)   // (a, b, c) order, as prolong_node
        if (use[s]) {
            num += w * ev[s];
            den += w;
        }
    const T val = den > (T)0 ? num / den : (T)0;
    if (add) out[p] += val;
    else out[p] = val;
}

// --------------------------------------------------------------- coarsest
// ---------------------------------------------------- exact junction solve
// Defect of the equation of row k of the junction solve: at an inside node
// f + Lap_h u (as a sum of differences), at ghost q g - L_G u.
// WB: the boundary blocks' write-back into u is still pending (it runs in the
// same launch), so the nodes marked NODE_WB are read from the write-back grid
// wb, which holds the values being copied into u.
template <typename T, int D, bool WB = false>
__device__ __forceinline__ T js_defect(const LevelView<T> &v, int32_t p, int32_t q, const T *wb = nullptr) {
    auto rd = [&](int64_t x) -> T { return (WB && (v.type[x] & NODE_WB)) ? wb[x] : v.u[x]; };
    if (q >= 0) {
        constexpr int K = D == 2 ? 9 : 27;
        T s = 0;
#pragma unroll
        for (int k = 0; k < K; k++) s += v.gw[(int64_t)k * v.ng + q] * rd(v.gstn[(int64_t)k * v.ng + q]);
        return v.gg[q] - s;
    }
    const T up = rd(p);
    T lap = (rd(p - 1) - up) + (rd(p + 1) - up) + (rd(p - v.s0) - up) + (rd(p + v.s0) - up);
    if (D == 3) lap += (rd(p - v.s1) - up) + (rd(p + v.s1) - up);
    return v.f[p] + lap * v.inv_h2;
}

// 16-byte vectors of T and their dot product (in component order)
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
    static __device__ __forceinline__ float dot(float s, float4 a, float4 b) {
        s = fmaf(a.x, b.x, s);
        s = fmaf(a.y, b.y, s);
        s = fmaf(a.z, b.z, s);
        return fmaf(a.w, b.w, s);
    }
};
template <>
struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
    static __device__ __forceinline__ double dot(double s, double2 a, double2 b) {
        s = fma(a.x, b.x, s);
        return fma(a.y, b.y, s);
    }
};

// u(node k) += sum_j Ainv_c[k - off_c, j] r_c[j] for rows k0 .. k0 + nr - 1
// (nr <= R) of one component c, by one warp: each lane takes 16-byte
// vectors of the padded rows and of the component's padded defects (both
// 16-byte aligned, zero pads), the defect vector shared by the R rows and
// U vectors a row in flight.  A lane sums its vectors of a row in index
// order, whatever R and U, so every row's value is independent of how rows
// are grouped.
template <typename T, int R, int U = 2>
__device__ __forceinline__ void js_apply_rows(T *__restrict__ u, const int32_t *__restrict__ node,
                                              const int32_t *__restrict__ off, const int64_t *__restrict__ aoff,
                                              const int32_t *__restrict__ roff, const T *__restrict__ inv,
                                              const T *__restrict__ r, int c, int k0, int nr, int lane) {
    using V = typename Vec16<T>::type;
    const int o = off[c];
    const int mp = (off[c + 1] - o + 3) & ~3;
    const V *a = reinterpret_cast<const V *>(inv + aoff[c] + (int64_t)(k0 - o) * mp);
    const V *rr = reinterpret_cast<const V *>(r + roff[c]);
    const int nv = mp / Vec16<T>::n, rs = nv;   // row stride in vectors
    T s[R];
#pragma unroll
    for (int i = 0; i < R; i++) s[i] = 0;
    for (int j0 = lane; j0 < nv; j0 += 32 * U) {
        V rv[U], av[R][U];
#pragma unroll
        for (int e = 0; e < U; e++)
            if (j0 + 32 * e < nv) {
                rv[e] = rr[j0 + 32 * e];
#pragma unroll
                for (int i = 0; i < R; i++)
                    if (i < nr) av[i][e] = a[(int64_t)i * rs + j0 + 32 * e];
            }
#pragma unroll
        for (int e = 0; e < U; e++)
            if (j0 + 32 * e < nv)
#pragma unroll
                for (int i = 0; i < R; i++)
                    if (i < nr) s[i] = Vec16<T>::dot(s[i], av[i][e], rv[e]);
    }
#pragma unroll
    for (int i = 0; i < R; i++) {
        T t = s[i];
        for (int w = 16; w > 0; w >>= 1) t += __shfl_xor_sync(0xffffffffu, t, w);
        if (lane == 0 && i < nr) u[node[k0 + i]] += t;
    }
}

// rows k0 .. k1 - 1 of the junction solve (any components) by one warp, in
// groups of at most R rows of one component
template <typename T, int R>
__device__ __forceinline__ void js_apply_span(T *__restrict__ u, const int32_t *__restrict__ node,
                                              const int32_t *__restrict__ comp, const int32_t *__restrict__ off,
                                              const int64_t *__restrict__ aoff, const int32_t *__restrict__ roff,
                                              const T *__restrict__ inv, const T *__restrict__ r, int k0, int k1,
                                              int lane) {
    for (int k = k0; k < k1;) {
        const int c = comp[k];
        const int e = min(min(k1, off[c + 1]), k + R);
        js_apply_rows<T, R>(u, node, off, aoff, roff, inv, r, c, k, e - k, lane);
        k = e;
    }
}

// one row k by one warp, launched before the defects it needs are written:
// the row of the inverse (up to MAXV vectors a lane, the rest after) and the
// row's node are loaded, then the warp waits for the previous launch
// (pdl_wait) and reads the defects and u.  The same sums as js_apply_rows.
template <typename T, int MAXV>
__device__ __forceinline__ void js_apply_row_early(T *__restrict__ u, const int32_t *__restrict__ node,
                                                   const int32_t *__restrict__ comp, const int32_t *__restrict__ off,
                                                   const int64_t *__restrict__ aoff, const int32_t *__restrict__ roff,
                                                   const T *__restrict__ inv, const T *__restrict__ r, int k,
                                                   int lane) {
    using V = typename Vec16<T>::type;
    const int c = comp[k], o = off[c];
    const int mp = (off[c + 1] - o + 3) & ~3;
    const V *a = reinterpret_cast<const V *>(inv + aoff[c] + (int64_t)(k - o) * mp);
    const int nv = mp / Vec16<T>::n;
    V av[MAXV];
#pragma unroll
    for (int e = 0; e < MAXV; e++)
        if (lane + 32 * e < nv) av[e] = a[lane + 32 * e];
    const int nd = node[k];
    const V *rr = reinterpret_cast<const V *>(r + roff[c]);
    pdl_wait();
    const T uo = lane == 0 ? u[nd] : (T)0;
    T s = 0;
#pragma unroll
    for (int e = 0; e < MAXV; e++)
        if (lane + 32 * e < nv) s = Vec16<T>::dot(s, av[e], rr[lane + 32 * e]);
    for (int j = lane + 32 * MAXV; j < nv; j += 32) s = Vec16<T>::dot(s, a[j], rr[j]);
    for (int w = 16; w > 0; w >>= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
    if (lane == 0) u[nd] = uo + s;
}

// one row k (the form of the fused coarse cycle)
template <typename T>
__device__ __forceinline__ void js_apply_row(T *__restrict__ u, const int32_t *__restrict__ node,
                                             const int32_t *__restrict__ comp, const int32_t *__restrict__ off,
                                             const int64_t *__restrict__ aoff, const int32_t *__restrict__ roff,
                                             const T *__restrict__ inv, const T *__restrict__ r, int k, int lane) {
    js_apply_rows<T, 1>(u, node, off, aoff, roff, inv, r, comp[k], k, 1, lane);
}

// e = A^-1 b on the coarsest level, rows blk, blk + nblk, ... of one CTA: b
// gathered into shared memory from f (inside) and the ghost data, each warp
// computing row dot products of the dense inverse.
template <typename T>
__device__ __forceinline__ void coarse_rows(const LevelView<T> &v, const int32_t *__restrict__ unk_node,
                                            const int32_t *__restrict__ unk_ghost, const T *__restrict__ Ainv,
                                            int m, int blk, int nblk) {
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    T *b = reinterpret_cast<T *>(smem_dyn);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int g = unk_ghost[i];
        b[i] = g < 0 ? v.f[unk_node[i]] : v.gg[g];
    }
    __syncthreads();
    const int warps = blockDim.x >> 5;
    const int lane = threadIdx.x & 31;
    for (int row = blk * warps + (threadIdx.x >> 5); row < m; row += nblk * warps) {
        const T *a = Ainv + (int64_t)row * m;
        T s = 0;
        for (int k = lane; k < m; k += 32) s += a[k] * b[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) v.u[unk_node[row]] = s;
    }
}

}  // namespace dev
}  // namespace gcmg
