// Device kernels of one multigrid level, templated on the precision T and
// the dimension D.  Grids are dense C-ordered n^D arrays (last axis
// contiguous); ghost records are slot-major so that consecutive threads read
// consecutive words.
#include <cuda_runtime.h>

#include <atomic>

#include "gcmg_internal.h"
#include "kernels.h"

namespace gcmg {

std::atomic<long long> g_launches{0};

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(int64_t total, int threads = kThreads) {
    int64_t b = (total + threads - 1) / threads;
    return (unsigned)(b > 0 ? b : 1);
}

// max-norm reduction on the bit pattern of a non-negative double (monotone
// for non-negative IEEE values); NaN is folded into +Inf so that it is seen.
__device__ __forceinline__ void atomic_max_abs(unsigned long long *bits, double v) {
    v = fabs(v);
    if (v != v) v = __longlong_as_double(0x7ff0000000000000ull);
    atomicMax(bits, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// block-wide max of |v| (all threads of the block must call), one atomic per block
__device__ __forceinline__ void reduce_norm(unsigned long long *bits, double v) {
    if (!bits) return;
    __shared__ double wmax[32];
    double a = fabs(v);
    if (a != a) a = __longlong_as_double(0x7ff0000000000000ull);
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

template <int D>
__device__ __forceinline__ bool decode_colour(int n, int color, int64_t t, int64_t s0, int64_t s1, int64_t &p) {
    // thread t -> node of the given colour (sum of indices even = 0 / odd = 1)
    const int hc = (n + 1) >> 1;
    int i0, i1 = 0, jj;
    if (D == 2) {
        i0 = (int)(t / hc);
        jj = (int)(t - (int64_t)i0 * hc);
    } else {
        jj = (int)(t % hc);
        const int64_t rest = t / hc;
        i1 = (int)(rest % n);
        i0 = (int)(rest / n);
    }
    if (i0 >= n) return false;
    const int last = 2 * jj + ((i0 + i1 + color) & 1);
    if (last >= n) return false;
    p = (int64_t)i0 * s0 + (D == 3 ? (int64_t)i1 * s1 : 0) + last;
    return true;
}

template <typename T, int D>
__device__ __forceinline__ T neighbour_sum(const T *__restrict__ u, int64_t p, int64_t s0, int64_t s1) {
    T s = u[p - 1] + u[p + 1] + u[p - s0] + u[p + s0];
    if (D == 3) s += u[p - s1] + u[p + s1];
    return s;
}

// ---------------------------------------------------------------- smoothers
// Gauss-Seidel form of Eq. (jac2d) on the inside nodes of one colour.
template <typename T, int D>
__global__ void k_rb_interior(LevelView<T> v, int color) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t p;
    if (!decode_colour<D>(v.n, color, t, v.s0, v.s1, p)) return;
    if ((v.type[p] & NODE_KIND) != NODE_IN) return;
    const T s = v.h2 * v.f[p] + neighbour_sum<T, D>(v.u, p, v.s0, v.s1);
    v.u[p] = s * (T)(1.0 / (2 * D));
}

// Both colours in one pass over the active 2D tiles (TILE_R x TILE_C nodes,
// axis 1 contiguous): u is staged with a 2-node halo, f and the node types
// with a 1-node halo; red nodes are updated on the tile and its 1-node halo
// (the values the neighbouring tiles compute for their own nodes), then black
// nodes on the tile, and the tile's inside nodes are stored.  Equal to a red
// half-sweep followed by a black half-sweep over the whole grid.
template <typename T>
__global__ void __launch_bounds__(256) k_rb_fused2d(LevelView<T> v, const int32_t *__restrict__ tiles) {
    constexpr int UR = TILE_R + 4, UC = TILE_C + 4, FR = TILE_R + 2, FC = TILE_C + 2;
    __shared__ T su[UR][UC];
    __shared__ T sf[FR][FC];
    __shared__ uint8_t sk[FR][FC];
    const int tile = tiles[blockIdx.x];
    const int i0 = (tile >> 16) * TILE_R, j0 = (tile & 0xffff) * TILE_C;
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
    // red (even index sum) on the tile and its 1-node halo
    for (int idx = threadIdx.x; idx < FR * FC; idx += blockDim.x) {
        const int r = idx / FC, cc = idx - r * FC;
        if (sk[r][cc] != NODE_IN || (((i0 - 1 + r) + (j0 - 1 + cc)) & 1)) continue;
        const int ur = r + 1, uc = cc + 1;
        su[ur][uc] = (sf[r][cc] + su[ur - 1][uc] + su[ur + 1][uc] + su[ur][uc - 1] + su[ur][uc + 1]) * (T)0.25;
    }
    __syncthreads();
    // black on the tile
    for (int idx = threadIdx.x; idx < TILE_R * TILE_C; idx += blockDim.x) {
        const int r = idx / TILE_C, cc = idx - r * TILE_C;
        if (sk[r + 1][cc + 1] != NODE_IN || (((i0 + r) + (j0 + cc)) & 1) == 0) continue;
        const int ur = r + 2, uc = cc + 2;
        su[ur][uc] = (sf[r + 1][cc + 1] + su[ur - 1][uc] + su[ur + 1][uc] + su[ur][uc - 1] + su[ur][uc + 1]) * (T)0.25;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TILE_R * TILE_C; idx += blockDim.x) {
        const int r = idx / TILE_C, cc = idx - r * TILE_C;
        if (sk[r + 1][cc + 1] != NODE_IN) continue;
        v.u[(int64_t)(i0 + r) * v.s0 + (j0 + cc)] = su[r + 2][cc + 2];
    }
}

// Same update over a compact list of band nodes of one colour (Sec. 3.2).
template <typename T, int D>
__global__ void k_rb_list(LevelView<T> v, const int32_t *__restrict__ list, int cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int64_t p = list[i];
    const T s = v.h2 * v.f[p] + neighbour_sum<T, D>(v.u, p, v.s0, v.s1);
    v.u[p] = s * (T)(1.0 / (2 * D));
}

// Ghost relaxation, Eqs. (dir2d)/(neu2d): new value from the current values.
template <typename T, int K>
__global__ void k_ghost_new(LevelView<T> v) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= v.ng) return;
    T s = 0;
#pragma unroll
    for (int k = 0; k < K; k++) s += v.gw[(int64_t)k * v.ng + q] * v.u[v.gstn[(int64_t)k * v.ng + q]];
    v.gtmp[q] = v.u[v.gnode[q]] + v.gc[q] * (v.gg[q] - s);
}

// same update restricted to a list of ghost numbers
template <typename T, int K>
__global__ void k_ghost_new_list(LevelView<T> v, const int32_t *__restrict__ list, int cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int q = list[i];
    T s = 0;
#pragma unroll
    for (int k = 0; k < K; k++) s += v.gw[(int64_t)k * v.ng + q] * v.u[v.gstn[(int64_t)k * v.ng + q]];
    v.gtmp[q] = v.u[v.gnode[q]] + v.gc[q] * (v.gg[q] - s);
}

template <typename T>
__global__ void k_ghost_store_list(LevelView<T> v, const int32_t *__restrict__ list, int cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int q = list[i];
    v.u[v.gnode[q]] = v.gtmp[q];
}

template <typename T>
__global__ void k_ghost_store(LevelView<T> v) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= v.ng) return;
    v.u[v.gnode[q]] = v.gtmp[q];
}

// ------------------------------------------------- shared-memory programs
// One CTA per component of a LocalProgram.  The component's node values, the
// ghost weights, stencil slots, g and mu dt are staged in shared memory; each
// thread keeps its inside-node entries (slot, neighbour slots, h^2 f) in
// registers.  Then an optional ghost sweep and reps x (red, black, Jacobi
// ghosts) run on the staged copy, and the write-back nodes are stored.  Used
// for the junction zones (components closed under their reads) and the 2D
// boundary blocks (halo = dependency cone of the sweeps, so the written values
// equal those of the global sweeps).
constexpr int LOCAL_THREADS = 512;
constexpr int LOCAL_EPT = 4;     // inside entries per thread and colour

template <typename T, int D>
__global__ void __launch_bounds__(LOCAL_THREADS) k_local(LocalView<T> J, int lead_ghost, int reps) {
    constexpr int K = D == 2 ? 9 : 27;
    extern __shared__ __align__(16) unsigned char smem_j[];
    const int c = blockIdx.x;
    const int n0 = J.node_off[c], nl = J.node_off[c + 1] - n0;
    const int i0 = J.int_off[c], ni = J.int_off[c + 1] - i0, nred = J.red_cnt[c], nblk = ni - nred;
    const int g0 = J.gh_off[c], ngh = J.gh_off[c + 1] - g0;
    T *val = reinterpret_cast<T *>(smem_j);
    T *gw = val + J.max_nodes;       // K per ghost
    T *gv = gw + (size_t)K * J.max_gh;
    T *gcv = gv + J.max_gh;
    T *gt = gcv + J.max_gh;
    int *gst = reinterpret_cast<int *>(gt + J.max_gh);   // K per ghost
    int *gme = gst + (size_t)K * J.max_gh;
    for (int i = threadIdx.x; i < nl; i += blockDim.x) val[i] = J.u[J.lnode[n0 + i]];
    for (int e = threadIdx.x; e < ngh; e += blockDim.x) {
        const int q = J.gh_q[g0 + e];
        gv[e] = J.gg[q];
        gcv[e] = J.gc[q];
        gme[e] = J.gh_me[g0 + e];
        for (int k = 0; k < K; k++) {
            gw[e * K + k] = J.gw[(int64_t)k * J.ng + q];
            gst[e * K + k] = J.gh_stn[(size_t)(g0 + e) * K + k];
        }
    }
    // this thread's inside entries: e-th red entry is threadIdx.x + e * blockDim.x
    int rme[LOCAL_EPT], rnb[LOCAL_EPT][2 * D], bme[LOCAL_EPT], bnb[LOCAL_EPT][2 * D];
    T rf[LOCAL_EPT], bf[LOCAL_EPT];
#pragma unroll
    for (int e = 0; e < LOCAL_EPT; e++) {
        const int ir = threadIdx.x + e * blockDim.x, ib = nred + threadIdx.x + e * blockDim.x;
        rme[e] = -1;
        bme[e] = -1;
        if (ir < nred) {
            rme[e] = J.int_me[i0 + ir];
            rf[e] = J.h2 * J.f[J.int_glob[i0 + ir]];
#pragma unroll
            for (int a = 0; a < 2 * D; a++) rnb[e][a] = J.int_nb[(size_t)(i0 + ir) * (2 * D) + a];
        }
        if (ib < ni) {
            bme[e] = J.int_me[i0 + ib];
            bf[e] = J.h2 * J.f[J.int_glob[i0 + ib]];
#pragma unroll
            for (int a = 0; a < 2 * D; a++) bnb[e][a] = J.int_nb[(size_t)(i0 + ib) * (2 * D) + a];
        }
    }
    (void)nblk;
    __syncthreads();
    const T inv = (T)(1.0 / (2 * D));
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
        for (int e = 0; e < LOCAL_EPT; e++)
            if (rme[e] >= 0) {
                T s = rf[e];
#pragma unroll
                for (int a = 0; a < 2 * D; a++) s += val[rnb[e][a]];
                val[rme[e]] = s * inv;
            }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < LOCAL_EPT; e++)
            if (bme[e] >= 0) {
                T s = bf[e];
#pragma unroll
                for (int a = 0; a < 2 * D; a++) s += val[bnb[e][a]];
                val[bme[e]] = s * inv;
            }
        __syncthreads();
        ghost_sweep();
    }
    const int nw = J.wb_cnt[c];
    for (int i = threadIdx.x; i < nw; i += blockDim.x) J.u[J.lnode[n0 + i]] = val[i];
}

// ------------------------------------------------------------------ defect
// r = f + Lap_h u on Omega_h (TGCS step 3); with zero_rest, 0 on outside
// nodes (ghost rows are written by k_defect_ghost).
template <typename T, int D>
__global__ void k_defect_interior(LevelView<T> v, bool zero_rest, unsigned long long *norm) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double val = 0.0;
    if (p < v.nn) {
        const uint8_t k = v.type[p] & NODE_KIND;
        if (k == NODE_IN) {
            // sum of differences: no cancellation of the O(u / h^2) terms
            const T up = v.u[p];
            T lap = (v.u[p - 1] - up) + (v.u[p + 1] - up) + (v.u[p - v.s0] - up) + (v.u[p + v.s0] - up);
            if (D == 3) lap += (v.u[p - v.s1] - up) + (v.u[p + v.s1] - up);
            const T r = v.f[p] + lap * v.inv_h2;
            v.r[p] = r;
            val = (double)r;
        } else if (zero_rest && k == NODE_OUT) {
            v.r[p] = 0;
        }
    }
    reduce_norm(norm, val);
}

template <typename T, int K>
__global__ void k_defect_ghost(LevelView<T> v, unsigned long long *norm) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    double val = 0.0;
    if (q < v.ng) {
        T s = 0;
#pragma unroll
        for (int k = 0; k < K; k++) s += v.gw[(int64_t)k * v.ng + q] * v.u[v.gstn[(int64_t)k * v.ng + q]];
        const T r = v.gg[q] - s;
        v.r[v.gnode[q]] = r;
        val = (double)r;
    }
    reduce_norm(norm, val);
}

// ---------------------------------------------------------------- extension
// One wavefront of the defect extension (Sec. 2.6).
template <typename T>
__global__ void k_extend(T *__restrict__ r, const int32_t *__restrict__ node, const uint8_t *__restrict__ cnt,
                         const int32_t *__restrict__ src, const T *__restrict__ w, int ne, int begin, int end) {
    const int i = begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= end) return;
    T s = 0;
    const int c = cnt[i];
    for (int k = 0; k < c; k++) s += w[(int64_t)k * ne + i] * r[src[(int64_t)k * ne + i]];
    r[node[i]] = s;
}

// ------------------------------------------------------------- restriction
// Partial transfer (Sec. 2.5) at a coarse node whose fine image is p: boxes
// prod_a [al_a, be_a] inside the member set, largest ones averaged, weights
// the tensor products of (1,2,1)/4, (2,2,0)/4, (0,2,2)/4, (0,4,0)/4.
template <int D>
__device__ __forceinline__ unsigned box_mask(int b) {
    // bit c of the 3^D neighbourhood (axis 0 slowest, offsets -1,0,1) inside box b;
    // interval code per axis: 0 [-1,1], 1 [-1,0], 2 [0,1], 3 [0,0]
    unsigned m = 0;
    const int cube = D == 2 ? 9 : 27;
    for (int c = 0; c < cube; c++) {
        int rem = c, ok = 1;
        for (int a = D - 1; a >= 0; a--) {
            const int o = rem % 3 - 1;
            rem /= 3;
            const int iv = (b >> (2 * a)) & 3;
            const int lo = (iv == 2 || iv == 3) ? 0 : -1;
            const int hi = (iv == 1 || iv == 3) ? 0 : 1;
            if (o < lo || o > hi) ok = 0;
        }
        if (ok) m |= 1u << c;
    }
    return m;
}

__device__ __forceinline__ double w1d(int iv, int o) {
    switch (iv) {
        case 0: return o == 0 ? 0.5 : 0.25;
        case 1: return o == 1 ? 0.0 : 0.5;
        case 2: return o == -1 ? 0.0 : 0.5;
        default: return o == 0 ? 1.0 : 0.0;
    }
}

template <typename T, int D>
__device__ T partial_transfer(const LevelView<T> &F, int64_t p, bool interior) {
    const int cube = D == 2 ? 9 : 27;
    const unsigned full = (1u << cube) - 1u;
    unsigned member = 0;
    for (int c = 0; c < cube; c++) {
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
    if (member == full) {
        best = 1;  // full weighting fast path
    } else {
        for (int b = 0; b < nbox; b++) {
            const unsigned m = box_mask<D>(b);
            if (m & ~member) continue;
            const int sz = __popc(m);
            if (sz > best) { best = sz; count = 1; }
            else if (sz == best) count++;
        }
        if (count == 0) return (T)0;
    }
    double acc = 0.0;
    for (int c = 0; c < cube; c++) {
        if (!((member >> c) & 1u)) continue;
        int rem = c;
        int64_t q = p;
        int o[3] = {0, 0, 0};
        for (int a = D - 1; a >= 0; a--) {
            o[a] = rem % 3 - 1;
            rem /= 3;
            q += o[a] * (a == D - 1 ? (int64_t)1 : (a == 0 ? F.s0 : F.s1));
        }
        double w = 0.0;
        if (member == full) {
            w = 1.0;
            for (int a = 0; a < D; a++) w *= w1d(0, o[a]);
        } else {
            for (int b = 0; b < nbox; b++) {
                const unsigned m = box_mask<D>(b);
                if ((m & ~member) || __popc(m) != best) continue;
                double wb = 1.0;
                for (int a = 0; a < D; a++) wb *= w1d((b >> (2 * a)) & 3, o[a]);
                w += wb;
            }
            w /= count;
        }
        if (w != 0.0) acc += w * (double)F.r[q];
    }
    return (T)acc;
}

// coarse interior nodes: transfer over Omega_h; other coarse nodes get 0
template <typename T, int D>
__global__ void k_restrict_interior(LevelView<T> F, LevelView<T> C, T *__restrict__ fc) {
    const int64_t X = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (X >= C.nn) return;
    if ((C.type[X] & NODE_KIND) != NODE_IN) { fc[X] = 0; return; }
    int64_t rem = X, p = 0;
    if (D == 2) {
        const int64_t j0 = rem / C.s0, j1 = rem - j0 * C.s0;
        p = 2 * j0 * F.s0 + 2 * j1;
    } else {
        const int64_t j0 = rem / C.s0;
        rem -= j0 * C.s0;
        const int64_t j1 = rem / C.s1, j2 = rem - j1 * C.s1;
        p = 2 * j0 * F.s0 + 2 * j1 * F.s1 + 2 * j2;
    }
    fc[X] = partial_transfer<T, D>(F, p, true);
}

// coarse ghosts: transfer over D_h - Omega_h (ghost defects and extended values)
template <typename T, int D>
__global__ void k_restrict_ghost(LevelView<T> F, LevelView<T> C, T *__restrict__ gc) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= C.ng) return;
    int64_t rem = C.gnode[q], p = 0;
    if (D == 2) {
        const int64_t j0 = rem / C.s0, j1 = rem - j0 * C.s0;
        p = 2 * j0 * F.s0 + 2 * j1;
    } else {
        const int64_t j0 = rem / C.s0;
        rem -= j0 * C.s0;
        const int64_t j1 = rem / C.s1, j2 = rem - j1 * C.s1;
        p = 2 * j0 * F.s0 + 2 * j1 * F.s1 + 2 * j2;
    }
    gc[q] = partial_transfer<T, D>(F, p, false);
}

// extension + partial transfer at the coarse ghosts as one sparse map from
// the fine ghost defects (read from the fine defect grid)
template <typename T>
__global__ void k_ghost_transfer(const T *__restrict__ rf, const int32_t *__restrict__ fgnode,
                                 const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                 const T *__restrict__ val, T *__restrict__ gc, int ngc) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= ngc) return;
    T s = 0;
    for (int j = ptr[q]; j < ptr[q + 1]; j++) s += val[j] * rf[fgnode[col[j]]];
    gc[q] = s;
}

// ------------------------------------------------------------ interpolation
// Bilinear / trilinear interpolation onto Omega_h u Gamma_h (Sec. 2.6),
// weights renormalised over the parents in Omega_2h u Gamma_2h.
template <typename T, int D>
__global__ void k_prolong(LevelView<T> F, LevelView<T> C, const T *__restrict__ e, T *__restrict__ out, bool add) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= F.nn) return;
    const uint8_t k = F.type[p] & NODE_KIND;
    if (k != NODE_IN && k != NODE_GHOST) {
        if (!add) out[p] = 0;
        return;
    }
    int j[3] = {0, 0, 0};
    int64_t rem = p;
    j[0] = (int)(rem / F.s0);
    rem -= (int64_t)j[0] * F.s0;
    if (D == 2) {
        j[1] = (int)rem;
    } else {
        j[1] = (int)(rem / F.s1);
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
                const T w = (T)(1.0 / (n1 * n2 * n3));
                num += w * e[X];
                den += w;
            }
    const T val = den > (T)0 ? num / den : (T)0;
    if (add) out[p] += val;
    else out[p] = val;
}

// --------------------------------------------------------------- coarsest
// e = A^-1 b on the coarsest level: b gathered from f (inside) and the ghost
// data; each warp computes rows of the dense inverse product.
template <typename T>
__global__ void k_coarse_solve(LevelView<T> v, const int32_t *__restrict__ unk_node,
                               const int32_t *__restrict__ unk_ghost, const T *__restrict__ Ainv, int m) {
    extern __shared__ unsigned char smem_raw[];
    T *b = reinterpret_cast<T *>(smem_raw);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int g = unk_ghost[i];
        b[i] = g < 0 ? v.f[unk_node[i]] : v.gg[g];
    }
    __syncthreads();
    const int warps = blockDim.x >> 5;
    const int lane = threadIdx.x & 31;
    for (int row = blockIdx.x * warps + (threadIdx.x >> 5); row < m; row += gridDim.x * warps) {
        const T *a = Ainv + (int64_t)row * m;
        T s = 0;
        for (int k = lane; k < m; k += 32) s += a[k] * b[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) v.u[unk_node[row]] = s;
    }
}

// ------------------------------------------------------- mixed precision
// FP64 defect -> FP32 right-hand side of the correction problem
__global__ void k_defect_to_f32(const uint8_t *__restrict__ type, const double *__restrict__ r64, float *__restrict__ f32,
                                int64_t nn) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nn) return;
    f32[p] = ((type[p] & NODE_KIND) == NODE_IN) ? (float)r64[p] : 0.0f;
}

__global__ void k_ghost_defect_to_f32(const int32_t *__restrict__ gnode, const double *__restrict__ r64,
                                      float *__restrict__ g32, int ng) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < ng) g32[q] = (float)r64[gnode[q]];
}

// u64 += e32 on Omega_h u Gamma_h
__global__ void k_add_correction(const uint8_t *__restrict__ type, double *__restrict__ u64, const float *__restrict__ e32,
                                 int64_t nn) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nn) return;
    const uint8_t k = type[p] & NODE_KIND;
    if (k == NODE_IN || k == NODE_GHOST) u64[p] += (double)e32[p];
}

// keep u = 0 off Omega_h u Gamma_h
template <typename T>
__global__ void k_mask_unknowns(const uint8_t *__restrict__ type, T *__restrict__ u, int64_t nn) {
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
    if (dim == 2) k_rb_interior<T, 2><<<blocks_for((int64_t)v.n * hc), kThreads, 0, s>>>(v, color);
    else k_rb_interior<T, 3><<<blocks_for((int64_t)v.n * v.n * hc), kThreads, 0, s>>>(v, color);
}

template <typename T>
void launch_rb_fused2d(const LevelView<T> &v, const int32_t *tiles, int ntiles, cudaStream_t s) {
    if (ntiles <= 0) return;
    g_launches++;
    k_rb_fused2d<T><<<ntiles, 256, 0, s>>>(v, tiles);
}

template <typename T>
void launch_rb_list(const LevelView<T> &v, int dim, const int32_t *list, int cnt, cudaStream_t s) {
    if (cnt <= 0) return;
    g_launches++;
    if (dim == 2) k_rb_list<T, 2><<<blocks_for(cnt), kThreads, 0, s>>>(v, list, cnt);
    else k_rb_list<T, 3><<<blocks_for(cnt), kThreads, 0, s>>>(v, list, cnt);
}

template <typename T>
void launch_ghost_relax(const LevelView<T> &v, int dim, cudaStream_t s) {
    if (v.ng <= 0) return;
    g_launches += 2;
    if (dim == 2) k_ghost_new<T, 9><<<blocks_for(v.ng), kThreads, 0, s>>>(v);
    else k_ghost_new<T, 27><<<blocks_for(v.ng), kThreads, 0, s>>>(v);
    k_ghost_store<T><<<blocks_for(v.ng), kThreads, 0, s>>>(v);
}

template <typename T>
void launch_ghost_relax_list(const LevelView<T> &v, int dim, const int32_t *list, int cnt, cudaStream_t s) {
    if (cnt <= 0) return;
    g_launches += 2;
    if (dim == 2) k_ghost_new_list<T, 9><<<blocks_for(cnt), kThreads, 0, s>>>(v, list, cnt);
    else k_ghost_new_list<T, 27><<<blocks_for(cnt), kThreads, 0, s>>>(v, list, cnt);
    k_ghost_store_list<T><<<blocks_for(cnt), kThreads, 0, s>>>(v, list, cnt);
}

template <typename T>
void launch_defect(const LevelView<T> &v, int dim, bool zero_rest, unsigned long long *norm, cudaStream_t s) {
    g_launches += v.ng > 0 ? 2 : 1;
    if (dim == 2) k_defect_interior<T, 2><<<blocks_for(v.nn), kThreads, 0, s>>>(v, zero_rest, norm);
    else k_defect_interior<T, 3><<<blocks_for(v.nn), kThreads, 0, s>>>(v, zero_rest, norm);
    if (v.ng > 0) {
        if (dim == 2) k_defect_ghost<T, 9><<<blocks_for(v.ng), kThreads, 0, s>>>(v, norm);
        else k_defect_ghost<T, 27><<<blocks_for(v.ng), kThreads, 0, s>>>(v, norm);
    }
}

template <typename T>
void launch_extend(T *r, const DevGeom &g, const T *ew, cudaStream_t s) {
    for (size_t w = 1; w < g.wave.size(); w++) {
        const int b = g.wave[w - 1], e = g.wave[w];
        if (e > b) g_launches++;
        if (e > b) k_extend<T><<<blocks_for(e - b), kThreads, 0, s>>>(r, g.enode, g.ecnt, g.esrc, ew, g.ne, b, e);
    }
}

template <typename T>
void launch_restrict_interior(const LevelView<T> &F, const LevelView<T> &C, int dim, T *fc, cudaStream_t s) {
    g_launches++;
    if (dim == 2) k_restrict_interior<T, 2><<<blocks_for(C.nn), kThreads, 0, s>>>(F, C, fc);
    else k_restrict_interior<T, 3><<<blocks_for(C.nn), kThreads, 0, s>>>(F, C, fc);
}

template <typename T>
void launch_restrict(const LevelView<T> &F, const LevelView<T> &C, int dim, T *fc, T *gc, cudaStream_t s) {
    g_launches += C.ng > 0 ? 2 : 1;
    if (dim == 2) {
        k_restrict_interior<T, 2><<<blocks_for(C.nn), kThreads, 0, s>>>(F, C, fc);
        if (C.ng > 0) k_restrict_ghost<T, 2><<<blocks_for(C.ng), kThreads, 0, s>>>(F, C, gc);
    } else {
        k_restrict_interior<T, 3><<<blocks_for(C.nn), kThreads, 0, s>>>(F, C, fc);
        if (C.ng > 0) k_restrict_ghost<T, 3><<<blocks_for(C.ng), kThreads, 0, s>>>(F, C, gc);
    }
}

template <typename T>
void launch_ghost_transfer(const T *rf, const int32_t *fgnode, const int32_t *ptr, const int32_t *col, const T *val,
                           T *gc, int ngc, cudaStream_t s) {
    if (ngc <= 0) return;
    g_launches++;
    k_ghost_transfer<T><<<blocks_for(ngc), kThreads, 0, s>>>(rf, fgnode, ptr, col, val, gc, ngc);
}

template <typename T>
void launch_prolong(const LevelView<T> &F, const LevelView<T> &C, int dim, const T *e, T *out, bool add,
                    cudaStream_t s) {
    g_launches++;
    if (dim == 2) k_prolong<T, 2><<<blocks_for(F.nn), kThreads, 0, s>>>(F, C, e, out, add);
    else k_prolong<T, 3><<<blocks_for(F.nn), kThreads, 0, s>>>(F, C, e, out, add);
}

template <typename T>
void launch_coarse_solve(const LevelView<T> &v, const DevGeom &g, const T *Ainv, cudaStream_t s) {
    const int m = g.nunk;
    if (m <= 0) return;
    g_launches++;
    const int threads = 512;
    const unsigned blocks = (unsigned)std::min(1024, (m + 15) / 16);
    k_coarse_solve<T><<<blocks, threads, (size_t)m * sizeof(T), s>>>(v, g.unk_node, g.unk_ghost, Ainv, m);
}

template <typename T>
size_t local_smem_bytes(const LocalView<T> &J, int dim) {
    const int K = dim == 2 ? 9 : 27;
    return sizeof(T) * ((size_t)J.max_nodes + (size_t)(K + 3) * J.max_gh) + sizeof(int) * (size_t)(K + 1) * J.max_gh;
}

bool local_fits_registers(int max_int_per_colour) { return max_int_per_colour <= LOCAL_THREADS * LOCAL_EPT; }

template <typename T>
void launch_local(const LocalView<T> &J, int dim, int lead_ghost, int reps, cudaStream_t s) {
    if (J.ncomp <= 0 || (reps <= 0 && !lead_ghost)) return;
    g_launches++;
    const size_t smem = local_smem_bytes(J, dim);
    if (dim == 2) k_local<T, 2><<<J.ncomp, LOCAL_THREADS, smem, s>>>(J, lead_ghost, reps);
    else k_local<T, 3><<<J.ncomp, LOCAL_THREADS, smem, s>>>(J, lead_ghost, reps);
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
    k_mask_unknowns<T><<<blocks_for(nn), kThreads, 0, s>>>(type, u, nn);
}

void launch_defect_to_f32(const DevGeom &g, const double *r64, float *f32, float *g32, cudaStream_t s) {
    g_launches += g.ng > 0 ? 2 : 1;
    k_defect_to_f32<<<blocks_for(g.nn), kThreads, 0, s>>>(g.type, r64, f32, g.nn);
    if (g.ng > 0) k_ghost_defect_to_f32<<<blocks_for(g.ng), kThreads, 0, s>>>(g.gnode, r64, g32, g.ng);
}

void launch_add_correction(const DevGeom &g, double *u64, const float *e32, cudaStream_t s) {
    g_launches++;
    k_add_correction<<<blocks_for(g.nn), kThreads, 0, s>>>(g.type, u64, e32, g.nn);
}

#define GCMG_INSTANTIATE(T)                                                                              \
    template void launch_rb<T>(const LevelView<T> &, int, int, cudaStream_t);                            \
    template void launch_rb_list<T>(const LevelView<T> &, int, const int32_t *, int, cudaStream_t);     \
    template void launch_rb_fused2d<T>(const LevelView<T> &, const int32_t *, int, cudaStream_t);       \
    template void launch_ghost_relax<T>(const LevelView<T> &, int, cudaStream_t);                         \
    template void launch_ghost_relax_list<T>(const LevelView<T> &, int, const int32_t *, int, cudaStream_t); \
    template void launch_defect<T>(const LevelView<T> &, int, bool, unsigned long long *, cudaStream_t); \
    template void launch_extend<T>(T *, const DevGeom &, const T *, cudaStream_t);                        \
    template void launch_restrict<T>(const LevelView<T> &, const LevelView<T> &, int, T *, T *, cudaStream_t); \
    template void launch_restrict_interior<T>(const LevelView<T> &, const LevelView<T> &, int, T *, cudaStream_t); \
    template void launch_ghost_transfer<T>(const T *, const int32_t *, const int32_t *, const int32_t *, const T *, \
                                           T *, int, cudaStream_t);                                              \
    template void launch_prolong<T>(const LevelView<T> &, const LevelView<T> &, int, const T *, T *, bool,  \
                                    cudaStream_t);                                                       \
    template void launch_coarse_solve<T>(const LevelView<T> &, const DevGeom &, const T *, cudaStream_t); \
    template void launch_mask_unknowns<T>(const uint8_t *, T *, int64_t, cudaStream_t);            \
    template size_t local_smem_bytes<T>(const LocalView<T> &, int);                                 \
    template void launch_local<T>(const LocalView<T> &, int, int, int, cudaStream_t);               \
    template void local_prepare<T>(int, size_t);

GCMG_INSTANTIATE(float)
GCMG_INSTANTIATE(double)

}  // namespace gcmg
