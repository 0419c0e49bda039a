// Device kernels of one multigrid level, templated on the precision T and
// the dimension D.  Grids are dense C-ordered n^D arrays (last axis
// contiguous); ghost records are slot-major so that consecutive threads read
// consecutive words.
#include <cuda_runtime.h>

#include <atomic>

#include "gcmg_internal.h"
#include "kernels.h"
#include "kernels_dev.cuh"

namespace gcmg {

std::atomic<long long> g_launches{0};

namespace {

using namespace dev;
constexpr int kThreads = 256;

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
    if (!decode_colour<D>(v.n, color, t, v.s0, v.s1, p)) return;
    if ((v.type[p] & NODE_KIND) != NODE_IN) return;
    const T s = v.h2 * v.f[p] + neighbour_sum<T, D>(v.u, p, v.s0, v.s1);
    v.u[p] = s * (T)(1.0 / (2 * D));
}

// both colours in one pass over the active 2D tiles
template <typename T, int TR, int TC>
__global__ void __launch_bounds__(256) k_rb_fused2d(LevelView<T> v, T *__restrict__ out,
                                                    const int32_t *__restrict__ tiles) {
    pdl_wait();
    rb_fused2d_body<T, TR, TC>(v, out, tiles[blockIdx.x]);
}

// Same update over a compact list of band nodes of one colour (Sec. 3.2).
template <typename T, int D>
__global__ void k_rb_list(LevelView<T> v, const int32_t *__restrict__ list, int cnt) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int64_t p = list[i];
    const T s = v.h2 * v.f[p] + neighbour_sum<T, D>(v.u, p, v.s0, v.s1);
    v.u[p] = s * (T)(1.0 / (2 * D));
}

// Ghost relaxation, Eqs. (dir2d)/(neu2d): new value from the current values.
template <typename T, int K>
__global__ void k_ghost_new(LevelView<T> v) {
    pdl_wait();
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
    pdl_wait();
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
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int q = list[i];
    v.u[v.gnode[q]] = v.gtmp[q];
}

template <typename T>
__global__ void k_ghost_store(LevelView<T> v) {
    pdl_wait();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= v.ng) return;
    v.u[v.gnode[q]] = v.gtmp[q];
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
template <typename T, int D>
__global__ void k_defect_interior(LevelView<T> v, bool zero_rest, unsigned long long *norm) {
    pdl_wait();
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const double val = p < v.nn ? defect_node<T, D>(v, p, zero_rest) : 0.0;
    reduce_norm(norm, val);
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
                          const T *__restrict__ val) {
    // FP32 instances let their dependents start now; FP64 ones do not (their
    // dependents are large FP64 launches whose early CTAs measured slower)
    if (sizeof(T) == 4) pdl_trigger();
    if (D == 3 || sizeof(T) == 8) {
        // the thread-per-index form: 3D ghost-transfer rows are long (tens
        // to hundreds of terms), where it measured 8x faster than a warp a
        // row; in FP64 the terms are plain reads of r
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
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < F.nn) prolong_node_early<T, D>(F, C, e, out, add, p);   // waits after reading the types
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
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double val = 0.0;
    if (p < v.nn) {
        val = defect_node<double, D>(v, p, false);   // 0 off Omega_h
        f32[p] = (float)val;
        e32[p] = 0.0f;
    }
    reduce_norm(norm, val);
}

// ... and its ghost rows: the ghost defects rounded to FP32
template <int K>
__global__ void k_defect_ghost_mixed(LevelView<double> v, unsigned long long *norm, float *__restrict__ g32) {
    pdl_trigger();
    pdl_wait();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    double val = 0.0;
    if (q < v.ng) {
        val = defect_ghost_item<double, K>(v, q);
        g32[q] = (float)val;
    }
    reduce_norm(norm, val);
}

// u64 += e32 on Omega_h u Gamma_h
__global__ void k_add_correction(const uint8_t *__restrict__ type, double *__restrict__ u64, const float *__restrict__ e32,
                                 int64_t nn) {
    pdl_trigger();
    pdl_wait();
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nn) return;
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
template <typename T, int SR>
__global__ void __launch_bounds__(128) k_rb_strip(LevelView<T> v, T *__restrict__ out,
                                                  const int32_t *__restrict__ strips, int ns) {
    pdl_wait();
    const int s = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (s < ns) rb_strip<T, SR>(v, out, strips[s]);   // uniform over the warp
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

template <typename T>
void launch_rb_list(const LevelView<T> &v, int dim, const int32_t *list, int cnt, cudaStream_t s) {
    if (cnt <= 0) return;
    g_launches++;
    if (dim == 2) pdl_launch(k_rb_list<T, 2>, dim3(blocks_for(cnt)), dim3(kThreads), 0, s, v, list, cnt);
    else pdl_launch(k_rb_list<T, 3>, dim3(blocks_for(cnt)), dim3(kThreads), 0, s, v, list, cnt);
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
    if (dim == 2) pdl_launch(k_defect_interior<T, 2>, dim3(blocks_for(v.nn)), dim3(kThreads), 0, s, v, zero_rest, norm);
    else pdl_launch(k_defect_interior<T, 3>, dim3(blocks_for(v.nn)), dim3(kThreads), 0, s, v, zero_rest, norm);
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
                    T *uc, cudaStream_t s) {
    const int64_t n = (gf.dim == 3 || sizeof(T) == 8) ? std::max<int64_t>(C.nn, C.ng) : C.nn + 32 * (int64_t)C.ng;
    constexpr bool from_r = sizeof(T) == 8;   // FP64: one defect pass first (see descend_item)
    if (from_r) launch_defect<T>(F, gf.dim, false, nullptr, s);
    g_launches++;
    if (gf.dim == 2)
        pdl_launch(k_descend<T, 2, from_r>, dim3(blocks_for(n)), dim3(kThreads), 0, s, F, C, fc, gc, uc, gf.gt_ptr, gf.gt_col, gt_val);
    else
        pdl_launch(k_descend<T, 3, from_r>, dim3(blocks_for(n)), dim3(kThreads), 0, s, F, C, fc, gc, uc, gf.gt_ptr, gf.gt_col, gt_val);
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
    if (dim == 2) pdl_launch(k_prolong<T, 2>, dim3(blocks_for(F.nn)), dim3(kThreads), 0, s, F, C, e, out, add);
    else pdl_launch(k_prolong<T, 3>, dim3(blocks_for(F.nn)), dim3(kThreads), 0, s, F, C, e, out, add);
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
    if (dim == 2) pdl_launch(k_defect_interior_mixed<2>, dim3(blocks_for(v.nn)), dim3(kThreads), 0, s, v, norm, f32, e32);
    else pdl_launch(k_defect_interior_mixed<3>, dim3(blocks_for(v.nn)), dim3(kThreads), 0, s, v, norm, f32, e32);
    if (v.ng > 0) {
        if (dim == 2) pdl_launch(k_defect_ghost_mixed<9>, dim3(blocks_for(v.ng)), dim3(kThreads), 0, s, v, norm, g32);
        else pdl_launch(k_defect_ghost_mixed<27>, dim3(blocks_for(v.ng)), dim3(kThreads), 0, s, v, norm, g32);
    }
}

void launch_add_correction(const DevGeom &g, double *u64, const float *e32, cudaStream_t s) {
    g_launches++;
    pdl_launch(k_add_correction, dim3(blocks_for(g.nn)), dim3(kThreads), 0, s, g.type, u64, e32, g.nn);
}

#define GCMG_INSTANTIATE(T)                                                                              \
    template void launch_rb<T>(const LevelView<T> &, int, int, cudaStream_t);                            \
    template void launch_rb_list<T>(const LevelView<T> &, int, const int32_t *, int, cudaStream_t);     \
    template void launch_rb_fused2d<T>(const LevelView<T> &, T *, const int32_t *, int, cudaStream_t);  \
    template void launch_rb_strip<T>(const LevelView<T> &, T *, const DevGeom &, cudaStream_t);           \
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
    template void launch_junction_solve<T>(const LevelView<T> &, const DevGeom &, const T *, T *, cudaStream_t, \
                                           const LocalView<T> *);                                                \
    template void launch_descend<T>(const LevelView<T> &, const LevelView<T> &, const DevGeom &, const T *, T *, T *, \
                                    T *, cudaStream_t);                                                            \
    template void launch_mask_unknowns<T>(const uint8_t *, T *, int64_t, cudaStream_t);            \
    template size_t local_smem_bytes<T>(const LocalView<T> &, int, bool);                                 \
    template void launch_local<T>(const LocalView<T> &, int, int, int, cudaStream_t);               \
    template void launch_local_copyback<T>(const LocalView<T> &, cudaStream_t);                      \
    template void local_prepare<T>(int, size_t);

GCMG_INSTANTIATE(float)
GCMG_INSTANTIATE(double)

}  // namespace gcmg
