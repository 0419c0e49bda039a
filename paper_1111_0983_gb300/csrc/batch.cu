// Batched multi-domain solves (gcmg_batch_*): many independent 2D domains of
// uneven grid sizes advance together.  Every step of the cycle is ONE kernel
// launch over all domains: each CTA reads a (view, start) item naming the
// domain level and the tile / component / node range it works on, and runs the
// same device body as the single-domain kernels (kernels_dev.cuh).  Levels are
// aligned by depth from the coarsest grid, so a 129^2 domain joins the descent
// later than a 1025^2 one; each domain still follows its own V-cycle.  The
// whole solve (FP32 cycles inside FP64 iterative refinement, per-domain
// convergence) is captured once into a CUDA graph with a device-side while
// loop.  The fused interior sweep comes in several tile shapes; the autotuner
// times them on the batch and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "ctx.h"
#include "gcmg_internal.h"
#include "kernels.h"
#include "kernels_dev.cuh"

using namespace gcmg;
using namespace gcmg::dev;

namespace {

struct BItem {
    int32_t view;    // index into the view table
    int32_t start;   // tile / component / first node / first ghost / block
};

// the junction-solve product of up to kJsRows rows of one component of one
// domain level, with every address resolved on the host
struct JsItem {
    const float *a;          // the first row of the chunk in the component's padded inverse
    const float *r;          // the component's padded defect vector
    const int32_t *node;     // the chunk's row nodes
    float *u0, *u1;          // the level's two u grids
    int rows, mp, dom, pad;  // rows of the chunk, padded row length, domain
};


// one level of one domain, in FP32 (the cycle precision of the batch)
struct BView32 {
    LevelView<float> v;      // this level (v.u: its first u grid)
    float *u2, *c_u2;        // second u grids of this level and of the next coarser one
    LevelView<float> c;      // next coarser level (when it exists)
    float *cf, *cg;          // coarser level's f and ghost data (restriction targets)
    const int32_t *tiles;    // active sweep strips of the selected height
    int ntiles;
    LocalView<float> bz, jz; // boundary blocks, junction zone
    const int32_t *gt_ptr, *gt_col;
    const float *gt_val;
    const int32_t *unk_node, *unk_ghost;
    const float *Ainv;
    int nunk;
    int dom;
    const int *active;       // per-domain flag: still iterating
    // exact junction solve of this level
    const int32_t *js_node, *js_ghost, *js_comp, *js_off, *js_roff, *js_rpos;
    const int64_t *js_aoff;
    const float *js_inv;
    float *js_r;
    int js_n;
};

// level 0 of one domain in FP64 plus its FP32 correction arrays
struct BView64 {
    LevelView<double> v;
    float *f32, *g32, *e32, *e32b;   // e32b: level 0's second FP32 grid
    int dom;
    const int *active;
};

constexpr int kThreads = 256;

// A dense item covers npt * kThreads consecutive indexes (nodes, ghosts,
// rows): thread t takes start + e * kThreads + t for e < npt.  npt is chosen
// per launch (launch argument): large launches take several indexes a thread
// so that the chain item -> view -> active flag is paid once for all of them.
template <class F>
__device__ __forceinline__ void for_span(const BItem &b, int npt, F &&f) {
    for (int e = 0; e < npt; e++) f((int64_t)b.start + (int64_t)e * kThreads + threadIdx.x);
}
constexpr int kCoarseBlocks = 4;     // CTAs per domain for the coarsest solve
constexpr int kVariants = 3;         // rows of the sweep strips (STRIP_W owned columns each)
const int kStripRows[kVariants] = {8, 16, 32};

// ---------------------------------------------------------------- kernels
// Launch argument `cur` / `src`: which of the level's two u grids holds u
// (0: v.u, 1: u2); the sweep reads that grid and writes the other.
__device__ __forceinline__ float *ugrid(const BView32 &w, int k) { return k ? w.u2 : w.v.u; }

// both colours of the sweep: an item is 4 consecutive strips of one view, one a warp
template <int SR>
__global__ void __launch_bounds__(128, 8) kb_fused(const BView32 *__restrict__ V, const BItem *__restrict__ it, int src) {
    const BItem b = it[blockIdx.x];
    if (!V[b.view].active[V[b.view].dom]) return;
    const BView32 &w = V[b.view];
    const int s = b.start + (threadIdx.x >> 5);
    if (s >= w.ntiles) return;   // uniform over the warp
    LevelView<float> v = w.v;
    v.u = ugrid(w, src);
    rb_strip<float, SR>(v, ugrid(w, src ^ 1), w.tiles[s]);
}

__global__ void __launch_bounds__(256) kb_local_copyback(const BView32 *__restrict__ V, const BItem *__restrict__ it,
                                                         int cur, int npt) {
    const BItem b = it[blockIdx.x];
    if (!V[b.view].active[V[b.view].dom]) return;
    float *u = ugrid(V[b.view], cur);
    for_span(b, npt, [&](int64_t i) { local_copyback<float>(V[b.view].bz, u, (int)i); });
}

template <int EPT>
__global__ void __launch_bounds__(LOCAL_THREADS, 2) kb_local(const BView32 *__restrict__ V,
                                                             const BItem *__restrict__ it, int junction,
                                                             int lead_ghost, int reps, int cur) {
    const BItem b = it[blockIdx.x];
    if (!V[b.view].active[V[b.view].dom]) return;
    const LocalView<float> &J = junction ? V[b.view].jz : V[b.view].bz;
    float *u = ugrid(V[b.view], cur);
    local_body<float, 2, EPT>(J, u, J.wb ? J.wb : u, b.start, lead_ghost, reps);
}

// exact junction solve: defects of the solved equations (dense items), then
// u += A_ZZ^-1 r (kJsWarpRows rows a warp, kJsRows rows an item)
constexpr int kJsWarpRows = 4;
constexpr int kJsRows = 8 * kJsWarpRows;

// WB: the boundary blocks' write-back is performed here too (items cover
// max(js_n, nwb) indexes); the defects read the write-back nodes from the
// write-back grid
template <bool WB>
__global__ void kb_js_defect(const BView32 *__restrict__ V, const BItem *__restrict__ it, int cur, int npt) {
    const BItem b = it[blockIdx.x];
    if (!V[b.view].active[V[b.view].dom]) return;
    const BView32 &w = V[b.view];
    LevelView<float> v = w.v;
    v.u = ugrid(w, cur);
    for_span(b, npt, [&](int64_t k) {
        if (WB) local_copyback<float>(w.bz, v.u, (int)k);
        if (k < w.js_n) w.js_r[w.js_rpos[k]] = js_defect<float, 2, WB>(v, w.js_node[k], w.js_ghost[k], w.bz.wb);
    });
}

// one chunk a CTA, kJsWarpRows rows a warp (each lane sums its vectors of a
// row in index order, as js_apply_rows); chain: descriptor -> active flag -> rows
__global__ void __launch_bounds__(256) kb_js_apply_chunk(const JsItem *__restrict__ items,
                                                        const int *__restrict__ active, int cur) {
    const JsItem q = items[blockIdx.x];
    if (!active[q.dom]) return;
    using V = Vec16<float>::type;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = w * kJsWarpRows;
    const int nr = min(kJsWarpRows, q.rows - i0);
    if (nr <= 0) return;   // uniform over the warp
    const int nv = q.mp / 4;
    const V *a = reinterpret_cast<const V *>(q.a + (int64_t)i0 * q.mp);
    const V *rr = reinterpret_cast<const V *>(q.r);
    constexpr int U = 2;
    float s[kJsWarpRows] = {};
    for (int j0 = lane; j0 < nv; j0 += 32 * U) {
        V rv[U], av[kJsWarpRows][U];
#pragma unroll
        for (int e = 0; e < U; e++)
            if (j0 + 32 * e < nv) {
                rv[e] = rr[j0 + 32 * e];
#pragma unroll
                for (int i = 0; i < kJsWarpRows; i++)
                    if (i < nr) av[i][e] = a[(int64_t)i * nv + j0 + 32 * e];
            }
#pragma unroll
        for (int e = 0; e < U; e++)
            if (j0 + 32 * e < nv)
#pragma unroll
                for (int i = 0; i < kJsWarpRows; i++)
                    if (i < nr) s[i] = Vec16<float>::dot(s[i], av[i][e], rv[e]);
    }
    float *u = cur ? q.u1 : q.u0;
#pragma unroll
    for (int i = 0; i < kJsWarpRows; i++) {
        float t = s[i];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0 && i < nr) u[q.node[i0 + i]] += t;
    }
}

// defect, restriction with the coarse-ghost transfer, and zero coarse u in
// one pass over the coarser level's nodes and ghosts (fine u in grid `cur`,
// coarse u = 0 into its first grid)
__global__ void kb_descend(const BView32 *__restrict__ V, const BItem *__restrict__ it, int cur, int npt) {
    const BItem b = it[blockIdx.x];
    if (!V[b.view].active[V[b.view].dom]) return;
    const BView32 &w = V[b.view];
    LevelView<float> v = w.v;
    v.u = ugrid(w, cur);
    for_span(b, npt, [&](int64_t i) {
        descend_item<float, 2>(v, w.c, w.cf, w.cg, w.c.u, w.gt_ptr, w.gt_col, w.gt_val, i);
    });
}

// zero u of the view's level (coarse = 0) or of its coarser level (coarse = 1)
__global__ void kb_zero(const BView32 *__restrict__ V, const BItem *__restrict__ it, int coarse, int npt) {
    const BItem b = it[blockIdx.x];
    if (!V[b.view].active[V[b.view].dom]) return;
    const LevelView<float> &v = coarse ? V[b.view].c : V[b.view].v;
    for_span(b, npt, [&](int64_t p) { if (p < v.nn) v.u[p] = 0.f; });
}

__global__ void kb_prolong(const BView32 *__restrict__ V, const BItem *__restrict__ it, int cur, int ccur,
                           int npt) {
    const BItem b = it[blockIdx.x];
    if (!V[b.view].active[V[b.view].dom]) return;
    const BView32 &w = V[b.view];
    float *e = ccur ? w.c_u2 : w.c.u;
    float *u = ugrid(w, cur);
    for_span(b, npt, [&](int64_t p) { if (p < w.v.nn) prolong_node<float, 2>(w.v, w.c, e, u, true, p); });
}

__global__ void kb_coarse(const BView32 *__restrict__ V, const BItem *__restrict__ it) {
    const BItem b = it[blockIdx.x];
    if (!V[b.view].active[V[b.view].dom]) return;
    const BView32 &w = V[b.view];
    coarse_rows<float>(w.v, w.unk_node, w.unk_ghost, w.Ainv, w.nunk, b.start, kCoarseBlocks);
}

// FP64 level 0: defect with per-domain norms (nodes, then ghosts)
// largest |x| over a thread's indexes; NaN wins
__device__ __forceinline__ double max_abs(double m, double x) {
    double a = fabs(x);
    if (a != a) a = __longlong_as_double(0x7ff0000000000000ll);
    return a > m ? a : m;
}

__global__ void kb_defect64(const BView64 *__restrict__ V, const BItem *__restrict__ it, unsigned long long *norms,
                            int ghosts, int npt) {
    const BItem b = it[blockIdx.x];
    if (!V[b.view].active[V[b.view].dom]) return;   // uniform per block
    const LevelView<double> &v = V[b.view].v;
    double m = 0.0;
    if (!ghosts) {
        for_span(b, npt, [&](int64_t p) { if (p < v.nn) m = max_abs(m, defect_node<double, 2>(v, p, false)); });
    } else {
        for_span(b, npt, [&](int64_t q) { if (q < v.ng) m = max_abs(m, defect_ghost_item<double, 9>(v, (int)q)); });
    }
    reduce_norm(norms + V[b.view].dom, m);
}

// ||(f, g)|| per domain
__global__ void kb_rhs_norm(const BView64 *__restrict__ V, const BItem *__restrict__ it, unsigned long long *norms,
                            int ghosts, int npt) {
    const BItem b = it[blockIdx.x];
    const LevelView<double> &v = V[b.view].v;
    double m = 0.0;
    if (!ghosts) {
        for_span(b, npt, [&](int64_t p) { if (p < v.nn && (v.type[p] & NODE_KIND) == NODE_IN) m = max_abs(m, v.f[p]); });
    } else {
        for_span(b, npt, [&](int64_t q) { if (q < v.ng) m = max_abs(m, v.gg[q]); });
    }
    reduce_norm(norms + V[b.view].dom, m);
}

// FP64 defect -> FP32 right-hand side; e32 = 0
__global__ void kb_to_f32(const BView64 *__restrict__ V, const BItem *__restrict__ it, int ghosts, int npt) {
    const BItem b = it[blockIdx.x];
    if (!V[b.view].active[V[b.view].dom]) return;
    const BView64 &w = V[b.view];
    if (!ghosts) {
        for_span(b, npt, [&](int64_t p) {
            if (p >= w.v.nn) return;
            w.f32[p] = ((w.v.type[p] & NODE_KIND) == NODE_IN) ? (float)w.v.r[p] : 0.f;
            w.e32[p] = 0.f;
        });
    } else {
        for_span(b, npt, [&](int64_t q) { if (q < w.v.ng) w.g32[q] = (float)w.v.r[w.v.gnode[q]]; });
    }
}

// u64 += e32 on Omega_h u Gamma_h
__global__ void kb_add(const BView64 *__restrict__ V, const BItem *__restrict__ it, int cur, int npt) {
    const BItem b = it[blockIdx.x];
    if (!V[b.view].active[V[b.view].dom]) return;
    const BView64 &w = V[b.view];
    const float *e = cur ? w.e32b : w.e32;
    for_span(b, npt, [&](int64_t p) {
        if (p >= w.v.nn) return;
        const uint8_t k = w.v.type[p] & NODE_KIND;
        if (k == NODE_IN || k == NODE_GHOST) w.v.u[p] += (double)e[p];
    });
}

// end of one refinement step: per-domain relative residual, loop condition
// (graph mode: sets the while node's condition; plain launches: writes it to *go)
__global__ void kb_check(cudaGraphConditionalHandle h, const unsigned long long *norms, const double *r0, double *rel,
                         int *m, int *active, int *steps_of, int ndom, double rtol, int max_steps, int *go) {
    __shared__ int pending;
    if (threadIdx.x == 0) pending = 0;
    __syncthreads();
    const int k = *m + 1;
    for (int d = threadIdx.x; d < ndom; d += blockDim.x) {
        if (!active[d]) continue;    // converged earlier: its work is skipped
        const double v = __longlong_as_double((long long)norms[d]) / r0[d];
        if (k <= 256) rel[(size_t)d * 257 + k] = v;
        steps_of[d] = k;
        if (!(v <= rtol) && v == v && !isinf(v)) atomicAdd(&pending, 1);
        else active[d] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *m = k;
        const unsigned more = (pending > 0 && k < max_steps) ? 1u : 0u;
        if (go) *go = (int)more;
        else cudaGraphSetConditional(h, more);
    }
}


// a captured launch: kernel kind, item range and parameters
struct Launch {
    enum Kind { FUSED, BOUNDARY, BOUNDARY_COPY, JUNCTION, JS_DEFECT, JS_APPLY, DESCEND, PROLONG, COARSE, ZERO };
    Kind kind;
    size_t off, count;
    size_t smem;
    int cur = 0, ccur = 0;   // which u grid holds u (this level, the next coarser one)
    int npt = 1;             // indexes a thread of a dense item
    int ept = LOCAL_EPT;     // shared-memory programs: inside entries per thread and colour
};

}  // namespace

struct gcmg_batch {
    std::vector<gcmg_ctx *> doms;
    cudaStream_t stream = nullptr, gstream = nullptr;
    int device = 0;
    int variant = 0;
    int add_cur = 0;    // the u grid that holds level 0's correction after a cycle
    bool use_graph = true;   // false: the steps as plain launches (for profilers)
    int *d_go = nullptr;     // loop condition of the plain-launch form
    double rtol = 1e-10;
    int max_steps = 100;
    // device tables
    std::vector<std::vector<int>> view_of;    // [dom][level] -> view index
    BView32 *d_v32 = nullptr;
    BView64 *d_v64 = nullptr;
    BItem *d_items = nullptr;
    JsItem *d_jsitems = nullptr;              // junction-solve chunks (JS_APPLY launches)
    std::vector<int32_t *> tile_bufs;         // tile lists per view for the selected shape
    std::vector<Launch> cycle;                // FP32 V-cycle over all domains
    size_t items64_nodes = 0, items64_ghosts = 0, n_items64_nodes = 0, n_items64_ghosts = 0;
    int npt64_nodes = 1, npt64_ghosts = 1;
    unsigned long long *d_norms = nullptr;
    double *d_r0 = nullptr, *d_rel = nullptr;
    int *d_m = nullptr;
    int *d_active = nullptr, *d_steps = nullptr;   // per domain
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<int> versions;
    long long graph_kernels = 0;
    std::string err;
};

namespace {

gcmg_status bfail(gcmg_batch *b, gcmg_status s, const std::string &m) {
    if (b) b->err = m;
    return s;
}

#define BATCH_GUARD(b, ...)                                                                     \
    try {                                                                                        \
        __VA_ARGS__                                                                              \
    } catch (const CudaFail &f) {                                                                \
        cudaGetLastError();                                                                      \
        return bfail(b, GCMG_E_CUDA, std::string(f.what) + ": " + cudaGetErrorString(f.e));      \
    } catch (const GeomError &g) {                                                               \
        return bfail(b, GCMG_E_GEOM, g.msg);                                                     \
    } catch (const std::bad_alloc &) {                                                           \
        return bfail(b, GCMG_E_OOM, "allocation failed");                                        \
    }

void free_tables(gcmg_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    for (void *p : {(void *)b->d_v32, (void *)b->d_v64, (void *)b->d_items, (void *)b->d_jsitems}) cudaFree(p);
    b->d_v32 = nullptr;
    b->d_v64 = nullptr;
    b->d_items = nullptr;
    b->d_jsitems = nullptr;
    for (int32_t *t : b->tile_bufs) cudaFree(t);
    b->tile_bufs.clear();
    b->cycle.clear();
}

size_t smem_of(const LocalView<float> &J) {
    LocalView<float> tmp = J;
    return local_smem_bytes<float>(tmp, 2);
}

// Builds the view tables and the launch schedule of one FP32 V-cycle.
void build_tables(gcmg_batch *b) {
    free_tables(b);
    const int nd = (int)b->doms.size();
    std::vector<BView32> v32;
    std::vector<BView64> v64;
    std::vector<int> ntile;   // tiles per view
    b->view_of.assign(nd, {});
    int kmax = 0;
    const int rows = kStripRows[b->variant];
    for (int d = 0; d < nd; d++) {
        gcmg_ctx *c = b->doms[d];
        const int nl = (int)c->H.size();
        kmax = std::max(kmax, nl - 1);
        for (int l = 0; l < nl; l++) {
            BView32 w;
            std::memset(&w, 0, sizeof(w));
            w.v = view<float>(c, l, c->D32[l]);
            w.u2 = c->D32[l].u2;
            if (l + 1 < nl) {
                w.c = view<float>(c, l + 1, c->D32[l + 1]);
                w.c_u2 = c->D32[l + 1].u2;
                w.cf = c->D32[l + 1].f;
                w.cg = c->D32[l + 1].gg;
            }
            std::vector<int32_t> t = strips_for(c->H[l], rows);
            int32_t *dt = nullptr;
            ck(cudaMalloc(&dt, std::max<size_t>(t.size(), 1) * sizeof(int32_t)), "cudaMalloc");
            b->tile_bufs.push_back(dt);
            if (!t.empty()) ck(cudaMemcpy(dt, t.data(), t.size() * sizeof(int32_t), cudaMemcpyHostToDevice), "tiles");
            w.tiles = dt;
            w.ntiles = (int)t.size();
            ntile.push_back((int)t.size());
            w.bz = lview<float>(c->G[l].bz, w.v, c->D32[l].r);
            w.jz = lview<float>(c->G[l].jz, w.v);
            w.gt_ptr = c->G[l].gt_ptr;
            w.gt_col = c->G[l].gt_col;
            w.gt_val = c->D32[l].gt_val;
            w.unk_node = c->G[l].unk_node;
            w.unk_ghost = c->G[l].unk_ghost;
            w.Ainv = c->D32[l].Ainv;
            w.nunk = c->G[l].nunk;
            w.dom = d;
            w.active = b->d_active;
            w.js_n = c->G[l].js_n;
            w.js_node = c->G[l].js_node;
            w.js_ghost = c->G[l].js_ghost;
            w.js_comp = c->G[l].js_comp;
            w.js_off = c->G[l].js_off;
            w.js_aoff = c->G[l].js_aoff;
            w.js_roff = c->G[l].js_roff;
            w.js_rpos = c->G[l].js_rpos;
            w.js_inv = c->D32[l].js_inv;
            w.js_r = c->D32[l].js_r;
            b->view_of[d].push_back((int)v32.size());
            v32.push_back(w);
            if (!c->G[l].bz.in_smem || (c->p.junction_sweeps > 0 && c->G[l].jz.ncomp > 0 && !c->G[l].jz.in_smem))
                throw GeomError{"a batched domain needs shared-memory boundary and junction programs"};
        }
        BView64 w64;
        std::memset(&w64, 0, sizeof(w64));
        w64.v = view<double>(c, 0, c->D64[0]);
        w64.f32 = c->D32[0].f;
        w64.g32 = c->D32[0].gg;
        w64.e32 = c->D32[0].u;
        w64.e32b = c->D32[0].u2;
        w64.dom = d;
        w64.active = b->d_active;
        v64.push_back(w64);
    }
    // items
    std::vector<BItem> items;
    std::vector<JsItem> jsitems;
    // dense ranges of the launch being built; emit_dense turns them into
    // items of npt * kThreads indexes, npt doubling (up to 8) while the
    // launch keeps at least four waves of 8 CTAs on every SM
    int nsm = 0;
    ck(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device), "attr");
    const int64_t fill = (int64_t)nsm * 8 * 4;
    std::vector<std::pair<int, int64_t>> pending;
    auto dense = [&](int view, int64_t count) {
        if (count > 0) pending.push_back({view, count});
    };
    auto emit_dense = [&]() {
        int64_t blocks = 0;
        for (const auto &pc : pending) blocks += (pc.second + kThreads - 1) / kThreads;
        int npt = 1;
        while (npt < 8 && blocks / (2 * npt) >= fill) npt *= 2;
        for (const auto &pc : pending)
            for (int64_t s = 0; s < pc.second; s += (int64_t)kThreads * npt) items.push_back({pc.first, (int32_t)s});
        pending.clear();
        return npt;
    };
    // u grid per depth (every domain level at one depth has the same history)
    std::vector<int> cur(kmax + 1, 0);
    auto add_launch = [&](Launch::Kind k, size_t before, size_t smem, int cu = 0, int ccu = 0, int npt = 1) {
        if (items.size() > before) {
            Launch L{k, before, items.size() - before, smem};
            L.cur = cu;
            L.ccur = ccu;
            L.npt = npt;
            b->cycle.push_back(L);
        }
    };
    // a launch over the pending dense ranges
    auto add_dense = [&](Launch::Kind k, int cu = 0, int ccu = 0) {
        const size_t before = items.size();
        const int npt = emit_dense();
        add_launch(k, before, 0, cu, ccu, npt);
    };
    const gcmg_params &p0 = b->doms[0]->p;
    auto relax = [&](int k) {
        size_t s0 = items.size();
        for (int d = 0; d < nd; d++) {
            const int l = (int)b->doms[d]->H.size() - 1 - k;
            if (l < 0) continue;
            const int vi = b->view_of[d][l];
            for (int i = 0; i < ntile[vi]; i += 4) items.push_back({vi, (int32_t)i});
        }
        add_launch(Launch::FUSED, s0, 0, cur[k]);   // reads grid cur[k], writes the other
        cur[k] ^= 1;
        for (int which = 0; which < 2; which++) {
            s0 = items.size();
            size_t smem = 0;
            int most = 0;   // most inside entries of one colour in a component
            for (int d = 0; d < nd; d++) {
                const int l = (int)b->doms[d]->H.size() - 1 - k;
                if (l < 0) continue;
                const int vi = b->view_of[d][l];
                const LocalView<float> &J = which ? v32[vi].jz : v32[vi].bz;
                // junction sweeps only without the exact solve (as in a single solve)
                if (which && (b->doms[d]->p.junction_sweeps <= 0 || p0.junction_solve)) continue;
                for (int c = 0; c < J.ncomp; c++) items.push_back({vi, c});
                if (J.ncomp) smem = std::max(smem, smem_of(J));
                if (J.ncomp) most = std::max(most, J.max_colour);
            }
            const size_t ncycle = b->cycle.size();
            add_launch(which ? Launch::JUNCTION : Launch::BOUNDARY, s0, smem, cur[k]);
            if (b->cycle.size() > ncycle && most <= LOCAL_THREADS) b->cycle.back().ept = 1;
            if (!which && !p0.junction_solve) {   // the boundary blocks' write-back, once all have staged
                for (int d = 0; d < nd; d++) {
                    const int l = (int)b->doms[d]->H.size() - 1 - k;
                    if (l >= 0) dense(b->view_of[d][l], v32[b->view_of[d][l]].bz.nwb);
                }
                add_dense(Launch::BOUNDARY_COPY, cur[k]);
            }
        }
        if (p0.junction_solve) {
            // with the boundary blocks' write-back (all views of a batch have
            // boundary programs with a write-back grid)
            for (int d = 0; d < nd; d++) {
                const int l = (int)b->doms[d]->H.size() - 1 - k;
                if (l < 0) continue;
                const BView32 &w = v32[b->view_of[d][l]];
                dense(b->view_of[d][l], std::max<int64_t>(w.js_n, w.bz.wb ? w.bz.nwb : 0));
            }
            add_dense(Launch::JS_DEFECT, cur[k]);
            // chunks of at most kJsRows rows of one component, addresses resolved here
            const size_t j0 = jsitems.size();
            for (int d = 0; d < nd; d++) {
                const int l = (int)b->doms[d]->H.size() - 1 - k;
                if (l < 0) continue;
                gcmg_ctx *c = b->doms[d];
                const DevGeom &g = c->G[l];
                const DevData<float> &D = c->D32[l];
                const std::vector<int32_t> &off = c->H[l].js_off;
                for (int cc = 0; cc < g.js_ncomp; cc++) {
                    const int o = off[cc], m = off[cc + 1] - o, mp = (m + 3) & ~3;
                    for (int r0 = o; r0 < o + m; r0 += kJsRows) {
                        JsItem q{};
                        q.a = D.js_inv + g.js_aoff_h[cc] + (int64_t)(r0 - o) * mp;
                        q.r = D.js_r + g.js_roff_h[cc];
                        q.node = g.js_node + r0;
                        q.u0 = D.u;
                        q.u1 = D.u2;
                        q.rows = std::min(kJsRows, o + m - r0);
                        q.mp = mp;
                        q.dom = d;
                        jsitems.push_back(q);
                    }
                }
            }
            if (jsitems.size() > j0) {
                Launch L{Launch::JS_APPLY, j0, jsitems.size() - j0, 0};
                L.cur = cur[k];
                b->cycle.push_back(L);
            }
        }
    };
    // the cycle at depth k (0: the coarsest level of every domain), as cycle()
    // of a single domain: nu1 relaxations, the descent (the coarser level then
    // starts from u = 0 in its first grid), gamma visits of depth k - 1 (one
    // when that is the coarsest), the interpolation, nu2 relaxations
    auto visit = [&](auto &self, int k) -> void {
        if (k == 0) {
            for (int d = 0; d < nd; d++) dense(b->view_of[d].back(), b->doms[d]->H.back().nn);
            add_dense(Launch::ZERO);
            const size_t s0 = items.size();
            size_t smem = 0;
            for (int d = 0; d < nd; d++) {
                for (int blk = 0; blk < kCoarseBlocks; blk++) items.push_back({b->view_of[d].back(), blk});
                smem = std::max(smem, sizeof(float) * (size_t)v32[b->view_of[d].back()].nunk);
            }
            add_launch(Launch::COARSE, s0, smem);
            return;
        }
        for (int r = 0; r < p0.nu1; r++) relax(k);
        for (int d = 0; d < nd; d++) {
            const int l = (int)b->doms[d]->H.size() - 1 - k;
            if (l >= 0) dense(b->view_of[d][l], std::max<int64_t>(b->doms[d]->H[l + 1].nn, b->doms[d]->H[l + 1].ng()));
        }
        add_dense(Launch::DESCEND, cur[k]);
        cur[k - 1] = 0;
        const int gam = k - 1 == 0 ? 1 : p0.gamma;
        for (int g = 0; g < gam; g++) self(self, k - 1);
        for (int d = 0; d < nd; d++) {
            const int l = (int)b->doms[d]->H.size() - 1 - k;
            if (l >= 0) dense(b->view_of[d][l], b->doms[d]->H[l].nn);
        }
        add_dense(Launch::PROLONG, cur[k], cur[k - 1]);
        for (int r = 0; r < p0.nu2; r++) relax(k);
    };
    cur[kmax] = 0;   // level 0's correction starts from 0 in its first grid
    visit(visit, kmax);
    b->add_cur = cur[kmax];
    // FP64 level-0 items (view index = domain)
    b->items64_nodes = items.size();
    for (int d = 0; d < nd; d++) dense(d, b->doms[d]->H[0].nn);
    b->npt64_nodes = emit_dense();
    b->n_items64_nodes = items.size() - b->items64_nodes;
    b->items64_ghosts = items.size();
    for (int d = 0; d < nd; d++) dense(d, b->doms[d]->H[0].ng());
    b->npt64_ghosts = emit_dense();
    b->n_items64_ghosts = items.size() - b->items64_ghosts;
    ck(cudaMalloc(&b->d_v32, v32.size() * sizeof(BView32)), "cudaMalloc");
    ck(cudaMalloc(&b->d_v64, v64.size() * sizeof(BView64)), "cudaMalloc");
    ck(cudaMalloc(&b->d_items, std::max<size_t>(items.size(), 1) * sizeof(BItem)), "cudaMalloc");
    ck(cudaMemcpy(b->d_v32, v32.data(), v32.size() * sizeof(BView32), cudaMemcpyHostToDevice), "views");
    ck(cudaMemcpy(b->d_v64, v64.data(), v64.size() * sizeof(BView64), cudaMemcpyHostToDevice), "views");
    ck(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BItem), cudaMemcpyHostToDevice), "items");
    ck(cudaMalloc(&b->d_jsitems, std::max<size_t>(jsitems.size(), 1) * sizeof(JsItem)), "cudaMalloc");
    if (!jsitems.empty())
        ck(cudaMemcpy(b->d_jsitems, jsitems.data(), jsitems.size() * sizeof(JsItem), cudaMemcpyHostToDevice),
           "junction items");
    b->versions.clear();
    for (gcmg_ctx *c : b->doms) b->versions.push_back(c->version);
}

template <int SR>
void launch_fused(const gcmg_batch *b, const Launch &L, cudaStream_t s) {
    kb_fused<SR><<<(unsigned)L.count, 128, 0, s>>>(b->d_v32, b->d_items + L.off, L.cur);
}

void launch_one(const gcmg_batch *b, const Launch &L, cudaStream_t s) {
    const BItem *it = b->d_items + L.off;
    const unsigned n = (unsigned)L.count;
    const int junction_sweeps = b->doms[0]->p.junction_sweeps, lambda = b->doms[0]->p.lambda;
    switch (L.kind) {
        case Launch::FUSED:
            switch (kStripRows[b->variant]) {   // the height the strip lists were built with
                case 8: launch_fused<8>(b, L, s); break;
                case 16: launch_fused<16>(b, L, s); break;
                default: launch_fused<32>(b, L, s); break;
            }
            break;
        case Launch::BOUNDARY:
            if (L.ept == 1) kb_local<1><<<n, LOCAL_THREADS, L.smem, s>>>(b->d_v32, it, 0, 1, lambda, L.cur);
            else kb_local<LOCAL_EPT><<<n, LOCAL_THREADS, L.smem, s>>>(b->d_v32, it, 0, 1, lambda, L.cur);
            break;
        case Launch::BOUNDARY_COPY: kb_local_copyback<<<n, 256, 0, s>>>(b->d_v32, it, L.cur, L.npt); break;
        case Launch::JUNCTION:
            if (L.ept == 1) kb_local<1><<<n, LOCAL_THREADS, L.smem, s>>>(b->d_v32, it, 1, 0, junction_sweeps, L.cur);
            else kb_local<LOCAL_EPT><<<n, LOCAL_THREADS, L.smem, s>>>(b->d_v32, it, 1, 0, junction_sweeps, L.cur);
            break;
        case Launch::JS_DEFECT: kb_js_defect<true><<<n, kThreads, 0, s>>>(b->d_v32, it, L.cur, L.npt); break;
        case Launch::JS_APPLY:
            kb_js_apply_chunk<<<n, 256, 0, s>>>(b->d_jsitems + L.off, b->d_active, L.cur);
            break;
        case Launch::DESCEND: kb_descend<<<n, kThreads, 0, s>>>(b->d_v32, it, L.cur, L.npt); break;
        case Launch::ZERO: kb_zero<<<n, kThreads, 0, s>>>(b->d_v32, it, 0, L.npt); break;
        case Launch::COARSE: kb_coarse<<<n, 512, L.smem, s>>>(b->d_v32, it); break;
        case Launch::PROLONG: kb_prolong<<<n, kThreads, 0, s>>>(b->d_v32, it, L.cur, L.ccur, L.npt); break;
    }
}

// one refinement step of every domain, then the FP64 defect norms
void step_body(gcmg_batch *b, cudaStream_t s) {
    const BItem *in = b->d_items + b->items64_nodes, *ig = b->d_items + b->items64_ghosts;
    kb_to_f32<<<(unsigned)b->n_items64_nodes, kThreads, 0, s>>>(b->d_v64, in, 0, b->npt64_nodes);
    if (b->n_items64_ghosts)
        kb_to_f32<<<(unsigned)b->n_items64_ghosts, kThreads, 0, s>>>(b->d_v64, ig, 1, b->npt64_ghosts);
    for (const Launch &L : b->cycle) launch_one(b, L, s);
    kb_add<<<(unsigned)b->n_items64_nodes, kThreads, 0, s>>>(b->d_v64, in, b->add_cur, b->npt64_nodes);
    ck(cudaMemsetAsync(b->d_norms, 0, b->doms.size() * sizeof(unsigned long long), s), "memset");
    kb_defect64<<<(unsigned)b->n_items64_nodes, kThreads, 0, s>>>(b->d_v64, in, b->d_norms, 0, b->npt64_nodes);
    if (b->n_items64_ghosts)
            kb_defect64<<<(unsigned)b->n_items64_ghosts, kThreads, 0, s>>>(b->d_v64, ig, b->d_norms, 1, b->npt64_ghosts);
}

long long step_kernels(const gcmg_batch *b) {
    return (long long)b->cycle.size() + 4 + (b->n_items64_ghosts ? 2 : 0) + 1;
}

void build_graph(gcmg_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    ck(cudaGraphCreate(&b->graph, 0), "cudaGraphCreate");
    cudaGraphConditionalHandle h;
    ck(cudaGraphConditionalHandleCreate(&h, b->graph, 1, cudaGraphCondAssignDefault), "conditional handle");
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)] = {};
    cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(raw);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    ck(cudaGraphAddNode(&node, b->graph, nullptr, nullptr, 0, &np), "cudaGraphAddNode");
    cudaGraph_t body = np.conditional.phGraph_out[0];
    ck(cudaStreamBeginCaptureToGraph(b->gstream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
       "begin capture");
    try {
        step_body(b, b->gstream);
        kb_check<<<1, 256, 0, b->gstream>>>(h, b->d_norms, b->d_r0, b->d_rel, b->d_m, b->d_active, b->d_steps,
                                            (int)b->doms.size(), b->rtol, b->max_steps, nullptr);
    } catch (...) {
        cudaGraph_t dummy;
        cudaStreamEndCapture(b->gstream, &dummy);
        throw;
    }
    cudaGraph_t captured;
    ck(cudaStreamEndCapture(b->gstream, &captured), "end capture");
    ck(cudaGraphInstantiate(&b->gexec, b->graph, 0), "cudaGraphInstantiate");
    b->graph_kernels = step_kernels(b);
}

bool stale(const gcmg_batch *b) {
    if (!b->d_items || b->versions.size() != b->doms.size()) return true;
    for (size_t d = 0; d < b->doms.size(); d++)
        if (b->doms[d]->version != b->versions[d]) return true;
    return false;
}

}  // namespace

extern "C" {

gcmg_status gcmg_batch_create(int count, const gcmg_params *params, const double *const *phi_dev, void *stream,
                              gcmg_batch **out) {
    if (!out) return GCMG_E_ARG;
    *out = nullptr;
    if (count <= 0 || !params || !phi_dev) return GCMG_E_ARG;
    for (int i = 0; i < count; i++) {
        const gcmg_params &p = params[i];
        if (!phi_dev[i] || check_params(p) != GCMG_OK || p.dim != 2 || p.precision != 1 || p.gamma != params[0].gamma ||
            p.nu1 != params[0].nu1 || p.nu2 != params[0].nu2 || p.lambda != params[0].lambda ||
            p.junction_sweeps != params[0].junction_sweeps || p.junction_solve != params[0].junction_solve)
            return GCMG_E_ARG;
    }
    gcmg_batch *b = new (std::nothrow) gcmg_batch;
    if (!b) return GCMG_E_OOM;
    *out = b;
    b->stream = (cudaStream_t)stream;
    b->rtol = params[0].rtol;
    b->max_steps = params[0].max_cycles;
    BATCH_GUARD(b, {
        ck(cudaGetDevice(&b->device), "cudaGetDevice");
        // level sets to the host, then host geometry of all domains in parallel
        std::vector<std::vector<double>> phi(count);
        for (int i = 0; i < count; i++) {
            int64_t nn = (int64_t)params[i].n * params[i].n;
            phi[i].resize(nn);
            ck(cudaMemcpyAsync(phi[i].data(), phi_dev[i], nn * sizeof(double), cudaMemcpyDeviceToHost, b->stream),
               "phi");
        }
        ck(cudaStreamSynchronize(b->stream), "sync");
        std::vector<std::vector<HostLevel>> H(count);
        std::vector<std::string> errs(count);
        std::atomic<int> next{0};
        const unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (unsigned t = 0; t < nt; t++)
            pool.emplace_back([&]() {
                for (int i = next++; i < count; i = next++) {
                    try {
                        prepare_levels(params[i], phi[i].data(), H[i]);
                    } catch (const GeomError &g) {
                        errs[i] = g.msg;
                    } catch (const std::bad_alloc &) {
                        errs[i] = "allocation failed";
                    }
                }
            });
        for (auto &t : pool) t.join();
        for (int i = 0; i < count; i++)
            if (!errs[i].empty()) return bfail(b, GCMG_E_GEOM, "domain " + std::to_string(i) + ": " + errs[i]);
        for (int i = 0; i < count; i++) {
            gcmg_ctx *c = nullptr;
            const gcmg_status s = create_from_levels(params[i], std::move(H[i]), b->stream, &c);
            if (s != GCMG_OK) {
                const std::string m = c ? c->err : std::string("create failed");
                if (c) gcmg_destroy(c);
                return bfail(b, s, "domain " + std::to_string(i) + ": " + m);
            }
            b->doms.push_back(c);
        }
        // W-cycles: the schedule is built per depth from the coarsest level up, so a
        // domain with fewer levels would sit under a parent depth it does not have
        // and be cycled gamma times a step
        if (params[0].gamma > 1)
            for (gcmg_ctx *c : b->doms)
                if (c->H.size() != b->doms[0]->H.size())
                    return bfail(b, GCMG_E_ARG, "W-cycle batches need domains with the same number of levels");
        int smax = 0;
        ck(cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device), "attr");
        ck(cudaFuncSetAttribute(kb_local<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax), "attr");
        ck(cudaFuncSetAttribute(kb_local<LOCAL_EPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax), "attr");
        ck(cudaFuncSetAttribute(kb_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize, smax), "attr");
        ck(cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking), "cudaStreamCreate");
        ck(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming), "cudaEventCreate");
        ck(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming), "cudaEventCreate");
        ck(cudaMalloc(&b->d_norms, count * sizeof(unsigned long long)), "cudaMalloc");
        ck(cudaMalloc(&b->d_r0, count * sizeof(double)), "cudaMalloc");
        ck(cudaMalloc(&b->d_rel, (size_t)count * 257 * sizeof(double)), "cudaMalloc");
        ck(cudaMalloc(&b->d_m, sizeof(int)), "cudaMalloc");
        ck(cudaMalloc(&b->d_active, count * sizeof(int)), "cudaMalloc");
        ck(cudaMalloc(&b->d_steps, count * sizeof(int)), "cudaMalloc");
        ck(cudaMalloc(&b->d_go, sizeof(int)), "cudaMalloc");
        return GCMG_OK;
    })
}

void gcmg_batch_destroy(gcmg_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->gstream) cudaStreamSynchronize(b->gstream);
    free_tables(b);
    for (gcmg_ctx *c : b->doms) gcmg_destroy(c);
    for (void *p : {(void *)b->d_norms, (void *)b->d_r0, (void *)b->d_rel, (void *)b->d_m, (void *)b->d_active,
                    (void *)b->d_steps, (void *)b->d_go})
        cudaFree(p);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    delete b;
}

const char *gcmg_batch_last_error(const gcmg_batch *b) { return b ? b->err.c_str() : "null batch"; }

int gcmg_batch_size(const gcmg_batch *b) { return b ? (int)b->doms.size() : 0; }

gcmg_ctx *gcmg_batch_domain(gcmg_batch *b, int i) {
    return (b && i >= 0 && i < (int)b->doms.size()) ? b->doms[i] : nullptr;
}

gcmg_status gcmg_batch_set_graph(gcmg_batch *b, int on) {
    if (!b) return GCMG_E_ARG;
    b->use_graph = on != 0;
    return GCMG_OK;
}

gcmg_status gcmg_batch_set_tiles(gcmg_batch *b, int variant) {
    if (!b || variant < 0 || variant >= kVariants) return bfail(b, GCMG_E_ARG, "bad tile variant");
    if (b->variant != variant) {
        b->variant = variant;
        b->versions.clear();   // rebuild tables at the next solve
    }
    return GCMG_OK;
}

gcmg_status gcmg_batch_solve(gcmg_batch *b, gcmg_stats *stats, int *steps) {
    if (!b) return GCMG_E_ARG;
    for (gcmg_ctx *c : b->doms)
        if (!c->rhs_set) return bfail(b, GCMG_E_STATE, "gcmg_set_rhs has not been called for every domain");
    BATCH_GUARD(b, {
        ck(cudaSetDevice(b->device), "cudaSetDevice");
        {   // coarsest inverses out of date: rebuild on host threads, then upload
            std::vector<int> dirty;
            for (int d = 0; d < (int)b->doms.size(); d++)
                if (b->doms[d]->H.back().ainv_dirty) dirty.push_back(d);
            std::vector<std::string> errs(dirty.size());
            std::atomic<int> next{0};
            const unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
            std::vector<std::thread> pool;
            for (unsigned t = 0; t < nt; t++)
                pool.emplace_back([&]() {
                    for (int i = next++; i < (int)dirty.size(); i = next++) {
                        try {
                            build_coarse_inverse(b->doms[dirty[i]]->H.back());
                        } catch (const GeomError &g) {
                            errs[i] = g.msg;
                        }
                    }
                });
            for (auto &t : pool) t.join();
            for (size_t i = 0; i < dirty.size(); i++) {
                if (!errs[i].empty()) return bfail(b, GCMG_E_GEOM, "domain " + std::to_string(dirty[i]) + ": " + errs[i]);
                upload_inverse(b->doms[dirty[i]]);
            }
        }
        bool rebuilt = false;
        {   // exact junction solves out of date: rebuild on host threads, then upload
            std::vector<std::pair<int, int>> dirty;   // (domain, level)
            for (int d = 0; d < (int)b->doms.size(); d++) {
                gcmg_ctx *c = b->doms[d];
                if (!c->p.junction_solve) continue;
                for (int l = 0; l < (int)c->H.size(); l++)
                    if (c->H[l].js_dirty) dirty.push_back({d, l});
            }
            std::vector<std::string> errs(dirty.size());
            std::atomic<int> next{0};
            const unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
            std::vector<std::thread> pool;
            for (unsigned t = 0; t < nt; t++)
                pool.emplace_back([&]() {
                    for (int i = next++; i < (int)dirty.size(); i = next++) {
                        gcmg_ctx *c = b->doms[dirty[i].first];
                        try {
                            build_junction_solve(c->H[dirty[i].second], c->p.junction_radius);
                        } catch (const GeomError &g) {
                            errs[i] = g.msg;
                        }
                    }
                });
            for (auto &t : pool) t.join();
            for (size_t i = 0; i < dirty.size(); i++) {
                const int d = dirty[i].first, l = dirty[i].second;
                if (!errs[i].empty()) return bfail(b, GCMG_E_GEOM, "domain " + std::to_string(d) + ": " + errs[i]);
                upload_js(b->doms[d], l);
                b->doms[d]->H[l].js_dirty = false;
                rebuilt = true;
            }
        }
        if (rebuilt || stale(b)) {
            build_tables(b);
            build_graph(b);
        }
        const int nd = (int)b->doms.size();
        cudaStream_t s = b->stream;
        const BItem *in = b->d_items + b->items64_nodes, *ig = b->d_items + b->items64_ghosts;
        {   // every domain starts active; the step kernels skip the inactive ones
            std::vector<int> ones(nd, 1), zeros(nd, 0);
            ck(cudaMemcpyAsync(b->d_active, ones.data(), nd * sizeof(int), cudaMemcpyHostToDevice, s), "active");
            ck(cudaMemcpyAsync(b->d_steps, zeros.data(), nd * sizeof(int), cudaMemcpyHostToDevice, s), "steps");
            ck(cudaMemsetAsync(b->d_rel, 0, (size_t)nd * 257 * sizeof(double), s), "memset");
            ck(cudaStreamSynchronize(s), "sync");   // the staging vectors die at scope end
        }
        for (gcmg_ctx *c : b->doms)
            ck(cudaMemsetAsync(c->D64[0].u, 0, c->H[0].nn * sizeof(double), s), "memset");
        // ||r0|| = ||(f, g)|| per domain
        ck(cudaMemsetAsync(b->d_norms, 0, nd * sizeof(unsigned long long), s), "memset");
        kb_rhs_norm<<<(unsigned)b->n_items64_nodes, kThreads, 0, s>>>(b->d_v64, in, b->d_norms, 0, b->npt64_nodes);
        if (b->n_items64_ghosts)
            kb_rhs_norm<<<(unsigned)b->n_items64_ghosts, kThreads, 0, s>>>(b->d_v64, ig, b->d_norms, 1, b->npt64_ghosts);
        std::vector<unsigned long long> bits(nd);
        ck(cudaMemcpyAsync(bits.data(), b->d_norms, nd * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s), "r0");
        ck(cudaStreamSynchronize(s), "sync");
        std::vector<double> r0(nd);
        for (int d = 0; d < nd; d++) {
            std::memcpy(&r0[d], &bits[d], sizeof(double));
            if (!(r0[d] > 0.0)) r0[d] = 1.0;
        }
        ck(cudaMemcpyAsync(b->d_r0, r0.data(), nd * sizeof(double), cudaMemcpyHostToDevice, s), "r0");
        // defect of u = 0 (the FP64 defect every step starts from)
        ck(cudaMemsetAsync(b->d_norms, 0, nd * sizeof(unsigned long long), s), "memset");
        kb_defect64<<<(unsigned)b->n_items64_nodes, kThreads, 0, s>>>(b->d_v64, in, b->d_norms, 0, b->npt64_nodes);
        if (b->n_items64_ghosts)
            kb_defect64<<<(unsigned)b->n_items64_ghosts, kThreads, 0, s>>>(b->d_v64, ig, b->d_norms, 1, b->npt64_ghosts);
        ck(cudaGetLastError(), "kernel launch");
        const int zero = 0;
        ck(cudaMemcpyAsync(b->d_m, &zero, sizeof(int), cudaMemcpyHostToDevice, s), "m");
        ck(cudaEventRecord(b->ev_in, s), "event");
        ck(cudaStreamWaitEvent(b->gstream, b->ev_in, 0), "wait");
        if (b->use_graph) {
            ck(cudaGraphLaunch(b->gexec, b->gstream), "cudaGraphLaunch");
        } else {   // the same steps as plain launches, the loop condition read back each step
            for (int go = 1; go;) {
                step_body(b, b->gstream);
                kb_check<<<1, 256, 0, b->gstream>>>(cudaGraphConditionalHandle{}, b->d_norms, b->d_r0, b->d_rel,
                                                    b->d_m, b->d_active, b->d_steps, nd, b->rtol, b->max_steps,
                                                    b->d_go);
                ck(cudaMemcpyAsync(&go, b->d_go, sizeof(int), cudaMemcpyDeviceToHost, b->gstream), "go");
                ck(cudaStreamSynchronize(b->gstream), "sync");
            }
        }
        ck(cudaEventRecord(b->ev_out, b->gstream), "event");
        ck(cudaStreamWaitEvent(s, b->ev_out, 0), "wait");
        int m = 0;
        ck(cudaMemcpyAsync(&m, b->d_m, sizeof(int), cudaMemcpyDeviceToHost, s), "m");
        ck(cudaStreamSynchronize(s), "sync");
        g_launches += 4 + b->graph_kernels * m;
        std::vector<double> rel((size_t)nd * 257, 0.0);
        ck(cudaMemcpy(rel.data(), b->d_rel, rel.size() * sizeof(double), cudaMemcpyDeviceToHost), "rel");
        std::vector<int> steps_of(nd, 0);
        ck(cudaMemcpy(steps_of.data(), b->d_steps, nd * sizeof(int), cudaMemcpyDeviceToHost), "steps");
        bool all = true;
        for (int d = 0; d < nd; d++) {
            const int kept = std::min(steps_of[d], 256);
            const double last = kept > 0 ? rel[(size_t)d * 257 + kept] : 1.0;
            const bool ok = last <= b->rtol;
            all = all && ok;
            if (stats) {
                gcmg_stats &st = stats[d];
                std::memset(&st, 0, sizeof(st));
                st.cycles = steps_of[d];
                st.converged = ok ? 1 : 0;
                st.rel_residual = last;
                st.r0_norm = r0[d];
                st.rel[0] = 1.0;
                for (int k = 1; k <= kept; k++) st.rel[k] = rel[(size_t)d * 257 + k];
            }
        }
        if (steps) *steps = m;
        if (!all) return bfail(b, GCMG_E_NOCONV, "not every domain converged");
        return GCMG_OK;
    })
}

gcmg_status gcmg_batch_get_solution(gcmg_batch *b, int i, double *u_dev) {
    if (!b || i < 0 || i >= (int)b->doms.size() || !u_dev) return bfail(b, GCMG_E_ARG, "bad argument");
    BATCH_GUARD(b, {
        const gcmg_ctx *c = b->doms[i];
        ck(cudaMemcpyAsync(u_dev, c->D64[0].u, c->H[0].nn * sizeof(double), cudaMemcpyDeviceToDevice, b->stream),
           "copy");
        ck(cudaStreamSynchronize(b->stream), "sync");
        return GCMG_OK;
    })
}

// Times one batched sweep set (all relaxations of one cycle) for each tile
// shape and selects the fastest; ms[k] receives the time of shape k.
gcmg_status gcmg_batch_autotune(gcmg_batch *b, int *best, double *ms) {
    if (!b) return GCMG_E_ARG;
    BATCH_GUARD(b, {
        ck(cudaSetDevice(b->device), "cudaSetDevice");
        cudaEvent_t e0, e1;
        ck(cudaEventCreate(&e0), "event");
        ck(cudaEventCreate(&e1), "event");
        {   // time the sweeps of every domain
            std::vector<int> ones(b->doms.size(), 1);
            ck(cudaMemcpy(b->d_active, ones.data(), ones.size() * sizeof(int), cudaMemcpyHostToDevice), "active");
        }
        double bestms = 1e30;
        int bestv = b->variant;
        for (int v = 0; v < kVariants; v++) {
            b->variant = v;
            build_tables(b);
            for (int rep = 0; rep < 3; rep++) {   // warm-up, then timed twice
                ck(cudaEventRecord(e0, b->stream), "event");
                for (const Launch &L : b->cycle)
                    if (L.kind == Launch::FUSED) launch_one(b, L, b->stream);
                ck(cudaEventRecord(e1, b->stream), "event");
            }
            ck(cudaEventSynchronize(e1), "sync");
            float t = 0.f;
            ck(cudaEventElapsedTime(&t, e0, e1), "elapsed");
            ck(cudaGetLastError(), "kernel launch");
            if (ms) ms[v] = t;
            if (t < bestms) { bestms = t; bestv = v; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->variant = bestv;
        b->versions.clear();
        if (best) *best = bestv;
        return GCMG_OK;
    })
}

}  // extern "C"
