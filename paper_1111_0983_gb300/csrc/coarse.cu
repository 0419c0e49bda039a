// The coarse end of the V-cycle in one launch.  Below a few hundred nodes a
// side every step of the cycle is a small kernel whose cost is its launch and
// its single wave, the same on a 257^2 level as on a 65^2 one.  One cluster
// of CC_SIZE CTAs therefore runs the whole V-cycle from the first level with
// at most fused_coarse_n nodes a side down to the coarsest grid and back: the
// same device bodies as the per-level kernels (sweep tiles, boundary-block
// programs, junction-solve rows, the fused descent, the dense coarsest solve,
// the interpolation), in the same order, with a hardware cluster barrier
// where one step must see the previous one's writes.  The results equal the
// per-level launches' bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ctx.h"
#include "gcmg_internal.h"
#include "kernels.h"
#include "kernels_dev.cuh"

namespace gcmg {

namespace {

constexpr int CC_SIZE = 8;          // CTAs of the cluster (portable size)
constexpr int CC_THREADS = 512;     // = LOCAL_THREADS, for the boundary-block programs

struct CoarseLevel {
    LevelView<float> v;             // v.u = u0
    float *u0, *u1;                 // the two u grids: the sweep reads one and writes the other
    float *f, *gg;                  // writable views of v.f, v.gg (targets of the descent)
    LocalView<float> bz;
    const int32_t *tiles;
    int ntiles;
    int js_n;
    const int32_t *js_node, *js_ghost, *js_comp, *js_off, *js_roff, *js_rpos;
    const int64_t *js_aoff;
    const float *js_inv;
    float *js_r;
    const int32_t *gt_ptr, *gt_col;
    const float *gt_val;
    const int32_t *unk_node, *unk_ghost;
    const float *Ainv;
    int nunk;
};

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// one relaxation of level L (as relax() in api.cu) starting from grid `cur`:
// the fused interior sweep into the other grid, the ghost sweep + lambda band
// sweeps of the boundary blocks, the exact junction solve; returns the grid
// that holds u afterwards
__device__ int cc_relax(const CoarseLevel &L, int cur, int lambda, int rank) {
    LevelView<float> v = L.v;
    v.u = cur ? L.u1 : L.u0;
    float *out = cur ? L.u0 : L.u1;
    for (int t = rank; t < L.ntiles; t += CC_SIZE) {
        dev::rb_fused2d_body<float, TILE_R, TILE_C>(v, out, L.tiles[t]);
        __syncthreads();
    }
    cluster_barrier();
    v.u = out;
    const LocalView<float> &bz = L.bz;
    for (int cpt = rank; cpt < bz.ncomp; cpt += CC_SIZE) {
        dev::local_body<float, 2>(bz, out, bz.wb, cpt, 1, lambda);
        __syncthreads();
    }
    cluster_barrier();
    for (int i = rank * CC_THREADS + threadIdx.x; i < bz.nwb; i += CC_SIZE * CC_THREADS)
        dev::local_copyback<float>(bz, out, i);
    cluster_barrier();
    if (L.js_n > 0) {
        for (int k = rank * CC_THREADS + threadIdx.x; k < L.js_n; k += CC_SIZE * CC_THREADS)
            L.js_r[L.js_rpos[k]] = dev::js_defect<float, 2>(v, L.js_node[k], L.js_ghost[k]);
        cluster_barrier();
        constexpr int warps = CC_THREADS / 32;
        for (int row = rank * warps + (threadIdx.x >> 5); row < L.js_n; row += CC_SIZE * warps)
            dev::js_apply_row<float>(out, L.js_node, L.js_comp, L.js_off, L.js_aoff, L.js_roff, L.js_inv, L.js_r, row,
                                     threadIdx.x & 31);
        cluster_barrier();
    }
    return cur ^ 1;
}

constexpr int CC_MAX_LEVELS = 16;

// Every CTA takes every loop trip and every barrier: the control flow below
// depends only on the kernel arguments and the level table.  Each level is
// entered with u = 0 in grid u0 (written by the descent into it).
__global__ void __launch_bounds__(CC_THREADS, 1)
    k_coarse_cycle(const CoarseLevel *__restrict__ Ls, int nl, int nu1, int nu2, int lambda) {
    const int rank = blockIdx.x;    // the grid is one cluster
    const int stride = CC_SIZE * CC_THREADS;
    int cur[CC_MAX_LEVELS];
    for (int l = 0; l + 1 < nl; l++) {
        const CoarseLevel &F = Ls[l], &C = Ls[l + 1];
        cur[l] = 0;
        for (int k = 0; k < nu1; k++) cur[l] = cc_relax(F, cur[l], lambda, rank);
        LevelView<float> fv = F.v;
        fv.u = cur[l] ? F.u1 : F.u0;
        const int64_t n = C.v.nn > C.v.ng ? C.v.nn : C.v.ng;
        for (int64_t i = rank * CC_THREADS + threadIdx.x; i < n; i += stride)
            dev::descend_item<float, 2>(fv, C.v, C.f, C.gg, C.u0, F.gt_ptr, F.gt_col, F.gt_val, i);
        cluster_barrier();
    }
    const CoarseLevel &K = Ls[nl - 1];
    cur[nl - 1] = 0;
    dev::coarse_rows<float>(K.v, K.unk_node, K.unk_ghost, K.Ainv, K.nunk, rank, CC_SIZE);
    cluster_barrier();
    for (int l = nl - 2; l >= 0; l--) {
        const CoarseLevel &F = Ls[l], &C = Ls[l + 1];
        LevelView<float> fv = F.v, cv = C.v;
        fv.u = cur[l] ? F.u1 : F.u0;
        cv.u = cur[l + 1] ? C.u1 : C.u0;
        for (int64_t p = rank * CC_THREADS + threadIdx.x; p < F.v.nn; p += stride)
            dev::prolong_node<float, 2>(fv, cv, cv.u, fv.u, true, p);
        cluster_barrier();
        for (int k = 0; k < nu2; k++) cur[l] = cc_relax(F, cur[l], lambda, rank);
    }
}

}  // namespace

// Chooses the first level of the fused coarse cycle and uploads its level
// table; c->coarse_l0 = -1 when the per-level launches must be used (FP64 or
// 3D cycles, W-cycles, junction sweeps, programs that do not fit in shared
// memory, or fused_coarse_n = 0).
void coarse_prepare(gcmg_ctx *c) {
    c->coarse_l0 = -1;
    const int nl = (int)c->H.size();
    if (c->p.fused_coarse_n <= 0 || c->p.precision != 1 || c->p.dim != 2 || c->p.gamma != 1 || nl < 2) return;
    if (!c->p.junction_solve && c->p.junction_sweeps > 0) return;
    int l0 = -1;
    for (int l = 1; l < nl - 1; l++)
        if (c->H[l].n <= c->p.fused_coarse_n) {
            l0 = l;
            break;
        }
    if (l0 < 0 || nl - l0 > CC_MAX_LEVELS) return;
    std::vector<CoarseLevel> tab;
    size_t smem = 0;
    for (int l = l0; l < nl; l++) {
        const DevGeom &g = c->G[l];
        DevData<float> &D = c->D32[l];
        if (l + 1 < nl && g.ng > 0 && (g.bz.ncomp == 0 || !g.bz.in_smem)) return;
        CoarseLevel L{};
        L.v = view<float>(c, l, D);
        L.u0 = D.u;
        L.u1 = D.u2;
        L.f = D.f;
        L.gg = D.gg;
        L.bz = lview<float>(g.bz, L.v, D.r);
        L.tiles = g.tiles;
        L.ntiles = g.ntiles;
        L.js_n = c->p.junction_solve ? g.js_n : 0;
        L.js_node = g.js_node;
        L.js_ghost = g.js_ghost;
        L.js_comp = g.js_comp;
        L.js_off = g.js_off;
        L.js_aoff = g.js_aoff;
        L.js_roff = g.js_roff;
        L.js_rpos = g.js_rpos;
        L.js_inv = D.js_inv;
        L.js_r = D.js_r;
        L.gt_ptr = g.gt_ptr;
        L.gt_col = g.gt_col;
        L.gt_val = D.gt_val;
        L.unk_node = g.unk_node;
        L.unk_ghost = g.unk_ghost;
        L.Ainv = D.Ainv;
        L.nunk = g.nunk;
        if (l + 1 < nl && g.bz.ncomp > 0) smem = std::max(smem, local_smem_bytes<float>(L.bz, 2));
        if (l + 1 == nl) smem = std::max(smem, sizeof(float) * (size_t)g.nunk);
        tab.push_back(L);
    }
    int dev_max = 0;
    ck(cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device), "attr");
    cudaFuncAttributes fa{};
    ck(cudaFuncGetAttributes(&fa, k_coarse_cycle), "attr");
    if (smem + fa.sharedSizeBytes > (size_t)dev_max) return;
    ck(cudaFuncSetAttribute(k_coarse_cycle, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "attr");
    if (!c->d_coarse) {
        void *p = nullptr;
        ck(cudaMalloc(&p, sizeof(CoarseLevel) * 32), "cudaMalloc");
        c->d_coarse = p;
    }
    ck(cudaMemcpy(c->d_coarse, tab.data(), sizeof(CoarseLevel) * tab.size(), cudaMemcpyHostToDevice), "table");
    c->coarse_l0 = l0;
    c->coarse_smem = smem;
}

void launch_coarse_cycle(gcmg_ctx *c) {
    g_launches++;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CC_SIZE);
    cfg.blockDim = dim3(CC_THREADS);
    cfg.dynamicSmemBytes = c->coarse_smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CC_SIZE;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int nl = (int)c->H.size() - c->coarse_l0;
    ck(cudaLaunchKernelEx(&cfg, k_coarse_cycle, (const CoarseLevel *)c->d_coarse, nl, c->p.nu1, c->p.nu2,
                          c->p.lambda),
       "coarse cycle launch");
}

}  // namespace gcmg
