// Internal: the context behind the C ABI (shared by api.cu and batch.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "gcmg_internal.h"

using gcmg::DevData;
using gcmg::DevGeom;
using gcmg::HostLevel;
using gcmg::LevelView;
using gcmg::LocalDev;
using gcmg::LocalView;

struct gcmg_ctx {
    gcmg_params p{};
    cudaStream_t stream = nullptr;
    int device = 0;
    std::vector<HostLevel> H;
    std::vector<DevGeom> G;
    std::vector<DevData<double>> D64;
    std::vector<DevData<float>> D32;
    bool rhs_set = false;
    bool js64 = false;                      // FP64 junction-solve inverses kept (single relaxations)
    // the fused coarse cycle (coarse.cu): its first level (-1: per-level
    // launches), level table on the device, dynamic shared memory
    int coarse_l0 = -1;
    double *relax_a = nullptr, *relax_b = nullptr;   // scratch grids of the single-step relaxation
    void *d_coarse = nullptr;
    size_t coarse_smem = 0;
    // Kaczmarz comparison smoother (smoother = 1): per level, the rows (an
    // inside band node p as p, ghost q as -(q + 1)) grouped by colour, and
    // the 26 colour offsets
    std::vector<int32_t *> kz_rows;
    std::vector<std::vector<int32_t>> kz_off;
    unsigned long long *d_norm = nullptr;   // two slots: defect norm, rhs norm
    unsigned long long *h_norm = nullptr;   // pinned
    // the solve loop as one CUDA graph: a device-side while loop over cycles
    cudaStream_t gstream = nullptr;         // capture / launch stream (never the legacy one)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // large 2D levels: the merged FP32 relaxation as two launches side by
    // side (strips on the stream, boundary blocks on sstream)
    cudaStream_t sstream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int split2d_strips = 0;       // levels with at least this many strips split (0: never; measured no faster)
    double *d_rel = nullptr;                // rel[0..256]
    double *d_r0 = nullptr;
    int *d_m = nullptr;
    // the 3D boundary relaxation in one launch (k_boundary3d): barrier words,
    // timeout flag; coop3d = 0 (default: measured faster, about 5 us a
    // barrier against 2-3 us a launch) runs it as one launch per phase;
    // phantom > 0 and spin make its barriers wait for CTAs that never arrive
    // (the timeout test)
    unsigned *d_bar = nullptr;
    int *d_err = nullptr;
    int coop3d = 0, bar_phantom = 0;
    int junction_blocks = 0;   // 3D junction zone in overlapping shared-memory blocks (gcmg_set_junction_blocks;
                               // measured slower at 513^3: 3.28 against 3.11 ms a cycle)
    int sweep3d = 3;   // 3D interior sweep: 0 k_rb_zmarch (shared-memory planes), 1 k_rb_stream3d (registers),
                       // 2 k_rb_span3d (row spans; FP32, else 1), 3 k_rb_rows (two in-place colour launches)
    int cluster3d = 0; // 1: 3D boundary phases of small levels (and junction sweeps) as one thread-block
                       // cluster (measured slower than one launch a phase inside the graph)
    unsigned bar_spin = 1u << 22;
    bool use_graph = true;
    long long graph_kernels = 0;            // kernels in one loop iteration
    long long graph_pro_kernels = 0;        // kernels before the loop
    struct SolveResult {                    // what a graph solve reports back (pinned)
        double r0;
        double rel[257];
        int m[2];                           // cycles done, consecutive cycles whose defect grew
    } *h_res = nullptr;
    // event timing of one fine-level kernel class during solves
    int timing_kind = -1;
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    double timed_bytes = 0.0;              // algorithmic bytes of the timed launches
    std::vector<int64_t> bz_units;         // per level: distinct values a boundary-block launch moves
    std::vector<void *> allocs;
    std::string err;
    int version = 0;                        // bumped when the boundary types change
};


namespace gcmg {

// a failed CUDA call, thrown by ck() and turned into GCMG_E_CUDA by the
// entry points (one type for every translation unit of the library)
struct CudaFail {
    cudaError_t e;
    const char *what;
};

inline void ck(cudaError_t e, const char *what) {
    if (e != cudaSuccess) throw CudaFail{e, what};
}

template <typename T>
LevelView<T> view(const gcmg_ctx *c, int l, const DevData<T> &D) {
    const HostLevel &L = c->H[l];
    const DevGeom &g = c->G[l];
    LevelView<T> v;
    v.n = L.n;
    v.nn = L.nn;
    v.s0 = L.stride[0];
    v.s1 = L.stride[1];
    v.s2 = L.dim == 3 ? L.stride[2] : 0;
    v.h2 = (T)(L.h * L.h);
    v.inv_h2 = (T)(1.0 / (L.h * L.h));
    v.type = g.type;
    v.u = D.u;
    v.f = D.f;
    v.r = D.r;
    v.ng = g.ng;
    v.gnode = g.gnode;
    v.gstn = g.gstn;
    v.gw = D.gw;
    v.gc = D.gc;
    v.gg = D.gg;
    v.gtmp = D.gtmp;
    v.chunks = g.chunks;
    v.clen = g.chunk_len;
    v.nchunks = g.nchunks;
    v.segs = reinterpret_cast<const int2 *>(g.sp_list);
    v.nsegs = g.nspl;
    v.gcode = g.gcode;
    v.gbase = g.gbase;
    return v;
}

template <typename T>
LocalView<T> lview(const LocalDev &z, const LevelView<T> &v, T *wb = nullptr) {
    LocalView<T> J;
    J.wb = wb;
    J.ncomp = z.ncomp;
    J.max_nodes = z.max_nodes;
    J.max_int = z.max_int;
    J.max_gh = z.max_gh;
    J.max_pre = z.max_pre;
    J.max_colour = z.max_colour;
    J.ng = v.ng;
    J.node_off = z.node_off; J.wb_cnt = z.wb_cnt; J.lnode = z.lnode; J.node_base = z.node_base;
    J.pre_off = z.pre_off; J.pre_red_cnt = z.pre_red_cnt; J.pre_me = z.pre_me; J.pre_nb = z.pre_nb;
    J.pre_glob = z.pre_glob;
    J.int_off = z.int_off; J.red_cnt = z.red_cnt; J.int_glob = z.int_glob; J.int_me = z.int_me; J.int_nb = z.int_nb;
    J.gh_off = z.gh_off; J.gh_me = z.gh_me; J.gh_q = z.gh_q; J.gh_stn = z.gh_stn;
    J.wb_list = z.wb_list;
    J.nwb = z.nwb;
    J.u = v.u; J.f = v.f; J.gg = v.gg; J.gc = v.gc; J.gw = v.gw;
    J.h2 = v.h2;
    return J;
}

// Host geometry of a context's levels (no CUDA calls; thread safe): the
// hierarchy of build_hierarchy plus the 2D boundary-block programs.
void prepare_levels(const gcmg_params &p, const double *phi_host, std::vector<HostLevel> &H);
// Validates p; GCMG_OK if usable.
gcmg_status check_params(const gcmg_params &p);
// Rebuilds (if out of date) and uploads the coarsest inverse; upload only.
void ensure_inverse(gcmg_ctx *c);
// builds and uploads the exact junction solves that are out of date with bc
void ensure_junction_solve(gcmg_ctx *c);
void upload_js(gcmg_ctx *c, int l);
void upload_inverse(gcmg_ctx *c);
// the fused coarse end of the V-cycle (coarse.cu)
void coarse_prepare(gcmg_ctx *c);
void launch_coarse_cycle(gcmg_ctx *c);
// Creates a context from prepared levels (uploads everything to the current device).
gcmg_status create_from_levels(const gcmg_params &p, std::vector<HostLevel> &&H, cudaStream_t stream, gcmg_ctx **out);

}  // namespace gcmg
