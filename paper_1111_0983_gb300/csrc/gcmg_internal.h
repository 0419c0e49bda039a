// Internal declarations of libgcmg: host-side geometry of every level, the
// device copies the kernels read, and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gcmg.h"

namespace gcmg {

constexpr int KMAX = 27;   // ghost stencil slots (3^3)
constexpr int STRIP_W = 60; // 2D sweep strips: owned columns (a warp holds 64)
constexpr int TILE_R = 16; // 2D interior tiles: rows (axis 0)
constexpr int TILE_C = 64; //                    columns (axis 1, contiguous)
constexpr int EMAX = 6;    // extension sources (2 d)
constexpr int CHUNK = 32;  // 3D active chunks: nodes along the contiguous axis (a warp)
// 3D fused sweep (k_rb_zmarch): a CTA owns ZM_TY rows (axis 1) x ZM_TX columns
// (axis 2, contiguous) and marches along axis 0 over at most ZM_SEG planes
constexpr int ZM_TY = 16, ZM_TX = 64, ZM_SEG = 32;
// 3D register-streaming sweep (k_rb_stream3d): a CTA owns SR_TY rows x SR_W
// columns, one warp per row (2 halo rows each side), one lane per column (2
// halo lanes each side), and marches along axis 0 over at most SR_SEG planes
constexpr int SR_TY = 12, SR_W = 28, SR_SEG = 64;
// 3D row-span sweep (k_rb_span3d): a CTA of SP_NW warps owns SP_NW - 4 rows
// (axis 1), one warp a row with 2 halo rows each side; lane l holds the nodes
// k0 + l + 32 c (c < C) of its row, a window of 32 C nodes along axis 2 of
// which the inner 32 C - 2 are owned; it marches along axis 0 over at most
// SP_SEG planes.  Per (plane, row) the level keeps the span of its unknowns
// and of its inside nodes, so that nothing outside them is read or written.
constexpr int SP_NW = 16, SP_J = SP_NW - 4, SP_SEG = 32, SP_CMIN = 2, SP_CMAX = 5;
// its inside-node masks: per plane (ZM_TY + 2) rows of ZM_TX + 2 bits (the
// tile and a 1-node halo), ZM_MROW words a row, planes padded to 16 bytes
constexpr int ZM_MROW = (ZM_TX + 2 + 31) / 32;
constexpr int ZM_MPLANE = ((ZM_TY + 2) * ZM_MROW + 3) / 4 * 4;

// NODE_WB marks, in the device copy of the type grid only, the nodes that the
// 2D boundary blocks write back through the write-back grid
enum : uint8_t { NODE_OUT = 0, NODE_IN = 1, NODE_GHOST = 2, NODE_KIND = 3, NODE_BAND = 4, NODE_WB = 8 };
enum : uint8_t { STENCIL_QUAD = 0, STENCIL_LIN = 1, STENCIL_CORNER = 2, STENCIL_AXIS = 3 };

struct GeomError {
    std::string msg;
};

// A set of independent components relaxed in shared memory by one CTA each.
// Component c stages the nodes lnode[node_off[c] .. node_off[c+1]) -- first
// the wb_cnt[c] nodes it writes back, then the other nodes it updates, then
// read-only nodes -- and runs: an optional ghost sweep, then reps x (red
// inside nodes, black inside nodes, Jacobi ghosts) on its updated nodes.
struct LocalProgram {
    std::vector<int32_t> node_off{0}, wb_cnt, lnode;
    std::vector<int32_t> node_base;   // per component: staged nodes without the pre-sweep's (they come last)
    std::vector<int32_t> int_off{0}, red_cnt, int_glob, int_me, int_nb;   // nb: 2 dim per entry
    std::vector<int32_t> gh_off{0}, gh_me, gh_q, gh_stn;                  // stn: 3^dim per entry
    // optional pre-sweep (2D boundary blocks): the interior red then black
    // update over every inside node the component reads, from the grid
    // before the relaxation's interior sweep (entries: slot, 2 dim neighbour
    // slots, global node for f)
    std::vector<int32_t> pre_off{0}, pre_red_cnt, pre_me, pre_nb, pre_glob;
    std::vector<int32_t> zred, zblack, zghost;   // union over components (global fallback)
    std::vector<int32_t> zred_src;   // 3D: red_sources of zred
    // components are overlapping blocks (3D junction zone): each writes back
    // through a separate grid, copied into u after the launch
    bool blocked = false;
    int max_nodes = 0, max_int = 0, max_gh = 0, max_pre = 0;
    int ncomp() const { return (int)wb_cnt.size(); }
};

// Geometry of one level, built on the host from phi (Sec. 2.2 - 2.6, 3.2).
struct HostLevel {
    int dim = 2, n = 0;
    double h = 0;
    double origin[3] = {-1.0, -1.0, -1.0};   // coordinates of node 0
    int64_t nn = 0;
    int64_t stride[3] = {0, 0, 0};
    std::vector<double> phi;
    std::vector<uint8_t> type;          // NODE_* (+ NODE_BAND)
    int64_t n_in = 0;
    // ghosts, increasing node index
    std::vector<int32_t> ghost_node;
    std::vector<double> B, nu;          // ng * dim
    std::vector<uint8_t> scase;         // STENCIL_*
    std::vector<int32_t> stn;           // ng * KMAX, per ghost
    std::vector<double> wD, wN;         // ng * KMAX
    std::vector<uint8_t> bc;            // 0 Dirichlet, 1 Neumann
    // 3D: the stencil of ghost q as a box when it is one (tensor-product
    // stencils): code m | 4 (axis 0 descending) | 8 (axis 1) | 16 (axis 2), m
    // = 3 (27 slots) or 2 (8 slots, the other 19 are the ghost itself), and
    // the node of slot 0; code 0: use the 27 stored nodes
    std::vector<uint8_t> gcode;
    std::vector<int32_t> gbase;
    // inside nodes of the extra-sweep band, split by colour
    std::vector<int32_t> band_red, band_black;
    std::vector<int32_t> band_red_src;   // 3D: red_sources of band_red
    // 2D tiles (TILE_R x TILE_C) holding inside nodes, packed (tile row << 16 | tile column)
    std::vector<int32_t> tiles;
    // 3D active chunks: runs of CHUNK nodes along the contiguous axis (start
    // at a multiple of CHUNK) holding an inside node or a ghost; first node
    // and length (the last run of a row is shorter)
    std::vector<int32_t> chunk;
    std::vector<uint8_t> chunk_len;
    // 3D fused-sweep work: pairs (tile row << 16 | tile column, first plane
    // << 16 | end plane), the planes of a tile that hold inside nodes or ghosts
    std::vector<int32_t> zm;
    // per item: offset (in ZM_MPLANE-word planes) of its inside-node masks
    // for planes first - 1 .. end, in zm_mask
    std::vector<int32_t> zm_moff;
    std::vector<uint32_t> zm_mask;
    // the same pairs for the SR_TY x SR_W tiles of the register-streaming sweep
    std::vector<int32_t> sr;
    // row-span sweep: per (plane i, row j), i * n + j, two words: the span of
    // the row's unknowns (lo | hi << 16) and of its inside nodes (the same
    // form); an empty span is lo = 0xffff, hi = 0.  Items: quadruples (row
    // block, window origin k0, first plane, end plane); sp_cols = C, the
    // columns a lane holds.  Empty when some row's inside nodes are not one
    // interval (the sweep then falls back to the tiles).
    std::vector<int32_t> sp_rows, sp;
    int sp_cols = 0;
    // segments of up to 64 consecutive inside nodes of a row, as pairs
    // (i * n + j, first | last << 16), in increasing node order: the work of
    // the one-colour row sweep (any domain)
    std::vector<int32_t> sp_list;
    // defect extension of this level (before restricting to the next coarser one)
    std::vector<int32_t> ext_node;      // ordered by upwind wavefront
    std::vector<uint8_t> ext_cnt;
    std::vector<int32_t> ext_src;       // ne * EMAX
    std::vector<double> ext_w;          // ne * EMAX
    std::vector<int> ext_wave;          // wavefront offsets into ext_node (size nwave + 1)
    // extension followed by the partial transfer at the coarse ghosts, as one
    // sparse map from this level's ghost defects to the next level's ghost
    // data (CSR over coarse ghosts; columns are this level's ghost numbers)
    std::vector<int32_t> gt_ptr, gt_col;
    std::vector<double> gt_val;
    // 3D: the inside nodes of the next coarser level whose fine image's 3^3
    // neighbourhood on this level is not all inside (the restriction's
    // partial transfer there searches its boxes; the others take full
    // weighting), in increasing order
    std::vector<int32_t> partial_coarse;
    // their 27 partial-transfer weights over this level's inside set, slot
    // major (27 x list size), computed in FP32 and in FP64 with the
    // operations of the device's partial transfer in the same order
    std::vector<float> partial_wf;
    std::vector<double> partial_wd;
    // shared-memory relaxation programs: the junction zone (depends on bc)
    // and, in 2D, the boundary blocks of the lambda extra sweeps
    LocalProgram junction, boundary;
    // exact junction solve (2D): the solved set split into independent
    // components; per component its nodes (increasing), their ghost numbers
    // (-1: inside node) and the dense inverse of their equations
    std::vector<int32_t> js_off;        // ncomp + 1 offsets into js_node
    std::vector<int32_t> js_node, js_ghost;
    std::vector<int64_t> js_aoff;       // ncomp + 1 offsets into js_inv
    std::vector<double> js_inv;         // per component m x m, row major
    bool js_dirty = true;               // out of date with bc
    // coarsest level: unknowns (node, ghost number or -1) and dense inverse
    std::vector<int32_t> unk_node, unk_ghost;
    std::vector<double> Ainv;           // nunk * nunk, row major
    bool ainv_dirty = true;             // Ainv out of date with bc

    int64_t ng() const { return (int64_t)ghost_node.size(); }
};

// The sources of the six axis neighbours of each 3D inside node of `list`,
// in the order of neighbour_sum (axis 2 -, +; axis 0 -, +; axis 1 -, +),
// slot major (6 x list size): the node, or -1 - q where the neighbour is
// ghost q, so that a red sweep can read the ghosts' new values from the
// Jacobi buffer while the same launch stores them.
std::vector<int32_t> red_sources(const HostLevel &L, const std::vector<int32_t> &list);

// Rebuilds a 3D level's row-span sweep items for C columns a lane and items
// of at most seg planes (C = 0: the cheapest C by the work model; seg = 0:
// SP_SEG).  Returns false (and leaves the level without items) when a row's
// inside nodes are not one interval.
bool build_span_items(HostLevel &L, int C = 0, int seg = 0);

// Builds all levels (throws GeomError).  phi: fine grid, n^dim values; h0:
// fine spacing (0: 2 / (n - 1)); origin: coordinates of node 0 (null: -1 on
// every axis).
void build_hierarchy(int dim, int n, int n_coarse, const double *phi, double delta_over_h,
                     std::vector<HostLevel> &levels, double h0 = 0.0, const double *origin = nullptr);
// Partial-transfer weights (Sec. 2.5) at the fine image p of a coarse node over
// the inside set (interior) or its complement; wt[3^dim], axis 0 slowest.
bool partial_transfer_weights(const HostLevel &F, int64_t p, bool interior, double *wt);
// Unknown numbering of the coarsest level (independent of bc).
void number_coarse_unknowns(HostLevel &L);
// Dense inverse of the coarsest system with the level's current bc (throws GeomError).
void build_coarse_inverse(HostLevel &L);
// Junction zone of the level's current bc (radius in h).
void build_junction(HostLevel &L, double radius, int mu = 0);
// The zone's unknowns as a mask (1 / 0, nn bytes).
std::vector<uint8_t> junction_zone_mask(const HostLevel &L, double radius);
// 2D sweep strips of `rows` x STRIP_W owned nodes holding inside nodes or
// ghosts, packed (row block << 16 | column block).
std::vector<int32_t> strips_for(const HostLevel &L, int rows);
// Exact junction solve of the level's current bc: the zone within radius h,
// grown by its ghosts' stencils and stripped of ghosts whose stencil leaves
// it, in components with the inverses of their equations (throws GeomError).
void build_junction_solve(HostLevel &L, double radius);
// Largest component of an exact junction solve.
constexpr int JS_MAX = 4096;
// 2D boundary blocks of the extra sweeps: block x block tiles with a halo
// covering the dependency cone of one ghost sweep + lambda (R, B, G) sweeps.
void build_boundary_blocks(HostLevel &L, int lambda, int block);

// --------------------------------------------------------------- device side
// A LocalProgram on the device.
struct LocalDev {
    int ncomp = 0, max_nodes = 0, max_int = 0, max_gh = 0, max_pre = 0;
    int max_colour = 0;   // most inside entries of one colour in a component
    int32_t *node_off = nullptr, *wb_cnt = nullptr, *lnode = nullptr, *node_base = nullptr;
    int32_t *pre_off = nullptr, *pre_red_cnt = nullptr, *pre_me = nullptr, *pre_nb = nullptr, *pre_glob = nullptr;
    bool has_pre = false;
    bool pre_in_smem = false;  // the FP32 program with its pre-sweep lists fits in shared memory
    int32_t *int_off = nullptr, *red_cnt = nullptr, *int_glob = nullptr, *int_me = nullptr, *int_nb = nullptr;
    int32_t *gh_off = nullptr, *gh_me = nullptr, *gh_q = nullptr, *gh_stn = nullptr;
    int nzred = 0, nzblack = 0, nzghost = 0;
    int32_t *zred = nullptr, *zblack = nullptr, *zghost = nullptr;
    int32_t *zred_src = nullptr;   // 3D: LocalProgram::zred_src
    bool blocked = false;          // LocalProgram::blocked
    int nwb = 0;
    int32_t *wb_list = nullptr;   // every component's write-back nodes, one flat list
    bool in_smem = true;       // false: relaxed by per-sweep launches over the union lists
    bool in_smem32 = true;     // the same for the FP32 program (smaller: 3D FP32 cycles use it)
};

// Integer geometry of a level on the device (shared by both precisions).
struct DevGeom {
    int dim = 2, n = 0;
    int64_t nn = 0;
    int ng = 0, nred = 0, nblack = 0, ne = 0, nunk = 0;
    uint8_t *type = nullptr;
    int32_t *gnode = nullptr;    // ng
    int32_t *gstn = nullptr;     // KMAX * ng, slot major
    uint8_t *gcode = nullptr;    // HostLevel::gcode, gbase (3D)
    int32_t *gbase = nullptr;
    int32_t *red = nullptr, *black = nullptr;
    int32_t *red_src = nullptr;  // 3D: HostLevel::band_red_src
    int ntiles = 0;
    int32_t *tiles = nullptr;    // active 2D interior tiles
    int nstrips = 0, strip_rows = 0;
    int32_t *strips = nullptr;   // active 2D sweep strips (strip_rows x STRIP_W owned nodes)
    int nzm = 0;                 // 3D fused-sweep work items (HostLevel::zm pairs)
    int32_t *zm = nullptr;
    int32_t *zm_moff = nullptr;  // and their inside-node masks
    uint32_t *zm_mask = nullptr;
    int nsr = 0;                 // register-streaming sweep items (HostLevel::sr pairs)
    int32_t *sr = nullptr;
    int nsp = 0, sp_cols = 0;    // row-span sweep items (HostLevel::sp quadruples), columns a lane
    int32_t *sp = nullptr;
    int32_t *sp_rows = nullptr;  // HostLevel::sp_rows
    int nspl = 0;                // segments of the one-colour row sweep (HostLevel::sp_list pairs)
    int32_t *sp_list = nullptr;
    int64_t nchunks = 0;         // 3D active chunks (HostLevel::chunk)
    int32_t *chunks = nullptr;
    uint8_t *chunk_len = nullptr;
    int32_t *enode = nullptr;    // ne
    uint8_t *ecnt = nullptr;     // ne
    int32_t *esrc = nullptr;     // EMAX * ne, slot major
    int32_t *gt_ptr = nullptr, *gt_col = nullptr;   // ghost transfer to the next level
    int npartial = 0;
    int32_t *partial_coarse = nullptr;                 // HostLevel::partial_coarse
    int32_t *unk_node = nullptr, *unk_ghost = nullptr;
    std::vector<int> wave;       // host copy of the wavefront offsets
    LocalDev jz, bz;             // junction zone / boundary blocks
    // exact junction solve: js_n rows in js_ncomp components.  On the device
    // each component's inverse has rows padded to a multiple of 4 entries
    // (zeros) and starts at js_aoff[c], a multiple of 4; its defects sit at
    // js_roff[c] (a multiple of 4) in the padded defect vector, row k's at
    // js_rpos[k], so that rows and defects are read as 16-byte vectors.
    int js_n = 0, js_ncomp = 0;
    int32_t *js_node = nullptr, *js_ghost = nullptr, *js_comp = nullptr, *js_off = nullptr;
    int32_t *js_roff = nullptr, *js_rpos = nullptr;
    int js_rlen = 0;                    // length of the padded defect vector
    std::vector<int64_t> js_aoff_h;     // host copies of the padded offsets (ncomp + 1)
    std::vector<int32_t> js_roff_h;
    int64_t *js_aoff = nullptr;
};

// Floating-point data of a level in precision T.
template <typename T>
struct DevData {
    T *u = nullptr, *f = nullptr, *r = nullptr;   // grids (may be null if unused)
    T *u2 = nullptr;     // second u grid: the 2D sweep reads one buffer and writes the other
    T *gw = nullptr;     // KMAX * ng ghost weights for the current bc, slot major
    T *gc = nullptr;     // ng relaxation coefficient mu dt
    T *gg = nullptr;     // ng boundary data (level 0) or restricted boundary defect
    T *gtmp = nullptr;   // ng new ghost values of a Jacobi sweep
    T *ew = nullptr;     // EMAX * ne extension weights, slot major
    T *gt_val = nullptr; // ghost transfer weights to the next level
    T *pt_w = nullptr;   // HostLevel::partial_wf / partial_wd
    T *Ainv = nullptr;   // nunk * nunk (coarsest level)
    T *js_inv = nullptr; // inverses of the junction-solve components
    T *js_r = nullptr;   // defects of the junction-solve equations (padded layout, zero pads)
};

// Kernel view of one level in precision T (passed by value).
template <typename T>
struct LevelView {
    int n;
    int64_t nn;
    int64_t s0, s1, s2;          // strides of axes 0, 1, 2 (s2 = 1 in 3D; 2D uses s0, s1)
    T h2;                        // h^2
    T inv_h2;
    const uint8_t *type;
    T *u;
    const T *f;
    T *r;
    int ng;
    const int32_t *gnode;
    const int32_t *gstn;
    const T *gw;
    const T *gc;
    const T *gg;
    T *gtmp;
    // 3D: the active chunks (null in 2D: kernels over nodes then cover the box)
    const int32_t *chunks = nullptr;
    const uint8_t *clen = nullptr;
    int64_t nchunks = 0;
    // 3D: segments of up to 64 consecutive inside nodes of a row (DevGeom::sp_list)
    const int2 *segs = nullptr;
    int nsegs = 0;
    // 3D: ghost stencils as boxes (DevGeom::gcode, gbase; null: gstn only)
    const uint8_t *gcode = nullptr;
    const int32_t *gbase = nullptr;
};

// One 3D boundary relaxation as a single launch (k_boundary3d): the Jacobi
// ghost sweep, lambda x (band red, band black, ghost sweep) and mu x the same
// over the junction-zone lists, with grid-wide barriers between the phases.
struct BoundaryProgram3 {
    const int32_t *red = nullptr, *black = nullptr;
    int nred = 0, nblack = 0;
    const int32_t *zred = nullptr, *zblack = nullptr, *zghost = nullptr;
    int nzred = 0, nzblack = 0, nzghost = 0;
    int lead = 1;       // start with the ghost sweep of the relaxation itself
    int lambda = 0;     // band sweeps
    int mu = 0;         // junction-zone sweeps over the global lists (0: none or done elsewhere)
    unsigned *bar = nullptr;   // barrier words: arrivals, generation (zero when idle)
    int *err = nullptr;        // set to 1 when a barrier wait ran out (GCMG_E_TIMEOUT)
    unsigned nbar = 0;         // CTAs the barrier waits for (the grid; more only in the timeout test)
    unsigned spin = 0;         // polls before a wait gives up
};

// Kernel view of a LocalDev program in precision T.
template <typename T>
struct LocalView {
    int ncomp, max_nodes, max_int, max_gh, max_pre, max_colour, ng;
    const int32_t *node_off, *wb_cnt, *lnode, *node_base;
    const int32_t *pre_off, *pre_red_cnt, *pre_me, *pre_nb, *pre_glob;
    const int32_t *int_off, *red_cnt, *int_glob, *int_me, *int_nb;
    const int32_t *gh_off, *gh_me, *gh_q, *gh_stn;
    T *u;
    T *wb;    // non-null: write-back target (boundary blocks, whose halos overlap); copied into u afterwards
    const int32_t *wb_list;   // the write-back nodes of all components (nwb)
    int nwb;
    const T *f, *gg, *gc, *gw;
    T h2;
};

}  // namespace gcmg
