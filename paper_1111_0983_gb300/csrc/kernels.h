// Launchers of the per-level kernels (kernels.cu).
#pragma once

#include <algorithm>
#include <atomic>

#include "gcmg_internal.h"

namespace gcmg {

extern std::atomic<long long> g_launches;   // kernels launched by this library

// Kaczmarz comparison smoother (kaczmarz.cu): `sweeps` sweeps, each over the
// colours c = 0..24 in order, a launch each, of the rows rows[off[c] ..
// off[c + 1]) (inside band node p as p, ghost q as -(q + 1)); in place on v.u
void launch_kaczmarz(const LevelView<double> &v, const int32_t *rows, const std::vector<int32_t> &off, int sweeps,
                     cudaStream_t s);

template <typename T>
void launch_rb(const LevelView<T> &v, int dim, int color, cudaStream_t s);
// one FP32 2D relaxation (interior sweep, ghost sweep, band sweeps) in one
// launch: strips and boundary blocks both read v.u and write out
// the same as two launches side by side: the boundary blocks on `side`, the
// strips' interior nodes on `s` (fork and join through the two events)
void launch_relax2d_split(const LevelView<float> &v, float *out, const DevGeom &g, const LocalView<float> &J,
                          int lambda, cudaStream_t s, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join);
void launch_relax2d(const LevelView<float> &v, float *out, const DevGeom &g, const LocalView<float> &J, int lambda,
                    cudaStream_t s);
// both colours of a 2D sweep over the active strips (one warp a strip, rows
// in registers): reads v.u, writes out
template <typename T>
void launch_rb_strip(const LevelView<T> &v, T *out, const DevGeom &g, cudaStream_t s);
// both colours of a 2D sweep over the active tiles: reads v.u, writes out
template <typename T>
void launch_rb_fused2d(const LevelView<T> &v, T *out, const int32_t *tiles, int ntiles, cudaStream_t s);
template <typename T>
void launch_rb_list(const LevelView<T> &v, int dim, const int32_t *list, int cnt, cudaStream_t s);
template <typename T>
void launch_ghost_relax(const LevelView<T> &v, int dim, cudaStream_t s);
// 3D: the red half of a band / junction-zone sweep (sources: red_sources)
// merged with the store of the ghosts' new values (glist null: all ghosts)
template <typename T>
void launch_rb_list_store(const LevelView<T> &v, const int32_t *list, const int32_t *src, int cnt,
                          const int32_t *glist, int gcnt, cudaStream_t s);
// the halves of a 3D Jacobi ghost sweep (list null: all ghosts)
template <typename T>
void launch_ghost_new(const LevelView<T> &v, const int32_t *list, int cnt, cudaStream_t s);
template <typename T>
void launch_ghost_store(const LevelView<T> &v, const int32_t *list, int cnt, cudaStream_t s);
template <typename T>
void launch_ghost_relax_list(const LevelView<T> &v, int dim, const int32_t *list, int cnt, cudaStream_t s);
template <typename T>
void launch_defect(const LevelView<T> &v, int dim, bool zero_rest, unsigned long long *norm, cudaStream_t s);
template <typename T>
void launch_extend(T *r, const DevGeom &g, const T *ew, cudaStream_t s);
template <typename T>
void launch_restrict(const LevelView<T> &F, const LevelView<T> &C, int dim, T *fc, T *gc, cudaStream_t s);
template <typename T>
void launch_restrict_interior(const LevelView<T> &F, const LevelView<T> &C, int dim, T *fc, cudaStream_t s);
// one descent of the cycle: coarse f = restricted fine defect (computed on the
// spot), coarse ghost data = transferred fine ghost defects, coarse u = 0
template <typename T>
void launch_descend(const LevelView<T> &F, const LevelView<T> &C, const DevGeom &gf, const T *gt_val, T *fc, T *gc,
                    T *uc, cudaStream_t s, const T *pt_w = nullptr);
template <typename T>
void launch_ghost_transfer(const T *rf, const int32_t *fgnode, const int32_t *ptr, const int32_t *col, const T *val,
                           T *gc, int ngc, cudaStream_t s);
template <typename T>
void launch_prolong(const LevelView<T> &F, const LevelView<T> &C, int dim, const T *e, T *out, bool add,
                    cudaStream_t s);
template <typename T>
void launch_coarse_solve(const LevelView<T> &v, const DevGeom &g, const T *Ainv, cudaStream_t s);
// exact junction solve: defects of the solved equations into r, then
// u += A_ZZ^-1 r per component.  pending: a 2D boundary-block program whose
// write-back into v.u is still to be done; the defect launch performs it.
template <typename T>
void launch_junction_solve(const LevelView<T> &v, const DevGeom &g, const T *inv, T *r, cudaStream_t s,
                           const LocalView<T> *pending = nullptr);
template <typename T>
void launch_mask_unknowns(const uint8_t *type, T *u, int64_t nn, cudaStream_t s);
// Boundary types of the ng ghosts of a level (step `step` = 2^l of the fine
// grid, n_l nodes a side): the fine mask (n^dim bytes) at the fine node
// nearest each ghost's B (B: ng * dim doubles), ties to the ghost's side
void launch_mask_types(int dim, int n, double h, const double *origin, int step, int n_l, const double *B,
                       const int32_t *gnode, int ng, const uint8_t *mask, uint8_t *types, cudaStream_t s);
// 3D: the boundary phase of one relaxation (ghost sweep, band sweeps,
// junction sweeps on global lists) as one launch with grid-wide barriers;
// phantom > 0 makes every barrier wait for CTAs that do not exist (the
// timeout test).  Returns false if the kernel cannot run here (then nothing
// was launched).
template <typename T>
bool launch_boundary3d(const LevelView<T> &v, BoundaryProgram3 P, int phantom, cudaStream_t s);
// the same phases as one thread-block cluster (hardware barriers); false if
// the launch failed (nothing was launched)
template <typename T>
bool launch_boundary3d_cluster(const LevelView<T> &v, const BoundaryProgram3 &P, cudaStream_t s);
// 3D: one red-black sweep (both colours) over the level's fused-sweep items,
// reading v.u and writing every node of the items into out
template <typename T>
void launch_rb_zmarch(const LevelView<T> &v, T *out, const DevGeom &g, cudaStream_t s);
// the same sweep with the planes in registers (a warp a row, a lane a column)
template <typename T>
void launch_rb_stream3d(const LevelView<T> &v, T *out, const DevGeom &g, cudaStream_t s);
// both colours of the interior sweep as two in-place launches over segments
// of the rows holding inside nodes; false when the level has no segment list
template <typename T>
bool launch_rb_rows(const LevelView<T> &v, const DevGeom &g, cudaStream_t s);
// the row-span sweep (FP32); false when the level has no items for it
bool launch_rb_span3d(const LevelView<float> &v, float *out, const DevGeom &g, cudaStream_t s);

template <typename T>
size_t local_smem_bytes(const LocalView<T> &J, int dim, bool pre = false);
// shared-memory programs; a program with a write-back grid (J.wb) leaves its
// write-back to launch_local_copyback or to launch_junction_solve
template <typename T>
void launch_local(const LocalView<T> &J, int dim, int lead_ghost, int reps, cudaStream_t s);
template <typename T>
void launch_local_copyback(const LocalView<T> &J, cudaStream_t s);
template <typename T>
void local_prepare(int dim, size_t smem);
// whether a program's largest component keeps its inside entries in registers
bool local_fits_registers(int max_int_per_colour);

// FP64 defect of level 0 and its norm (as launch_defect), also writing the
// next FP32 correction problem: f32 = defect at inside nodes (0 elsewhere),
// g32 = ghost defects, e32 = 0
void launch_defect_mixed(const LevelView<double> &v, int dim, unsigned long long *norm, float *f32, float *g32,
                         float *e32, cudaStream_t s);
void launch_add_correction(const DevGeom &g, double *u64, const float *e32, cudaStream_t s);

}  // namespace gcmg
