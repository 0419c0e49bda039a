// C ABI of libgcmg (include/gcmg.h): context lifetime, hierarchy upload,
// cycle schedule and the solve loops.  The per-level arithmetic lives in
// kernels.cu; geometry construction in setup.cpp.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "ctx.h"
#include "gcmg_internal.h"
#include "kernels.h"

using namespace gcmg;

namespace {


template <typename T>
T *dalloc(gcmg_ctx *c, size_t count) {
    if (count == 0) count = 1;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw std::bad_alloc();
    }
    c->allocs.push_back(p);
    return static_cast<T *>(p);
}

template <typename T>
T *upload(gcmg_ctx *c, const T *host, size_t count) {
    T *d = dalloc<T>(c, count);
    if (count) ck(cudaMemcpyAsync(d, host, count * sizeof(T), cudaMemcpyHostToDevice, c->stream), "upload");
    return d;
}

int kslots(int dim) { return dim == 2 ? 9 : 27; }

// 3D levels whose ghost and band lists hold at most this many entries run a
// relaxation's boundary phases as one thread-block cluster (16 CTAs of 1024
// threads: four entries a thread a phase)
constexpr int64_t kClusterWork = 65536;

// Rows of the Kaczmarz comparison smoother on level l (2D): the ghosts and the
// inside nodes of the band, grouped by the colour (i mod 5) + 5 (j mod 5) of
// their node, increasing node index within a colour
void build_kaczmarz_rows(gcmg_ctx *c, int l) {
    const HostLevel &L = c->H[l];
    std::vector<int32_t> gid(L.nn, -1);
    for (int64_t q = 0; q < L.ng(); q++) gid[L.ghost_node[q]] = (int32_t)q;
    std::vector<std::vector<int32_t>> by(25);
    for (int64_t p = 0; p < L.nn; p++) {
        const int kind = L.type[p] & NODE_KIND;
        const bool in = kind == NODE_IN && (L.type[p] & NODE_BAND);
        if (!in && kind != NODE_GHOST) continue;
        const int64_t i = p / L.n, j = p % L.n;
        by[(int)(i % 5) + 5 * (int)(j % 5)].push_back(in ? (int32_t)p : -(gid[p] + 1));
    }
    std::vector<int32_t> rows, off{0};
    for (const auto &b : by) {
        rows.insert(rows.end(), b.begin(), b.end());
        off.push_back((int32_t)rows.size());
    }
    if ((int)c->kz_rows.size() <= l) {
        c->kz_rows.resize(l + 1, nullptr);
        c->kz_off.resize(l + 1);
    }
    c->kz_rows[l] = upload<int32_t>(c, rows.data(), rows.size());
    c->kz_off[l] = off;
}

// slot-major copies of per-ghost / per-extension-node arrays
template <typename S, typename T>
std::vector<T> slot_major(const std::vector<S> &src, int64_t count, int width, int used) {
    std::vector<T> out((size_t)count * used);
    for (int64_t i = 0; i < count; i++)
        for (int k = 0; k < used; k++) out[(size_t)k * count + i] = (T)src[(size_t)i * width + k];
    return out;
}

template <typename T>
void upload_ghost_data(gcmg_ctx *c, int l, DevData<T> &D, bool alloc) {
    const HostLevel &L = c->H[l];
    const int64_t ng = L.ng();
    const int K = kslots(L.dim);
    std::vector<double> w((size_t)ng * KMAX);
    std::vector<T> coef(ng);
    const double cN = c->p.c_neumann_factor * 2.0 * L.h / (3.0 * std::sqrt((double)L.dim));
    for (int64_t q = 0; q < ng; q++) {
        const double *src = (L.bc[q] ? L.wN.data() : L.wD.data()) + q * KMAX;
        std::memcpy(&w[q * KMAX], src, sizeof(double) * KMAX);
        coef[q] = (T)(L.bc[q] ? cN : c->p.c_dirichlet);
    }
    std::vector<T> ws = slot_major<double, T>(w, ng, KMAX, K);
    if (alloc) {
        D.gw = dalloc<T>(c, ws.size());
        D.gc = dalloc<T>(c, ng);
    }
    ck(cudaMemcpyAsync(D.gw, ws.data(), ws.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream), "gw");
    ck(cudaMemcpyAsync(D.gc, coef.data(), coef.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream), "gc");
    if (l + 1 == (int)c->H.size() && alloc) D.Ainv = dalloc<T>(c, L.unk_node.size() * L.unk_node.size());
    // synchronous: the staging vectors die at return
    ck(cudaStreamSynchronize(c->stream), "sync");
}

template <typename T>
void alloc_data(gcmg_ctx *c, int l, DevData<T> &D, bool grids) {
    const HostLevel &L = c->H[l];
    upload_ghost_data<T>(c, l, D, true);
    D.gg = dalloc<T>(c, L.ng());
    D.gtmp = dalloc<T>(c, L.ng());
    const int64_t ne = (int64_t)L.ext_node.size();
    std::vector<T> ew = slot_major<double, T>(L.ext_w, ne, EMAX, EMAX);
    D.ew = upload<T>(c, ew.data(), ew.size());
    std::vector<T> gtv(L.gt_val.begin(), L.gt_val.end());
    D.gt_val = upload<T>(c, gtv.data(), gtv.size());
    if (!L.partial_coarse.empty()) {
        if constexpr (std::is_same<T, float>::value) D.pt_w = upload<T>(c, L.partial_wf.data(), L.partial_wf.size());
        else D.pt_w = upload<T>(c, L.partial_wd.data(), L.partial_wd.size());
    }
    ck(cudaStreamSynchronize(c->stream), "sync");
    if (grids) {
        D.u = dalloc<T>(c, L.nn);
        D.u2 = dalloc<T>(c, L.nn);
        D.f = dalloc<T>(c, L.nn);
        D.r = dalloc<T>(c, L.nn);
        ck(cudaMemsetAsync(D.u, 0, L.nn * sizeof(T), c->stream), "memset");
        ck(cudaMemsetAsync(D.u2, 0, L.nn * sizeof(T), c->stream), "memset");
        ck(cudaMemsetAsync(D.f, 0, L.nn * sizeof(T), c->stream), "memset");
        ck(cudaMemsetAsync(D.r, 0, L.nn * sizeof(T), c->stream), "memset");
    }
}

void upload_geometry(gcmg_ctx *c, int l) {
    const HostLevel &L = c->H[l];
    DevGeom g;
    g.dim = L.dim;
    g.n = L.n;
    g.nn = L.nn;
    g.ng = (int)L.ng();
    g.nred = (int)L.band_red.size();
    g.nblack = (int)L.band_black.size();
    g.ne = (int)L.ext_node.size();
    g.type = upload<uint8_t>(c, L.type.data(), L.type.size());
    g.gnode = upload<int32_t>(c, L.ghost_node.data(), L.ghost_node.size());
    std::vector<int32_t> stn = slot_major<int32_t, int32_t>(L.stn, g.ng, KMAX, kslots(L.dim));
    g.gstn = upload<int32_t>(c, stn.data(), stn.size());
    g.red = upload<int32_t>(c, L.band_red.data(), L.band_red.size());
    if (!L.gcode.empty()) {
        g.gcode = upload<uint8_t>(c, L.gcode.data(), L.gcode.size());
        g.gbase = upload<int32_t>(c, L.gbase.data(), L.gbase.size());
    }
    if (!L.band_red_src.empty()) g.red_src = upload<int32_t>(c, L.band_red_src.data(), L.band_red_src.size());
    g.ntiles = (int)L.tiles.size();
    g.tiles = upload<int32_t>(c, L.tiles.data(), L.tiles.size());
    if (L.dim == 2) {
        // FP32 sweeps use strips of 8 rows (measured faster than the tiles on
        // every level: 4097^2 fine level 2.9 TB/s against 1.42, 1025^2 7.3 us
        // against 9.4); FP64 sweeps, bound by the FP64 pipe, keep the tiles
        const std::vector<int32_t> st = strips_for(L, 8);
        g.strip_rows = 8;
        g.nstrips = (int)st.size();
        g.strips = upload<int32_t>(c, st.data(), st.size());
    }
    if (!L.zm.empty()) {
        g.nzm = (int)(L.zm.size() / 2);
        g.zm = upload<int32_t>(c, L.zm.data(), L.zm.size());
        g.zm_moff = upload<int32_t>(c, L.zm_moff.data(), L.zm_moff.size());
        g.zm_mask = upload<uint32_t>(c, L.zm_mask.data(), L.zm_mask.size());
    }
    if (!L.sr.empty()) {
        g.nsr = (int)(L.sr.size() / 2);
        g.sr = upload<int32_t>(c, L.sr.data(), L.sr.size());
    }
    if (!L.sp.empty()) {
        g.nsp = (int)(L.sp.size() / 4);
        g.sp_cols = L.sp_cols;
        g.sp = upload<int32_t>(c, L.sp.data(), L.sp.size());
        g.sp_rows = upload<int32_t>(c, L.sp_rows.data(), L.sp_rows.size());
    }
    if (!L.sp_list.empty()) {
        g.nspl = (int)(L.sp_list.size() / 2);
        g.sp_list = upload<int32_t>(c, L.sp_list.data(), L.sp_list.size());
    }
    if (!L.chunk.empty()) {
        g.nchunks = (int64_t)L.chunk.size();
        g.chunks = upload<int32_t>(c, L.chunk.data(), L.chunk.size());
        g.chunk_len = upload<uint8_t>(c, L.chunk_len.data(), L.chunk_len.size());
    }
    g.black = upload<int32_t>(c, L.band_black.data(), L.band_black.size());
    g.enode = upload<int32_t>(c, L.ext_node.data(), L.ext_node.size());
    g.ecnt = upload<uint8_t>(c, L.ext_cnt.data(), L.ext_cnt.size());
    std::vector<int32_t> es = slot_major<int32_t, int32_t>(L.ext_src, g.ne, EMAX, EMAX);
    g.esrc = upload<int32_t>(c, es.data(), es.size());
    g.wave = L.ext_wave;
    g.gt_ptr = upload<int32_t>(c, L.gt_ptr.data(), L.gt_ptr.size());
    if (!L.partial_coarse.empty()) {
        g.npartial = (int)L.partial_coarse.size();
        g.partial_coarse = upload<int32_t>(c, L.partial_coarse.data(), L.partial_coarse.size());
    }
    g.gt_col = upload<int32_t>(c, L.gt_col.data(), L.gt_col.size());
    if (l + 1 == (int)c->H.size()) {
        g.nunk = (int)L.unk_node.size();
        g.unk_node = upload<int32_t>(c, L.unk_node.data(), L.unk_node.size());
        g.unk_ghost = upload<int32_t>(c, L.unk_ghost.data(), L.unk_ghost.size());
    }
    ck(cudaStreamSynchronize(c->stream), "sync");
    c->G.push_back(g);
}

void free_tracked(gcmg_ctx *c, void *p) {
    if (!p) return;
    for (size_t i = 0; i < c->allocs.size(); i++)
        if (c->allocs[i] == p) {
            cudaFree(p);
            c->allocs.erase(c->allocs.begin() + i);
            return;
        }
}

// (re)uploads a local program of level l
void upload_program(gcmg_ctx *c, const LocalProgram &J, LocalDev &z) {
    int32_t **arrs[] = {&z.node_off, &z.wb_cnt, &z.lnode, &z.int_off, &z.red_cnt, &z.int_glob,
                        &z.int_me, &z.int_nb, &z.gh_off, &z.gh_me, &z.gh_q, &z.gh_stn,
                        &z.zred, &z.zblack, &z.zghost, &z.wb_list, &z.node_base,
                        &z.pre_off, &z.pre_red_cnt, &z.pre_me, &z.pre_nb, &z.pre_glob, &z.zred_src};
    for (int32_t **a : arrs) { free_tracked(c, *a); *a = nullptr; }
    z.ncomp = J.ncomp();
    z.max_nodes = J.max_nodes;
    z.max_int = J.max_int;
    z.max_gh = J.max_gh;
    z.max_pre = J.max_pre;
    z.max_colour = 0;
    for (int k = 0; k < J.ncomp(); k++)
        z.max_colour = std::max({z.max_colour, J.red_cnt[k], J.int_off[k + 1] - J.int_off[k] - J.red_cnt[k]});
    z.nzred = z.nzblack = z.nzghost = 0;
    if (z.ncomp == 0) return;
    z.node_off = upload<int32_t>(c, J.node_off.data(), J.node_off.size());
    z.wb_cnt = upload<int32_t>(c, J.wb_cnt.data(), J.wb_cnt.size());
    z.lnode = upload<int32_t>(c, J.lnode.data(), J.lnode.size());
    z.node_base = upload<int32_t>(c, J.node_base.data(), J.node_base.size());
    z.has_pre = !J.pre_me.empty();
    z.pre_off = upload<int32_t>(c, J.pre_off.data(), J.pre_off.size());
    z.pre_red_cnt = upload<int32_t>(c, J.pre_red_cnt.data(), J.pre_red_cnt.size());
    z.pre_me = upload<int32_t>(c, J.pre_me.data(), J.pre_me.size());
    z.pre_nb = upload<int32_t>(c, J.pre_nb.data(), J.pre_nb.size());
    z.pre_glob = upload<int32_t>(c, J.pre_glob.data(), J.pre_glob.size());
    z.int_off = upload<int32_t>(c, J.int_off.data(), J.int_off.size());
    z.red_cnt = upload<int32_t>(c, J.red_cnt.data(), J.red_cnt.size());
    z.int_glob = upload<int32_t>(c, J.int_glob.data(), J.int_glob.size());
    z.int_me = upload<int32_t>(c, J.int_me.data(), J.int_me.size());
    z.int_nb = upload<int32_t>(c, J.int_nb.data(), J.int_nb.size());
    z.gh_off = upload<int32_t>(c, J.gh_off.data(), J.gh_off.size());
    z.gh_me = upload<int32_t>(c, J.gh_me.data(), J.gh_me.size());
    z.gh_q = upload<int32_t>(c, J.gh_q.data(), J.gh_q.size());
    z.gh_stn = upload<int32_t>(c, J.gh_stn.data(), J.gh_stn.size());
    z.nzred = (int)J.zred.size();
    z.nzblack = (int)J.zblack.size();
    z.nzghost = (int)J.zghost.size();
    z.zred = upload<int32_t>(c, J.zred.data(), J.zred.size());
    z.zblack = upload<int32_t>(c, J.zblack.data(), J.zblack.size());
    z.zghost = upload<int32_t>(c, J.zghost.data(), J.zghost.size());
    z.zred_src = J.zred_src.empty() ? nullptr : upload<int32_t>(c, J.zred_src.data(), J.zred_src.size());
    z.blocked = J.blocked;
    std::vector<int32_t> wb;
    for (int k = 0; k < z.ncomp; k++)
        wb.insert(wb.end(), J.lnode.begin() + J.node_off[k], J.lnode.begin() + J.node_off[k] + J.wb_cnt[k]);
    z.nwb = (int)wb.size();
    z.wb_list = upload<int32_t>(c, wb.data(), wb.size());
    ck(cudaStreamSynchronize(c->stream), "sync");
}

// sets NODE_WB in the device type grid of level l at the boundary blocks'
// write-back nodes (the host types stay as built)
void mark_writeback(gcmg_ctx *c, int l) {
    const HostLevel &L = c->H[l];
    const LocalProgram &J = L.boundary;
    if (J.ncomp() == 0) return;
    std::vector<uint8_t> t(L.type);
    for (int k = 0; k < J.ncomp(); k++)
        for (int i = J.node_off[k]; i < J.node_off[k] + J.wb_cnt[k]; i++) t[J.lnode[i]] |= NODE_WB;
    ck(cudaMemcpy(c->G[l].type, t.data(), t.size(), cudaMemcpyHostToDevice), "types");
}

template <typename T>
std::vector<DevData<T>> &data(gcmg_ctx *c);
template <>
std::vector<DevData<double>> &data<double>(gcmg_ctx *c) { return c->D64; }
template <>
std::vector<DevData<float>> &data<float>(gcmg_ctx *c) { return c->D32; }

// values moved by one boundary-block launch of level l: each distinct
// staged node (u read), inside entry (f read), ghost (3^d weights, g, mu dt)
// and write-back node (u write) once; halo re-reads of overlapping blocks
// and the program's index arrays are not counted
int64_t boundary_units(const HostLevel &L) {
    const LocalProgram &J = L.boundary;
    if (J.ncomp() == 0) return 0;
    std::vector<uint8_t> seen(L.nn, 0), gseen(L.ng(), 0);
    int64_t units = 0;
    for (int32_t p : J.lnode)
        if (!(seen[p] & 1)) { seen[p] |= 1; units++; }
    for (int32_t p : J.int_glob)
        if (!(seen[p] & 2)) { seen[p] |= 2; units++; }
    const int K = L.dim == 2 ? 9 : 27;
    for (int32_t q : J.gh_q)
        if (!gseen[q]) { gseen[q] = 1; units += K + 2; }
    for (int32_t w : J.wb_cnt) units += w;
    return units;
}

// events around the launches of the kernel class being timed (fine level;
// every level for the boundary blocks); `bytes`: that launch's algorithmic bytes
void timer_mark(gcmg_ctx *c, int kind, int l, double bytes = 0.0) {
    if (c->timing_kind != kind || (l != 0 && kind != GCMG_KERNEL_BOUNDARY)) return;
    if (c->events_used % 2 == 0) c->timed_bytes += bytes;
    if (c->events_used == c->events.size()) {
        if (c->events.size() >= 65536) return;
        cudaEvent_t e;
        ck(cudaEventCreate(&e), "cudaEventCreate");
        c->events.push_back(e);
    }
    ck(cudaEventRecord(c->events[c->events_used++], c->stream), "cudaEventRecord");
}

// One relaxation R_h followed by the lambda extra sweeps (Sec. 2.4, 3.2) and
// the junction relaxation.  2D: the sweep reads v.u and writes `out`, every
// later step works on `out` in place; 3D: in place on v.u.  `wb` is a free
// grid that takes the boundary blocks' write-back.  Returns the grid that
// holds u afterwards.
template <typename T>
T *relax(gcmg_ctx *c, LevelView<T> v, T *out, T *wb, int l, bool extra) {
    const int dim = c->p.dim;
    const DevGeom &g = c->G[l];
    if constexpr (std::is_same<T, float>::value) {
        // FP32 2D: the interior sweep, the ghost sweep and the band sweeps in one
        // launch (strips and boundary blocks both read v.u, write out); the
        // blocks store straight into out, so no write-back is pending
        if (dim == 2 && extra && g.nstrips > 0 && g.bz.ncomp > 0 && g.bz.in_smem && g.bz.pre_in_smem) {
            // algorithmic bytes: the interior sweep's (u, f read and u written
            // once per inside node) and the boundary blocks' distinct values
            const double bytes = c->timing_kind >= 0
                                     ? ((double)c->bz_units[l] + 3.0 * (double)c->H[l].n_in) * sizeof(T)
                                     : 0.0;
            timer_mark(c, GCMG_KERNEL_SMOOTH, l, bytes);
            timer_mark(c, GCMG_KERNEL_BOUNDARY, l, bytes);
            if (c->split2d_strips > 0 && g.nstrips >= c->split2d_strips) {
                if (!c->sstream) {
                    ck(cudaStreamCreateWithFlags(&c->sstream, cudaStreamNonBlocking), "cudaStreamCreate");
                    ck(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "cudaEventCreate");
                    ck(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "cudaEventCreate");
                }
                launch_relax2d_split(v, out, g, lview<T>(g.bz, v), c->p.lambda, c->stream, c->sstream, c->ev_fork,
                                     c->ev_join);
            } else {
                launch_relax2d(v, out, g, lview<T>(g.bz, v), c->p.lambda, c->stream);
            }
            timer_mark(c, GCMG_KERNEL_BOUNDARY, l);
            timer_mark(c, GCMG_KERNEL_SMOOTH, l);
            v.u = out;
            if (c->p.junction_solve) {
                const DevData<T> &D = data<T>(c)[l];
                launch_junction_solve<T>(v, g, D.js_inv, D.js_r, c->stream, nullptr);
            } else if (c->p.junction_sweeps > 0 && g.jz.ncomp > 0) {
                if (g.jz.in_smem) {
                    launch_local<T>(lview<T>(g.jz, v), dim, 0, c->p.junction_sweeps, c->stream);
                } else {
                    for (int k = 0; k < c->p.junction_sweeps; k++) {
                        launch_rb_list<T>(v, dim, g.jz.zred, g.jz.nzred, c->stream);
                        launch_rb_list<T>(v, dim, g.jz.zblack, g.jz.nzblack, c->stream);
                        launch_ghost_relax_list<T>(v, dim, g.jz.zghost, g.jz.nzghost, c->stream);
                    }
                }
            }
            return v.u;
        }
    }
    if (dim == 2) {
        timer_mark(c, GCMG_KERNEL_SMOOTH, l);
        if (sizeof(T) == 4 && g.nstrips > 0) launch_rb_strip<T>(v, out, g, c->stream);
        else launch_rb_fused2d<T>(v, out, g.tiles, g.ntiles, c->stream);
        timer_mark(c, GCMG_KERNEL_SMOOTH, l);
        v.u = out;
        if (c->p.smoother == 1) {   // the Kaczmarz comparison (plain FP64 only)
            if constexpr (std::is_same<T, double>::value)
                launch_kaczmarz(v, c->kz_rows[l], c->kz_off[l], extra ? c->p.lambda : 1, c->stream);
            return v.u;
        }
    } else if (g.nzm > 0) {
        // 3D: both colours in one pass over the active tiles (reads v.u, writes out)
        const double bytes = c->timing_kind >= 0 ? 3.0 * (double)c->H[l].n_in * sizeof(T) : 0.0;
        timer_mark(c, GCMG_KERNEL_SMOOTH, l, bytes);
        bool done = false, in_place = false;
        if (c->sweep3d == 3) done = in_place = launch_rb_rows<T>(v, g, c->stream);
        if constexpr (std::is_same<T, float>::value)
            if (!done && c->sweep3d == 2) done = launch_rb_span3d(v, out, g, c->stream);
        if (!done && c->sweep3d >= 1 && g.nsr > 0) launch_rb_stream3d<T>(v, out, g, c->stream);
        else if (!done) launch_rb_zmarch<T>(v, out, g, c->stream);
        timer_mark(c, GCMG_KERNEL_SMOOTH, l);
        if (!in_place) v.u = out;
    } else {
        for (int colour = 0; colour < 2; colour++) {
            timer_mark(c, GCMG_KERNEL_SMOOTH, l);
            launch_rb<T>(v, dim, colour, c->stream);
            timer_mark(c, GCMG_KERNEL_SMOOTH, l);
        }
    }
    LocalView<T> bzv{};
    const LocalView<T> *pending = nullptr;   // boundary-block write-back still to do
    if (extra && g.bz.ncomp > 0 && g.bz.in_smem) {
        // ghost sweep + lambda band sweeps in one shared-memory launch
        bzv = lview<T>(g.bz, v, wb);
        const double bytes = c->timing_kind == GCMG_KERNEL_BOUNDARY ? (double)c->bz_units[l] * sizeof(T) : 0.0;
        timer_mark(c, GCMG_KERNEL_BOUNDARY, l, bytes);
        launch_local<T>(bzv, dim, 1, c->p.lambda, c->stream);
        timer_mark(c, GCMG_KERNEL_BOUNDARY, l);
        if (bzv.wb) pending = &bzv;
    } else {
        // 3D: one launch a phase (default); gcmg_set_boundary3d 1: on levels
        // whose lists hold at most kClusterWork entries the ghost sweep, the
        // band sweeps and (on global lists) the junction sweeps as one
        // thread-block cluster with hardware barriers between the phases;
        // 2: all phases as one grid with software barriers
        bool done = false, zdone = false;
        BoundaryProgram3 P;
        const bool jz_smem = dim == 3 && sizeof(T) == 4 ? g.jz.in_smem32 : g.jz.in_smem;
        if (dim == 3 && c->p.smoother == 0 && g.ng > 0) {
            P.red = g.red;
            P.nred = g.nred;
            P.black = g.black;
            P.nblack = g.nblack;
            P.lambda = extra ? c->p.lambda : 0;
            const bool jglob =
                extra && !c->p.junction_solve && c->p.junction_sweeps > 0 && g.jz.ncomp > 0 && !jz_smem;
            if (jglob) {
                P.zred = g.jz.zred;
                P.nzred = g.jz.nzred;
                P.zblack = g.jz.zblack;
                P.nzblack = g.jz.nzblack;
                P.zghost = g.jz.zghost;
                P.nzghost = g.jz.nzghost;
                P.mu = c->p.junction_sweeps;
            }
            P.bar = c->d_bar;
            P.err = c->d_err;
            P.spin = c->bar_spin;
            timer_mark(c, GCMG_KERNEL_BOUNDARY, l);
            if (c->coop3d) {
                done = launch_boundary3d<T>(v, P, c->bar_phantom, c->stream);
                zdone = done && jglob;
            } else if (c->cluster3d) {
                const int64_t big = std::max<int64_t>({(int64_t)g.ng, g.nred, g.nblack, (int64_t)P.nzred,
                                                       (int64_t)P.nzblack, (int64_t)P.nzghost});
                if (big <= kClusterWork) {
                    done = launch_boundary3d_cluster<T>(v, P, c->stream);
                    zdone = done && jglob;
                }
            }
            if (done) timer_mark(c, GCMG_KERNEL_BOUNDARY, l);
        }
        // mode 0 in 3D: the store of each Jacobi ghost sweep (its new values
        // wait in gtmp) is merged into the launch of the next red sweep,
        // whose updates read the ghosts' new values from gtmp (red_sources):
        // three launches a band or junction sweep instead of four
        const bool merged = !done && dim == 3 && extra && c->p.smoother == 0 && g.ng > 0 && g.red_src &&
                            !c->coop3d;
        if (merged) {
            const bool zmerge = !c->p.junction_solve && c->p.junction_sweeps > 0 && g.jz.ncomp > 0 &&
                                !jz_smem && g.jz.zred_src;
            launch_ghost_new<T>(v, nullptr, g.ng, c->stream);
            for (int k = 0; k < c->p.lambda; k++) {
                launch_rb_list_store<T>(v, g.red, g.red_src, g.nred, nullptr, g.ng, c->stream);
                launch_rb_list<T>(v, dim, g.black, g.nblack, c->stream);
                launch_ghost_new<T>(v, nullptr, g.ng, c->stream);
            }
            timer_mark(c, GCMG_KERNEL_BOUNDARY, l);
            if (zmerge) {   // the first red zone sweep stores every ghost, later ones the zone's
                for (int k = 0; k < c->p.junction_sweeps; k++) {
                    launch_rb_list_store<T>(v, g.jz.zred, g.jz.zred_src, g.jz.nzred, k == 0 ? nullptr : g.jz.zghost,
                                            k == 0 ? g.ng : g.jz.nzghost, c->stream);
                    launch_rb_list<T>(v, dim, g.jz.zblack, g.jz.nzblack, c->stream);
                    launch_ghost_new<T>(v, g.jz.zghost, g.jz.nzghost, c->stream);
                }
                launch_ghost_store<T>(v, g.jz.zghost, g.jz.nzghost, c->stream);
                return v.u;
            }
            launch_ghost_store<T>(v, nullptr, g.ng, c->stream);
        } else if (!done) {
            launch_ghost_relax<T>(v, dim, c->stream);
            if (extra)
                for (int k = 0; k < c->p.lambda; k++) {
                    launch_rb_list<T>(v, dim, g.red, g.nred, c->stream);
                    launch_rb_list<T>(v, dim, g.black, g.nblack, c->stream);
                    launch_ghost_relax<T>(v, dim, c->stream);
                }
            if (dim == 3 && c->p.smoother == 0 && g.ng > 0) timer_mark(c, GCMG_KERNEL_BOUNDARY, l);
        }
        if (!extra || zdone) return v.u;
    }
    if (c->p.junction_solve) {
        const DevData<T> &D = data<T>(c)[l];
        launch_junction_solve<T>(v, g, D.js_inv, D.js_r, c->stream, pending);
        return v.u;
    }
    if (pending) launch_local_copyback<T>(*pending, c->stream);
    if (c->p.junction_sweeps > 0 && g.jz.ncomp > 0) {
        const bool jz_smem = dim == 3 && sizeof(T) == 4 ? g.jz.in_smem32 : g.jz.in_smem;
        if (jz_smem && g.jz.blocked) {   // overlapping blocks: write back through wb, then copy
            const LocalView<T> J = lview<T>(g.jz, v, wb);
            launch_local<T>(J, dim, 0, c->p.junction_sweeps, c->stream);
            launch_local_copyback<T>(J, c->stream);
        } else if (jz_smem) {
            launch_local<T>(lview<T>(g.jz, v), dim, 0, c->p.junction_sweeps, c->stream);
        } else {
            for (int k = 0; k < c->p.junction_sweeps; k++) {
                launch_rb_list<T>(v, dim, g.jz.zred, g.jz.nzred, c->stream);
                launch_rb_list<T>(v, dim, g.jz.zblack, g.jz.nzblack, c->stream);
                launch_ghost_relax_list<T>(v, dim, g.jz.zghost, g.jz.nzghost, c->stream);
            }
        }
    }
    return v.u;
}

// decides whether a program's components fit in shared memory
void check_program_fits(gcmg_ctx *c, LocalDev &z) {
    if (z.ncomp == 0) return;
    LevelView<double> dummy{};
    const size_t need = local_smem_bytes<double>(lview<double>(z, dummy), c->p.dim);
    int dev_max = 0;
    ck(cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device), "attr");
    z.in_smem = need <= (size_t)dev_max && local_fits_registers(z.max_int);
    LevelView<float> dummy32{};
    z.in_smem32 = local_smem_bytes<float>(lview<float>(z, dummy32), c->p.dim) <= (size_t)dev_max &&
                  local_fits_registers(z.max_int);
    if (!z.in_smem && !z.in_smem32) return;    // relaxed from global memory instead
    z.pre_in_smem = z.in_smem && z.has_pre &&
                    local_smem_bytes<float>(lview<float>(z, dummy32), c->p.dim, true) <= (size_t)dev_max;
    // the attribute is per kernel: allow the device maximum once for all levels
    local_prepare<double>(c->p.dim, (size_t)dev_max);
    local_prepare<float>(c->p.dim, (size_t)dev_max);
}

// TGCS (Sec. 2.4) applied recursively: V (gamma = 1) or W (gamma = 2) cycle
// on level l starting from u (one of the level's two grids); returns the grid
// that holds the level's u at the end.
template <typename T>
T *cycle(gcmg_ctx *c, int l, T *u) {
    std::vector<DevData<T>> &D = data<T>(c);
    const int last = (int)c->H.size() - 1;
    const int dim = c->p.dim;
    auto at = [&](int k, T *p) {
        LevelView<T> v = view<T>(c, k, D[k]);
        v.u = p;
        return v;
    };
    auto other = [&](T *p) { return p == D[l].u ? D[l].u2 : D[l].u; };
    if (sizeof(T) == 4 && l == c->coarse_l0) {   // the rest of the cycle in one launch (from D[l].u)
        launch_coarse_cycle(c);
        return ((c->p.nu1 + c->p.nu2) & 1) ? D[l].u2 : D[l].u;
    }
    if (l == last) {
        launch_coarse_solve<T>(at(l, u), c->G[l], D[l].Ainv, c->stream);
        return u;
    }
    for (int k = 0; k < c->p.nu1; k++) u = relax<T>(c, at(l, u), other(u), D[l].r, l, true);
    // defect (TGCS step 3), composite restriction (step 4) with the defect
    // extension at the coarse ghosts (Sec. 2.6), and e_2h = 0: one launch
    timer_mark(c, GCMG_KERNEL_RESTRICT, l);
    launch_descend<T>(at(l, u), at(l + 1, D[l + 1].u), c->G[l], D[l].gt_val, D[l + 1].f, D[l + 1].gg, D[l + 1].u,
                      c->stream, D[l].pt_w);
    timer_mark(c, GCMG_KERNEL_RESTRICT, l);
    const int gam = (l + 1 == last) ? 1 : c->p.gamma;
    T *uc = D[l + 1].u;
    for (int k = 0; k < gam; k++) uc = cycle<T>(c, l + 1, uc);
    timer_mark(c, GCMG_KERNEL_PROLONG, l);
    launch_prolong<T>(at(l, u), at(l + 1, uc), dim, uc, u, true, c->stream);
    timer_mark(c, GCMG_KERNEL_PROLONG, l);
    for (int k = 0; k < c->p.nu2; k++) u = relax<T>(c, at(l, u), other(u), D[l].r, l, true);
    return u;
}

// ||(f, g)||_inf: f over the inside nodes (those of the active chunks where
// the level has them), g over the ghosts
__global__ void k_rhs_norm(LevelView<double> lv, const double *g, int ng, unsigned long long *bits) {
    __shared__ double wmax[32];
    const uint8_t *type = lv.type;
    const double *f = lv.f;
    const int64_t nt = lv.chunks ? lv.nchunks * CHUNK : lv.nn;
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt || i < ng;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = i;
        bool ok = i < nt;
        if (ok && lv.chunks) {   // thread i: node i % CHUNK of chunk i / CHUNK
            ok = (int)(i % CHUNK) < (lv.clen[i / CHUNK] & 63);
            p = (int64_t)lv.chunks[i / CHUNK] + i % CHUNK;
        }
        if (ok && (type[p] & NODE_KIND) == NODE_IN) v = fmax(v, fabs(f[p]));
        if (i < ng) v = fmax(v, fabs(g[i]));
        if (v != v) v = __longlong_as_double(0x7ff0000000000000ll);
    }
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0 && v > 0.0) atomicMax(bits, (unsigned long long)__double_as_longlong(v));
    }
}

double read_norm(gcmg_ctx *c) {
    ck(cudaMemcpyAsync(c->h_norm, c->d_norm, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream),
       "norm");
    ck(cudaStreamSynchronize(c->stream), "sync");
    double v;
    std::memcpy(&v, c->h_norm, sizeof(double));
    return v;
}

// FP64 defect of level 0 and its norm; in the mixed form it also sets up
// the next FP32 correction problem (see launch_defect_mixed)
void fine_defect(gcmg_ctx *c) {
    ck(cudaMemsetAsync(c->d_norm, 0, sizeof(unsigned long long), c->stream), "memset");
    if (c->p.precision == 0)
        launch_defect<double>(view<double>(c, 0, c->D64[0]), c->p.dim, false, c->d_norm, c->stream);
    else
        launch_defect_mixed(view<double>(c, 0, c->D64[0]), c->p.dim, c->d_norm, c->D32[0].f, c->D32[0].gg,
                            c->D32[0].u, c->stream);
}

double fine_defect_norm(gcmg_ctx *c) {
    fine_defect(c);
    return read_norm(c);
}

// whether a bounded barrier wait of k_boundary3d ran out since the last
// check (synchronises the stream); if so the flag and the barrier words are
// cleared for the next launch
bool barrier_timed_out(gcmg_ctx *c) {
    if (!c->d_err) return false;
    int e = 0;
    ck(cudaMemcpyAsync(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "err");
    ck(cudaStreamSynchronize(c->stream), "sync");
    if (!e) return false;
    ck(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream), "memset");
    ck(cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned), c->stream), "memset");
    ck(cudaStreamSynchronize(c->stream), "sync");
    return true;
}

// end of one loop iteration: records rel[m] and sets the while condition;
// r0[1] holds the previous relative residual, m[1] the number of consecutive
// cycles whose defect grew (the loop stops once it reaches `diverge` > 0),
// m[2] the cycle limit (device-resident, so gcmg_set_max_cycles needs no new graph)
__global__ void k_loop_check(cudaGraphConditionalHandle h, const unsigned long long *bits, double *r0,
                             double *rel, int *m, double rtol, int diverge) {
    const int max_cycles = m[2];
    const double nr = __longlong_as_double((long long)*bits);
    const int k = m[0] + 1;
    m[0] = k;
    const double v = nr / r0[0];
    if (k <= 256) rel[k] = v;
    m[1] = v > r0[1] ? m[1] + 1 : 0;
    r0[1] = v;
    const bool grew = diverge > 0 && m[1] >= diverge;
    const bool go = (v == v) && !isinf(v) && v > rtol && k < max_cycles && !grew;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// start of a graph solve: r0 = ||(f, g)|| (slot 1 of d_norm) and the
// defect's norm (slot 0) are on the device; records r0 and rel[0], zeroes
// the cycle count and opens the loop unless the start already converged
__global__ void k_loop_start(cudaGraphConditionalHandle h, const unsigned long long *bits, double *r0_out,
                             double *rel, int *m, double rtol) {
    const double r0 = __longlong_as_double((long long)bits[1]);
    const double rel0 = r0 > 0.0 ? __longlong_as_double((long long)bits[0]) / r0 : 0.0;
    r0_out[0] = r0;
    r0_out[1] = rel0;
    rel[0] = rel0;
    m[0] = 0;
    m[1] = 0;
    cudaGraphSetConditional(h, (r0 > 0.0 && !(rel0 <= rtol)) ? 1u : 0u);
}

// what precedes the loop in a graph solve: ||(f, g)||, the first defect and
// its norm (in the mixed form also the first FP32 problem), k_loop_start
void solve_prologue(gcmg_ctx *c, cudaGraphConditionalHandle h) {
    const DevGeom &g0 = c->G[0];
    const HostLevel &L0 = c->H[0];
    ck(cudaMemsetAsync(c->d_norm + 1, 0, sizeof(unsigned long long), c->stream), "memset");
    const LevelView<double> lv = view<double>(c, 0, c->D64[0]);
    const int64_t cnt = std::max<int64_t>(lv.chunks ? lv.nchunks * CHUNK : L0.nn, L0.ng());
    const unsigned nb = (unsigned)std::min<int64_t>((cnt + 255) / 256, 4096);
    k_rhs_norm<<<nb, 256, 0, c->stream>>>(lv, c->D64[0].gg, g0.ng, c->d_norm + 1);
    g_launches++;
    fine_defect(c);
    k_loop_start<<<1, 1, 0, c->stream>>>(h, c->d_norm, c->d_r0, c->d_rel, c->d_m, c->p.rtol);
    g_launches++;
}

// one iteration of the solve loop: a cycle (plain) or a refinement step
// (mixed), then the FP64 defect and its norm
void loop_body(gcmg_ctx *c) {
    const DevGeom &g0 = c->G[0];
    const HostLevel &L0 = c->H[0];
    if (c->p.precision == 0) {
        double *u = cycle<double>(c, 0, c->D64[0].u);
        // an odd number of 2D sweeps leaves u in the second grid: the loop
        // body must end where it starts
        if (u != c->D64[0].u)
            ck(cudaMemcpyAsync(c->D64[0].u, u, L0.nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "copy");
    } else {
        // the FP32 problem (right-hand side, e = 0) was set up by the FP64
        // defect that ended the previous iteration or preceded the loop
        float *e = cycle<float>(c, 0, c->D32[0].u);
        launch_add_correction(g0, c->D64[0].u, e, c->stream);
    }
    fine_defect(c);
}

void destroy_graph(gcmg_ctx *c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
}

void build_graph(gcmg_ctx *c) {
    destroy_graph(c);
    if (!c->gstream) ck(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!c->ev_in) ck(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming), "cudaEventCreate");
    if (!c->ev_out) ck(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming), "cudaEventCreate");
    if (!c->h_res) ck(cudaMallocHost((void **)&c->h_res, sizeof(gcmg_ctx::SolveResult)), "cudaMallocHost");
    ck(cudaGraphCreate(&c->graph, 0), "cudaGraphCreate");
    cudaGraphConditionalHandle h;
    ck(cudaGraphConditionalHandleCreate(&h, c->graph, 1, cudaGraphCondAssignDefault), "conditional handle");
    // the prologue, captured into the graph ahead of the loop node
    cudaStream_t saved0 = c->stream;
    c->stream = c->gstream;
    ck(cudaStreamBeginCaptureToGraph(c->gstream, c->graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
       "begin capture");
    const long long before0 = g_launches.load();
    try {
        solve_prologue(c, h);
        c->graph_pro_kernels = g_launches.load() - before0;
        g_launches -= c->graph_pro_kernels;   // counted when executed
    } catch (...) {
        cudaGraph_t dummy;
        cudaStreamEndCapture(c->gstream, &dummy);
        c->stream = saved0;
        throw;
    }
    c->stream = saved0;
    {
        cudaGraph_t captured;
        ck(cudaStreamEndCapture(c->gstream, &captured), "end capture");
    }
    // the prologue is a chain: its one node without dependents precedes the loop
    size_t nn = 0;
    ck(cudaGraphGetNodes(c->graph, nullptr, &nn), "graph nodes");
    std::vector<cudaGraphNode_t> nodes(nn);
    ck(cudaGraphGetNodes(c->graph, nodes.data(), &nn), "graph nodes");
    std::vector<cudaGraphNode_t> leaves;
    for (cudaGraphNode_t x : nodes) {
        size_t nd = 0;
        ck(cudaGraphNodeGetDependentNodes(x, nullptr, nullptr, &nd), "graph edges");
        if (nd == 0) leaves.push_back(x);
    }
    alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)] = {};
    cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(np_raw);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    ck(cudaGraphAddNode(&node, c->graph, leaves.data(), nullptr, leaves.size(), &np), "cudaGraphAddNode");
    cudaGraph_t body = np.conditional.phGraph_out[0];
    cudaStream_t saved = c->stream;
    c->stream = c->gstream;
    ck(cudaStreamBeginCaptureToGraph(c->gstream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
       "begin capture");
    const long long before = g_launches.load();
    try {
        loop_body(c);
        k_loop_check<<<1, 1, 0, c->gstream>>>(h, c->d_norm, c->d_r0, c->d_rel, c->d_m, c->p.rtol,
                                              c->p.diverge_cycles);
        g_launches++;
        c->graph_kernels = g_launches.load() - before;
        g_launches -= c->graph_kernels;   // counted when executed
    } catch (...) {
        cudaGraph_t dummy;
        cudaStreamEndCapture(c->gstream, &dummy);
        c->stream = saved;
        throw;
    }
    c->stream = saved;
    cudaGraph_t captured;
    ck(cudaStreamEndCapture(c->gstream, &captured), "end capture");
    ck(cudaGraphInstantiate(&c->gexec, c->graph, 0), "cudaGraphInstantiate");
}

gcmg_status fail(gcmg_ctx *c, gcmg_status s, const std::string &m) {
    if (c) c->err = m;
    return s;
}

#define GCMG_GUARD(ctx, ...)                                                                  \
    try {                                                                                     \
        __VA_ARGS__                                                                           \
    } catch (const CudaFail &f) {                                                             \
        cudaGetLastError();                                                                   \
        return fail(ctx, GCMG_E_CUDA, std::string(f.what) + ": " + cudaGetErrorString(f.e));  \
    } catch (const GeomError &g) {                                                            \
        return fail(ctx, GCMG_E_GEOM, g.msg);                                                 \
    } catch (const std::bad_alloc &) {                                                        \
        return fail(ctx, GCMG_E_OOM, "allocation failed");                                    \
    } catch (const std::exception &e) {                                                       \
        return fail(ctx, GCMG_E_ARG, e.what());                                               \
    }

bool valid_level(const gcmg_ctx *c, int l) { return c && l >= 0 && l < (int)c->H.size(); }

void check_launch() { ck(cudaGetLastError(), "kernel launch"); }

}  // namespace

namespace gcmg {

gcmg_status check_params(const gcmg_params &q) {
    const gcmg_params *p = &q;
    if (p->dim < 2 || p->dim > 3 || p->n_coarse < 3 || p->n <= p->n_coarse) return GCMG_E_ARG;
    int m = p->n;
    while (m > p->n_coarse) {
        if ((m - 1) % 2) return GCMG_E_ARG;
        m = (m - 1) / 2 + 1;
    }
    if (m != p->n_coarse) return GCMG_E_ARG;
    const double nn = std::pow((double)p->n, p->dim);
    if (nn >= 2147483647.0) return GCMG_E_ARG;   // 32-bit node indices
    if (p->gamma < 1 || p->gamma > 2 || p->nu1 < 0 || p->nu2 < 0 || p->lambda < 0) return GCMG_E_ARG;
    if (p->precision < 0 || p->precision > 1 || p->max_cycles < 1 || p->max_cycles > 256) return GCMG_E_ARG;
    if (p->junction_sweeps < 0 || p->junction_radius < 0.0 || p->junction_radius > 64.0) return GCMG_E_ARG;
    if (p->junction_solve < 0 || p->junction_solve > 1 || p->fused_coarse_n < 0) return GCMG_E_ARG;
    if (p->smoother < 0 || p->smoother > 1) return GCMG_E_ARG;
    if (!(p->h >= 0.0) || !std::isfinite(p->h) || p->diverge_cycles < 0) return GCMG_E_ARG;
    for (int a = 0; a < p->dim; a++)
        if (!std::isfinite(p->origin[a])) return GCMG_E_ARG;
    if (p->smoother == 1 && (p->dim != 2 || p->precision != 0 || p->junction_solve || p->junction_sweeps))
        return GCMG_E_ARG;
    return GCMG_OK;
}

void prepare_levels(const gcmg_params &p, const double *phi_host, std::vector<HostLevel> &H) {
    build_hierarchy(p.dim, p.n, p.n_coarse, phi_host, p.delta_over_h, H, p.h, p.origin);
    if (p.dim == 2)
        for (auto &L : H) build_boundary_blocks(L, p.lambda, 32);
}

gcmg_status create_from_levels(const gcmg_params &q, std::vector<HostLevel> &&H, cudaStream_t stream, gcmg_ctx **out) {
    const gcmg_params *p = &q;
    gcmg_ctx *c = new (std::nothrow) gcmg_ctx;
    if (!c) return GCMG_E_OOM;
    *out = c;
    c->p = *p;
    c->stream = stream;
    c->H = std::move(H);
    GCMG_GUARD(c, {
        ck(cudaGetDevice(&c->device), "cudaGetDevice");
        const int nl = (int)c->H.size();
        for (int l = 0; l < nl; l++) upload_geometry(c, l);
        if (p->smoother == 1)
            for (int l = 0; l < nl; l++) build_kaczmarz_rows(c, l);
        if (p->dim == 2)
            for (int l = 0; l < nl; l++) {
                upload_program(c, c->H[l].boundary, c->G[l].bz);
                check_program_fits(c, c->G[l].bz);
                mark_writeback(c, l);
            }
        c->D64.resize(nl);
        for (int l = 0; l < nl; l++) alloc_data<double>(c, l, c->D64[l], p->precision == 0 || l == 0);
        if (p->precision == 1) {
            c->D32.resize(nl);
            for (int l = 0; l < nl; l++) alloc_data<float>(c, l, c->D32[l], true);
        }
        c->d_norm = dalloc<unsigned long long>(c, 2);
        c->d_rel = dalloc<double>(c, 257);
        c->d_r0 = dalloc<double>(c, 2);   // r0, the last relative residual
        c->d_m = dalloc<int>(c, 3);       // cycles, consecutive growing cycles, cycle limit
        c->d_bar = dalloc<unsigned>(c, 2);
        c->d_err = dalloc<int>(c, 1);
        const int maxc = p->max_cycles;
        ck(cudaMemcpyAsync(c->d_m + 2, &maxc, sizeof(int), cudaMemcpyHostToDevice, c->stream), "max cycles");
        ck(cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned), c->stream), "memset");
        ck(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream), "memset");
        ck(cudaMallocHost((void **)&c->h_norm, 2 * sizeof(unsigned long long)), "cudaMallocHost");
        ck(cudaStreamSynchronize(c->stream), "sync");
        return GCMG_OK;
    })
}

void upload_inverse(gcmg_ctx *c) {
    const HostLevel &L = c->H.back();
    const size_t m2 = L.unk_node.size() * L.unk_node.size();
    ck(cudaMemcpy(c->D64.back().Ainv, L.Ainv.data(), m2 * sizeof(double), cudaMemcpyHostToDevice), "Ainv");
    if (!c->D32.empty()) {
        std::vector<float> A(L.Ainv.begin(), L.Ainv.end());
        ck(cudaMemcpy(c->D32.back().Ainv, A.data(), m2 * sizeof(float), cudaMemcpyHostToDevice), "Ainv");
    }
}

// (re)uploads the exact junction solve of level l
void upload_js(gcmg_ctx *c, int l) {
    const HostLevel &L = c->H[l];
    DevGeom &g = c->G[l];
    for (int32_t **a : {&g.js_node, &g.js_ghost, &g.js_comp, &g.js_off, &g.js_roff, &g.js_rpos}) {
        free_tracked(c, *a);
        *a = nullptr;
    }
    free_tracked(c, g.js_aoff);
    g.js_aoff = nullptr;
    auto drop = [&](auto &D) {
        free_tracked(c, D.js_inv);
        free_tracked(c, D.js_r);
        D.js_inv = nullptr;
        D.js_r = nullptr;
    };
    drop(c->D64[l]);
    if (!c->D32.empty()) drop(c->D32[l]);
    g.js_n = (int)L.js_node.size();
    g.js_ncomp = L.js_off.empty() ? 0 : (int)L.js_off.size() - 1;
    g.js_rlen = 0;
    g.js_aoff_h.clear();
    g.js_roff_h.clear();
    if (g.js_n == 0) return;
    // padded device layout: component c's rows have mp = m rounded up to a
    // multiple of 4 entries, its defects occupy mp slots from roff[c]
    std::vector<int32_t> comp(g.js_n), rpos(g.js_n), roff(g.js_ncomp + 1);
    std::vector<int64_t> aoff(g.js_ncomp + 1);
    int64_t na = 0;
    int32_t nr = 0;
    for (int k = 0; k < g.js_ncomp; k++) {
        const int m = L.js_off[k + 1] - L.js_off[k], mp = (m + 3) & ~3;
        aoff[k] = na;
        roff[k] = nr;
        for (int i = 0; i < m; i++) {
            comp[L.js_off[k] + i] = k;
            rpos[L.js_off[k] + i] = nr + i;
        }
        na += (int64_t)m * mp;
        nr += mp;
    }
    aoff[g.js_ncomp] = na;
    roff[g.js_ncomp] = nr;
    g.js_rlen = nr;
    g.js_aoff_h = aoff;
    g.js_roff_h = roff;
    std::vector<double> inv((size_t)na, 0.0);
    for (int k = 0; k < g.js_ncomp; k++) {
        const int m = L.js_off[k + 1] - L.js_off[k], mp = (m + 3) & ~3;
        for (int i = 0; i < m; i++)
            std::copy_n(L.js_inv.begin() + L.js_aoff[k] + (int64_t)i * m, m, inv.begin() + aoff[k] + (int64_t)i * mp);
    }
    g.js_node = upload<int32_t>(c, L.js_node.data(), L.js_node.size());
    g.js_ghost = upload<int32_t>(c, L.js_ghost.data(), L.js_ghost.size());
    g.js_comp = upload<int32_t>(c, comp.data(), comp.size());
    g.js_off = upload<int32_t>(c, L.js_off.data(), L.js_off.size());
    g.js_roff = upload<int32_t>(c, roff.data(), roff.size());
    g.js_rpos = upload<int32_t>(c, rpos.data(), rpos.size());
    g.js_aoff = upload<int64_t>(c, aoff.data(), aoff.size());
    // FP64 for FP64 cycles and single relaxations (gcmg_relax), FP32 for FP32
    // cycles; the defect vectors start at zero and their pads stay zero
    if (c->p.precision == 0 || c->js64) {
        const std::vector<double> zero(nr, 0.0);
        c->D64[l].js_inv = upload<double>(c, inv.data(), inv.size());
        c->D64[l].js_r = upload<double>(c, zero.data(), zero.size());
    }
    if (!c->D32.empty()) {
        const std::vector<float> inv32(inv.begin(), inv.end()), zero(nr, 0.f);
        c->D32[l].js_inv = upload<float>(c, inv32.data(), inv32.size());
        c->D32[l].js_r = upload<float>(c, zero.data(), zero.size());
    }
    ck(cudaStreamSynchronize(c->stream), "sync");   // the staging vectors die at return
}

// builds and uploads the exact junction solves that are out of date with bc
void ensure_junction_solve(gcmg_ctx *c) {
    if (!c->p.junction_solve) return;
    for (int l = 0; l < (int)c->H.size(); l++) {
        HostLevel &L = c->H[l];
        if (!L.js_dirty) continue;
        destroy_graph(c);   // a captured graph holds the arrays reallocated below
        build_junction_solve(L, c->p.junction_radius);
        upload_js(c, l);
        L.js_dirty = false;
    }
}

void ensure_inverse(gcmg_ctx *c) {
    if (!c->H.back().ainv_dirty) return;
    build_coarse_inverse(c->H.back());
    upload_inverse(c);
}

}  // namespace gcmg

extern "C" {

gcmg_status gcmg_create_grid(const gcmg_grid *grid, const double *phi_dev, const gcmg_params *p, void *stream,
                             gcmg_ctx **out) {
    if (out) *out = nullptr;
    if (!grid || !p || !phi_dev || !out) return GCMG_E_ARG;
    if (grid->dim < 2 || grid->dim > 3 || !(grid->h > 0.0) || !std::isfinite(grid->h)) return GCMG_E_ARG;
    for (int a = 1; a < grid->dim; a++)
        if (grid->n[a] != grid->n[0]) return GCMG_E_ARG;
    if (grid->n[0] < 3 || grid->n[0] > 65537) return GCMG_E_ARG;
    gcmg_params q = *p;
    q.dim = grid->dim;
    q.n = (int)grid->n[0];
    q.h = grid->h;
    for (int a = 0; a < 3; a++) q.origin[a] = a < grid->dim ? grid->origin[a] : -1.0;
    return gcmg_create(&q, phi_dev, stream, out);
}

gcmg_status gcmg_default_params(gcmg_params *p, int dim, int n, int n_coarse) {
    if (!p) return GCMG_E_ARG;
    std::memset(p, 0, sizeof(*p));
    p->dim = dim;
    p->n = n;
    p->n_coarse = n_coarse;
    p->nu1 = 2;
    p->nu2 = 1;
    p->lambda = 5;
    p->gamma = 1;
    p->delta_over_h = 3.0;
    p->c_dirichlet = 0.9;
    p->c_neumann_factor = 0.9;
    p->precision = 0;
    p->max_cycles = 100;
    p->rtol = 1e-10;
    // 2D: an exact solve of the zone within 20h; 3D: the zone is a tube around
    // junction curves, too large for dense inverses, where 10 sweeps within 2h
    // keep the factor bounded (more sweeps on a wider 3D zone amplify a local
    // ghost mode)
    p->junction_solve = dim == 2 ? 1 : 0;
    p->junction_sweeps = dim == 3 ? 10 : 0;
    p->junction_radius = dim == 3 ? 2.0 : 20.0;
    p->fused_coarse_n = 0;   // measured slower than the per-level launches on GB300
    p->smoother = 0;
    p->h = 0.0;               // 2 / (n - 1): the box [-1,1]^d
    p->origin[0] = p->origin[1] = p->origin[2] = -1.0;
    p->diverge_cycles = 3;
    return GCMG_OK;
}

gcmg_status gcmg_create(const gcmg_params *p, const double *phi_dev, void *stream, gcmg_ctx **out) {
    if (!out) return GCMG_E_ARG;
    *out = nullptr;
    if (!p || !phi_dev) return GCMG_E_ARG;
    if (check_params(*p) != GCMG_OK) return GCMG_E_ARG;
    int64_t nn = 1;
    for (int a = 0; a < p->dim; a++) nn *= p->n;
    std::vector<double> phi(nn);
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(phi.data(), phi_dev, nn * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return GCMG_E_CUDA;
    }
    std::vector<HostLevel> H;
    try {
        prepare_levels(*p, phi.data(), H);
    } catch (const GeomError &g) {
        gcmg_ctx *c = new (std::nothrow) gcmg_ctx;
        if (!c) return GCMG_E_OOM;
        c->err = g.msg;
        *out = c;
        return GCMG_E_GEOM;
    } catch (const std::bad_alloc &) {
        return GCMG_E_OOM;
    }
    return create_from_levels(*p, std::move(H), s, out);
}

void gcmg_destroy(gcmg_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    destroy_graph(c);
    if (c->gstream) { cudaStreamSynchronize(c->gstream); cudaStreamDestroy(c->gstream); }
    if (c->sstream) { cudaStreamSynchronize(c->sstream); cudaStreamDestroy(c->sstream); }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    for (void *p : c->allocs) cudaFree(p);
    if (c->d_coarse) cudaFree(c->d_coarse);
    if (c->h_norm) cudaFreeHost(c->h_norm);
    if (c->h_res) cudaFreeHost(c->h_res);
    delete c;
}

const char *gcmg_last_error(const gcmg_ctx *c) { return c ? c->err.c_str() : "null context"; }

int gcmg_num_levels(const gcmg_ctx *c) { return c ? (int)c->H.size() : 0; }

int gcmg_level_n(const gcmg_ctx *c, int l) { return valid_level(c, l) ? c->H[l].n : 0; }

gcmg_status gcmg_num_ghosts(const gcmg_ctx *c, int l, int64_t *count) {
    if (!valid_level(c, l) || !count) return GCMG_E_ARG;
    *count = c->H[l].ng();
    return GCMG_OK;
}

gcmg_status gcmg_num_unknowns(const gcmg_ctx *c, int l, int64_t *count) {
    if (!valid_level(c, l) || !count) return GCMG_E_ARG;
    *count = c->H[l].n_in + c->H[l].ng();
    return GCMG_OK;
}

gcmg_status gcmg_ghost_geometry(const gcmg_ctx *c, int l, int64_t *node, double *B, double *nu, uint8_t *scase) {
    if (!valid_level(c, l)) return GCMG_E_ARG;
    const HostLevel &L = c->H[l];
    const int64_t ng = L.ng();
    for (int64_t q = 0; q < ng; q++) {
        if (node) node[q] = L.ghost_node[q];
        if (scase) scase[q] = L.scase[q];
    }
    if (B) std::memcpy(B, L.B.data(), sizeof(double) * ng * L.dim);
    if (nu) std::memcpy(nu, L.nu.data(), sizeof(double) * ng * L.dim);
    return GCMG_OK;
}

gcmg_status gcmg_ghost_equations(const gcmg_ctx *c, int l, int64_t *stn, double *wD, double *wN) {
    if (!valid_level(c, l)) return GCMG_E_ARG;
    const HostLevel &L = c->H[l];
    const int64_t total = L.ng() * KMAX;
    for (int64_t i = 0; i < total; i++) {
        if (stn) stn[i] = L.stn[i];
        if (wD) wD[i] = L.wD[i];
        if (wN) wN[i] = L.wN[i];
    }
    return GCMG_OK;
}

gcmg_status gcmg_node_types(const gcmg_ctx *c, int l, uint8_t *types) {
    if (!valid_level(c, l) || !types) return GCMG_E_ARG;
    std::memcpy(types, c->H[l].type.data(), c->H[l].nn);
    return GCMG_OK;
}

gcmg_status gcmg_set_bc_types(gcmg_ctx *c, int l, const uint8_t *types) {
    if (!valid_level(c, l) || !types) return fail(c, GCMG_E_ARG, "bad level or pointer");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        HostLevel &L = c->H[l];
        destroy_graph(c);   // the junction arrays are reallocated below
        c->version++;
        for (int64_t q = 0; q < L.ng(); q++) L.bc[q] = types[q] ? 1 : 0;
        if (l + 1 == (int)c->H.size()) L.ainv_dirty = true;   // rebuilt before the next solve
        if (c->p.junction_solve) {
            L.js_dirty = true;                                  // rebuilt before the next solve
        } else {
            build_junction(L, c->p.junction_radius, c->junction_blocks ? c->p.junction_sweeps : 0);
            upload_program(c, L.junction, c->G[l].jz);
            check_program_fits(c, c->G[l].jz);
        }
        upload_ghost_data<double>(c, l, c->D64[l], false);
        if (!c->D32.empty()) upload_ghost_data<float>(c, l, c->D32[l], false);
        return GCMG_OK;
    })
}

gcmg_status gcmg_debug_barrier(gcmg_ctx *c, int enable, int phantom_blocks, unsigned spin_limit) {
    if (!c || phantom_blocks < 0 || spin_limit == 0) return fail(c, GCMG_E_ARG, "bad argument");
    destroy_graph(c);   // a captured graph holds the old launch parameters
    c->coop3d = enable ? 1 : 0;
    c->cluster3d = 0;
    c->bar_phantom = phantom_blocks;
    c->bar_spin = spin_limit;
    return GCMG_OK;
}

gcmg_status gcmg_set_boundary3d(gcmg_ctx *c, int mode) {
    if (!c || mode < 0 || mode > 2) return fail(c, GCMG_E_ARG, "bad argument");
    destroy_graph(c);
    c->cluster3d = mode == 1 ? 1 : 0;
    c->coop3d = mode == 2 ? 1 : 0;
    return GCMG_OK;
}

gcmg_status gcmg_set_sweep3d(gcmg_ctx *c, int variant) {
    if (!c || variant < 0 || variant > 3) return fail(c, GCMG_E_ARG, "bad argument");
    destroy_graph(c);
    c->sweep3d = variant;
    return GCMG_OK;
}

gcmg_status gcmg_set_span3d(gcmg_ctx *c, int columns, int planes) {
    if (!c || columns < 0 || (columns > 0 && (columns < SP_CMIN || columns > SP_CMAX)) || planes < 0 ||
        planes > SP_SEG)
        return fail(c, GCMG_E_ARG, "bad argument");
    if (c->p.dim != 3) return GCMG_OK;
    GCMG_GUARD(c, {
        destroy_graph(c);
        ck(cudaStreamSynchronize(c->stream), "sync");
        for (size_t l = 0; l < c->H.size(); l++) {
            HostLevel &L = c->H[l];
            DevGeom &g = c->G[l];
            if (L.nn >= ((int64_t)1 << 31)) continue;
            build_span_items(L, columns, planes);
            g.nsp = 0;
            g.sp_cols = 0;
            if (L.sp.empty()) continue;
            g.sp_cols = L.sp_cols;
            g.sp = upload<int32_t>(c, L.sp.data(), L.sp.size());
            g.sp_rows = upload<int32_t>(c, L.sp_rows.data(), L.sp_rows.size());
            g.nsp = (int)(L.sp.size() / 4);
        }
        ck(cudaStreamSynchronize(c->stream), "sync");
    })
    return GCMG_OK;
}

gcmg_status gcmg_set_junction_blocks(gcmg_ctx *c, int enable) {
    if (!c) return GCMG_E_ARG;
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        destroy_graph(c);
        c->junction_blocks = enable ? 1 : 0;
        if (!c->p.junction_solve)
            for (size_t l = 0; l < c->H.size(); l++) {
                HostLevel &L = c->H[l];
                if (L.ng() == 0) continue;
                build_junction(L, c->p.junction_radius, c->junction_blocks ? c->p.junction_sweeps : 0);
                upload_program(c, L.junction, c->G[l].jz);
                check_program_fits(c, c->G[l].jz);
            }
        return GCMG_OK;
    })
}

gcmg_status gcmg_set_max_cycles(gcmg_ctx *c, int max_cycles) {
    if (!c || max_cycles < 1 || max_cycles > 256) return fail(c, GCMG_E_ARG, "max_cycles outside [1, 256]");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        c->p.max_cycles = max_cycles;
        // ordered before the next solve's graph launch, which waits on this stream
        ck(cudaMemcpyAsync(c->d_m + 2, &max_cycles, sizeof(int), cudaMemcpyHostToDevice, c->stream), "max cycles");
        ck(cudaStreamSynchronize(c->stream), "sync");
        return GCMG_OK;
    })
}

gcmg_status gcmg_set_split2d(gcmg_ctx *c, int min_strips) {
    if (!c || min_strips < 0) return fail(c, GCMG_E_ARG, "bad argument");
    destroy_graph(c);
    c->split2d_strips = min_strips;
    return GCMG_OK;
}

int gcmg_junction_mode(const gcmg_ctx *c, int l) {
    if (!valid_level(c, l)) return -1;
    const LocalDev &z = c->G[l].jz;
    const bool smem = c->p.dim == 3 && c->p.precision == 1 ? z.in_smem32 : z.in_smem;
    if (z.ncomp == 0 || !smem) return 0;
    return z.blocked ? 2 : 1;
}

gcmg_status gcmg_span3d_info(const gcmg_ctx *c, int l, int *items, int *columns) {
    if (!valid_level(c, l) || !items || !columns) return GCMG_E_ARG;
    *items = c->G[l].nsp;
    *columns = c->G[l].sp_cols;
    return GCMG_OK;
}

gcmg_status gcmg_bc_types(const gcmg_ctx *c, int l, uint8_t *types) {
    if (!valid_level(c, l) || !types) return GCMG_E_ARG;
    const HostLevel &L = c->H[l];
    if (L.ng() > 0) std::memcpy(types, L.bc.data(), (size_t)L.ng());
    return GCMG_OK;
}

gcmg_status gcmg_set_bc_types_from_mask(gcmg_ctx *c, const uint8_t *mask_dev) {
    if (!c || !mask_dev) return fail(c, GCMG_E_ARG, "null pointer");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        const HostLevel &F = c->H[0];
        int64_t mx = 0;
        for (const HostLevel &L : c->H) mx = std::max<int64_t>(mx, L.ng());
        if (mx == 0) return GCMG_OK;
        std::vector<void *> tmp;   // call-scoped device buffers
        auto scratch = [&](size_t bytes) {
            void *p = nullptr;
            if (cudaMalloc(&p, bytes) != cudaSuccess) {
                cudaGetLastError();
                for (void *q : tmp) cudaFree(q);
                throw std::bad_alloc();
            }
            tmp.push_back(p);
            return p;
        };
        double *B = static_cast<double *>(scratch((size_t)mx * F.dim * sizeof(double)));
        int32_t *gn = static_cast<int32_t *>(scratch((size_t)mx * sizeof(int32_t)));
        uint8_t *ty = static_cast<uint8_t *>(scratch((size_t)mx));
        std::vector<uint8_t> types;
        gcmg_status st = GCMG_OK;
        try {
            for (int l = 0; l < (int)c->H.size() && st == GCMG_OK; l++) {
                const HostLevel &L = c->H[l];
                const int64_t ng = L.ng();
                if (ng == 0) continue;
                ck(cudaMemcpyAsync(B, L.B.data(), ng * L.dim * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                   "B");
                ck(cudaMemcpyAsync(gn, L.ghost_node.data(), ng * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream),
                   "ghost nodes");
                launch_mask_types(L.dim, F.n, F.h, F.origin, 1 << l, L.n, B, gn, (int)ng, mask_dev, ty, c->stream);
                types.resize(ng);
                ck(cudaMemcpyAsync(types.data(), ty, ng, cudaMemcpyDeviceToHost, c->stream), "types");
                ck(cudaStreamSynchronize(c->stream), "sync");
                st = gcmg_set_bc_types(c, l, types.data());
            }
        } catch (...) {
            cudaStreamSynchronize(c->stream);
            for (void *q : tmp) cudaFree(q);
            throw;
        }
        for (void *q : tmp) cudaFree(q);
        return st;
    })
}

gcmg_status gcmg_residual(gcmg_ctx *c, const double *u_dev, double *r_dev, double *rel_norm) {
    if (!c || !u_dev || !r_dev) return fail(c, GCMG_E_ARG, "null pointer");
    if (!c->rhs_set) return fail(c, GCMG_E_STATE, "gcmg_set_rhs has not been called");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        const HostLevel &L0 = c->H[0];
        const DevGeom &g0 = c->G[0];
        LevelView<double> v = view<double>(c, 0, c->D64[0]);
        // ||(f, g)|| into slot 1, the defect's norm into slot 0
        ck(cudaMemsetAsync(c->d_norm, 0, 2 * sizeof(unsigned long long), c->stream), "memset");
        const int64_t cnt = std::max<int64_t>(v.chunks ? v.nchunks * CHUNK : L0.nn, L0.ng());
        const unsigned nb = (unsigned)std::min<int64_t>((cnt + 255) / 256, 4096);
        k_rhs_norm<<<nb, 256, 0, c->stream>>>(v, c->D64[0].gg, g0.ng, c->d_norm + 1);
        g_launches++;
        v.u = const_cast<double *>(u_dev);
        v.r = r_dev;
        launch_defect<double>(v, c->p.dim, true, c->d_norm, c->stream);
        check_launch();
        ck(cudaMemcpyAsync(c->h_norm, c->d_norm, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           c->stream), "norms");
        ck(cudaStreamSynchronize(c->stream), "sync");
        double rn, r0;
        std::memcpy(&rn, &c->h_norm[0], sizeof(double));
        std::memcpy(&r0, &c->h_norm[1], sizeof(double));
        if (rel_norm) *rel_norm = r0 > 0.0 ? rn / r0 : 0.0;
        return GCMG_OK;
    })
}

gcmg_status gcmg_set_rhs(gcmg_ctx *c, const double *f_dev, const double *g_dev) {
    if (!c || !f_dev || (!g_dev && c->H[0].ng() > 0)) return fail(c, GCMG_E_ARG, "null pointer");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        const HostLevel &L = c->H[0];
        ck(cudaMemcpyAsync(c->D64[0].f, f_dev, L.nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "f");
        if (L.ng() > 0)
            ck(cudaMemcpyAsync(c->D64[0].gg, g_dev, L.ng() * sizeof(double), cudaMemcpyDeviceToDevice, c->stream),
               "g");
        ck(cudaStreamSynchronize(c->stream), "sync");
        c->rhs_set = true;
        return GCMG_OK;
    })
}

gcmg_status gcmg_set_rhs_level(gcmg_ctx *c, int l, const double *f_dev, const double *g_dev) {
    if (!valid_level(c, l) || !f_dev || (!g_dev && c->H[l].ng() > 0)) return fail(c, GCMG_E_ARG, "bad argument");
    if (c->p.precision != 0) return fail(c, GCMG_E_STATE, "per-level data needs a plain FP64 context");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        const HostLevel &L = c->H[l];
        ck(cudaMemcpyAsync(c->D64[l].f, f_dev, L.nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "f");
        if (L.ng() > 0)
            ck(cudaMemcpyAsync(c->D64[l].gg, g_dev, L.ng() * sizeof(double), cudaMemcpyDeviceToDevice, c->stream),
               "g");
        ck(cudaStreamSynchronize(c->stream), "sync");
        if (l == 0) c->rhs_set = true;
        return GCMG_OK;
    })
}

gcmg_status gcmg_fmg(gcmg_ctx *c, int nu, double *u_dev) {
    if (!c || !u_dev || nu < 0) return fail(c, GCMG_E_ARG, "bad argument");
    if (c->p.precision != 0) return fail(c, GCMG_E_STATE, "full multigrid runs in a plain FP64 context");
    if (!c->rhs_set) return fail(c, GCMG_E_STATE, "gcmg_set_rhs has not been called");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        ensure_inverse(c);
        ensure_junction_solve(c);
        const int last = (int)c->H.size() - 1;
        std::vector<DevData<double>> &D = c->D64;
        launch_coarse_solve<double>(view<double>(c, last, D[last]), c->G[last], D[last].Ainv, c->stream);
        double *uc = D[last].u;   // the grid that holds the current level's solution
        for (int l = last - 1; l >= 0; l--) {
            LevelView<double> F = view<double>(c, l, D[l]), C = view<double>(c, l + 1, D[l + 1]);
            launch_prolong<double>(F, C, c->p.dim, uc, D[l].u, false, c->stream);
            double *u = D[l].u;
            for (int k = 0; k < nu; k++) u = cycle<double>(c, l, u);
            uc = u;
        }
        check_launch();
        ck(cudaMemcpyAsync(u_dev, uc, c->H[0].nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "u out");
        ck(cudaStreamSynchronize(c->stream), "sync");
        return GCMG_OK;
    })
}

gcmg_status gcmg_solve(gcmg_ctx *c, double *u_dev, gcmg_stats *stats) {
    if (!c || !u_dev) return fail(c, GCMG_E_ARG, "null pointer");
    if (!c->rhs_set) return fail(c, GCMG_E_STATE, "gcmg_set_rhs has not been called");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        const HostLevel &L0 = c->H[0];
        const DevGeom &g0 = c->G[0];
        ensure_inverse(c);
        ensure_junction_solve(c);
        if (!c->gexec) coarse_prepare(c);   // the captured graph keeps the chosen path
        double *u = c->D64[0].u;   // internal buffer: the captured graph uses fixed pointers
        if (u_dev != u)
            ck(cudaMemcpyAsync(u, u_dev, L0.nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "u in");
        launch_mask_unknowns<double>(g0.type, u, L0.nn, c->stream);
        gcmg_stats st;
        std::memset(&st, 0, sizeof(st));
        int m = 0;
        double rel = 0.0;
        bool ok = false, diverged = false;
        if (c->use_graph && c->timing_kind < 0) {
            // one graph: ||(f, g)||, the first defect, then the loop; one
            // read-back at the end
            if (!c->gexec) build_graph(c);
            ck(cudaEventRecord(c->ev_in, c->stream), "event");
            ck(cudaStreamWaitEvent(c->gstream, c->ev_in, 0), "wait");
            ck(cudaGraphLaunch(c->gexec, c->gstream), "cudaGraphLaunch");
            ck(cudaEventRecord(c->ev_out, c->gstream), "event");
            ck(cudaStreamWaitEvent(c->stream, c->ev_out, 0), "wait");
            gcmg_ctx::SolveResult *R = c->h_res;
            ck(cudaMemcpyAsync(&R->r0, c->d_r0, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "r0");
            ck(cudaMemcpyAsync(R->rel, c->d_rel, sizeof(R->rel), cudaMemcpyDeviceToHost, c->stream), "rel");
            ck(cudaMemcpyAsync(R->m, c->d_m, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream), "m");
            ck(cudaStreamSynchronize(c->stream), "sync");
            m = R->m[0];
            diverged = c->p.diverge_cycles > 0 && R->m[1] >= c->p.diverge_cycles;
            g_launches += c->graph_pro_kernels + c->graph_kernels * m;
            const int kept = std::min(m, 256);
            std::memcpy(st.rel, R->rel, (kept + 1) * sizeof(double));
            st.r0_norm = R->r0;
            rel = st.rel[kept];
            ok = R->r0 == 0.0 || rel <= c->p.rtol;
        } else {
            // ||r0|| = ||(f, g)||
            ck(cudaMemsetAsync(c->d_norm, 0, sizeof(unsigned long long), c->stream), "memset");
            {
                const LevelView<double> lv = view<double>(c, 0, c->D64[0]);
                const int64_t cnt = std::max<int64_t>(lv.chunks ? lv.nchunks * CHUNK : L0.nn, L0.ng());
                const unsigned nb = (unsigned)std::min<int64_t>((cnt + 255) / 256, 4096);
                k_rhs_norm<<<nb, 256, 0, c->stream>>>(lv, c->D64[0].gg, g0.ng, c->d_norm);
                g_launches++;
            }
            check_launch();
            const double r0 = read_norm(c);
            st.r0_norm = r0;
            if (r0 > 0.0) rel = fine_defect_norm(c) / r0;
            st.rel[0] = rel;
            ok = (r0 == 0.0) || rel <= c->p.rtol;
            int grow = 0;
            while (!ok && m < c->p.max_cycles) {
                loop_body(c);
                check_launch();
                m++;
                const double prev = rel;
                rel = read_norm(c) / r0;
                if (m <= 256) st.rel[m] = rel;
                if (!(rel == rel) || std::isinf(rel)) break;
                ok = rel <= c->p.rtol;
                grow = rel > prev ? grow + 1 : 0;
                if (!ok && c->p.diverge_cycles > 0 && grow >= c->p.diverge_cycles) {
                    diverged = true;
                    break;
                }
            }
        }
        if (u_dev != u)
            ck(cudaMemcpyAsync(u_dev, u, L0.nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "u out");
        ck(cudaStreamSynchronize(c->stream), "sync");
        if (barrier_timed_out(c)) return fail(c, GCMG_E_TIMEOUT, "a grid barrier of the 3D boundary relaxation "
                                                                "gave up waiting");
        st.cycles = m;
        st.converged = ok ? 1 : 0;
        st.diverged = (!ok && diverged) ? 1 : 0;
        st.rel_residual = rel;
        if (stats) *stats = st;
        if (!ok) return fail(c, GCMG_E_NOCONV, st.diverged ? "diverged: the defect grew in consecutive cycles"
                                                         : "not converged");
        return GCMG_OK;
    })
}

// f at the inside nodes of the finest level, read by the device straight from
// a host buffer it can address (page-locked memory): the solver reads f only
// on Omega_h, so the other n^d - |Omega_h| values need not cross the link.
// Nodes visited as in k_rhs_norm (the active chunks in 3D, else every node).
__global__ void k_gather_inside(LevelView<double> lv, const double *__restrict__ src, double *__restrict__ dst) {
    const uint8_t *type = lv.type;
    const int64_t nt = lv.chunks ? lv.nchunks * CHUNK : lv.nn;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = i;
        if (lv.chunks) {
            if ((int)(i % CHUNK) >= (lv.clen[i / CHUNK] & 63)) continue;
            p = (int64_t)lv.chunks[i / CHUNK] + i % CHUNK;
        }
        if ((type[p] & NODE_KIND) == NODE_IN) dst[p] = src[p];
    }
}

// u (all nn values) stored by the device straight into a host buffer it can
// address: 16-byte stores where both buffers allow them
__global__ void k_store_host(const double *__restrict__ src, double *__restrict__ dst, int64_t nn) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
        const double2 *s2 = reinterpret_cast<const double2 *>(src);
        double2 *d2 = reinterpret_cast<double2 *>(dst);
        for (int64_t i = t0; i < nn / 2; i += stride) d2[i] = s2[i];
        if (t0 == 0 && (nn & 1)) dst[nn - 1] = src[nn - 1];
    } else {
        for (int64_t i = t0; i < nn; i += stride) dst[i] = src[i];
    }
}

// the device address of a page-locked host buffer, or null for other memory
const void *mapped_host(const void *p) {
    cudaPointerAttributes pa;
    std::memset(&pa, 0, sizeof(pa));
    const bool ok = cudaPointerGetAttributes(&pa, p) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    cudaGetLastError();   // an unregistered pointer may leave an error behind
    return ok ? pa.devicePointer : nullptr;
}

gcmg_status gcmg_solve_host(gcmg_ctx *c, const double *f_host, const double *g_host, double *u_host,
                            gcmg_stats *stats) {
    if (!c || !f_host || !u_host) return fail(c, GCMG_E_ARG, "null pointer");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        const HostLevel &L = c->H[0];
        // page-locked f: the device reads the inside nodes' values itself;
        // any other host memory: one copy of all n^d values
        const void *f_mapped = mapped_host(f_host);
        if (f_mapped) {
            const LevelView<double> lv = view<double>(c, 0, c->D64[0]);
            const int64_t cnt = lv.chunks ? lv.nchunks * CHUNK : L.nn;
            const unsigned nb = (unsigned)std::min<int64_t>((cnt + 255) / 256, 8192);
            k_gather_inside<<<nb, 256, 0, c->stream>>>(lv, static_cast<const double *>(f_mapped), c->D64[0].f);
            g_launches++;
            check_launch();
        } else {
            ck(cudaMemcpyAsync(c->D64[0].f, f_host, L.nn * sizeof(double), cudaMemcpyHostToDevice, c->stream), "f");
        }
        if (L.ng() > 0)
            ck(cudaMemcpyAsync(c->D64[0].gg, g_host, L.ng() * sizeof(double), cudaMemcpyHostToDevice, c->stream),
               "g");
        c->rhs_set = true;
        double *u = c->D64[0].u;
        ck(cudaMemsetAsync(u, 0, L.nn * sizeof(double), c->stream), "memset");
        gcmg_status s = gcmg_solve(c, u, stats);
        // page-locked u: the device stores it; other host memory: one copy
        void *u_mapped = const_cast<void *>(mapped_host(u_host));
        if (u_mapped) {
            const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((L.nn / 2 + 255) / 256, 152 * 16));
            k_store_host<<<nb, 256, 0, c->stream>>>(u, static_cast<double *>(u_mapped), L.nn);
            g_launches++;
            check_launch();
        } else {
            ck(cudaMemcpyAsync(u_host, u, L.nn * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "u");
        }
        ck(cudaStreamSynchronize(c->stream), "sync");
        return s;
    })
}

// ------------------------------------------------------------ single steps
gcmg_status gcmg_defect(gcmg_ctx *c, int l, const double *u, const double *f, const double *g, double *r,
                        double *norm) {
    if (!valid_level(c, l) || !u || !f || !r) return fail(c, GCMG_E_ARG, "bad argument");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        LevelView<double> v = view<double>(c, l, c->D64[l]);
        v.u = const_cast<double *>(u);
        v.f = f;
        v.gg = g;
        v.r = r;
        ck(cudaMemsetAsync(c->d_norm, 0, sizeof(unsigned long long), c->stream), "memset");
        launch_defect<double>(v, c->p.dim, true, c->d_norm, c->stream);
        check_launch();
        const double nv = read_norm(c);
        if (norm) *norm = nv;
        return GCMG_OK;
    })
}

gcmg_status gcmg_relax(gcmg_ctx *c, int l, double *u, const double *f, const double *g, int with_extra) {
    if (!valid_level(c, l) || !u || !f) return fail(c, GCMG_E_ARG, "bad argument");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        ensure_junction_solve(c);
        if (c->p.junction_solve && !c->js64) {   // FP64 inverses for FP64 relaxations
            c->js64 = true;
            for (int k = 0; k < (int)c->H.size(); k++) {
                if (c->H[k].js_node.empty() || c->D64[k].js_inv) continue;
                destroy_graph(c);   // a captured graph holds the arrays reallocated below
                upload_js(c, k);
            }
        }
        // the sweep writes into a scratch grid (initialised with u), the other
        // steps work there, and the result goes back into u
        const size_t nn = (size_t)c->H[l].nn;
        if (!c->relax_a) {
            size_t mx = 0;
            for (const auto &L : c->H) mx = std::max(mx, (size_t)L.nn);
            c->relax_a = dalloc<double>(c, mx);
            c->relax_b = dalloc<double>(c, mx);
        }
        ck(cudaMemcpyAsync(c->relax_a, u, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "copy");
        LevelView<double> v = view<double>(c, l, c->D64[l]);
        v.u = u;
        v.f = f;
        v.gg = g;
        double *res = relax<double>(c, v, c->relax_a, c->relax_b, l, with_extra != 0);
        if (res != u) ck(cudaMemcpyAsync(u, res, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "copy");
        check_launch();
        ck(cudaStreamSynchronize(c->stream), "sync");
        if (barrier_timed_out(c)) return fail(c, GCMG_E_TIMEOUT, "a grid barrier gave up waiting");
        return GCMG_OK;
    })
}

gcmg_status gcmg_extend(gcmg_ctx *c, int l, double *r) {
    if (!valid_level(c, l) || !r) return fail(c, GCMG_E_ARG, "bad argument");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        launch_extend<double>(r, c->G[l], c->D64[l].ew, c->stream);
        check_launch();
        ck(cudaStreamSynchronize(c->stream), "sync");
        return GCMG_OK;
    })
}

gcmg_status gcmg_restrict(gcmg_ctx *c, int l, const double *r, double *fc, double *gc) {
    if (!valid_level(c, l + 1) || l < 0 || !r || !fc || (!gc && c->H[l + 1].ng() > 0))
        return fail(c, GCMG_E_ARG, "bad argument");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        LevelView<double> v = view<double>(c, l, c->D64[l]);
        v.r = const_cast<double *>(r);
        LevelView<double> vc = view<double>(c, l + 1, c->D64[l + 1]);
        launch_restrict<double>(v, vc, c->p.dim, fc, gc, c->stream);
        check_launch();
        ck(cudaStreamSynchronize(c->stream), "sync");
        return GCMG_OK;
    })
}

gcmg_status gcmg_prolong(gcmg_ctx *c, int l, const double *ec, double *out) {
    if (!valid_level(c, l + 1) || l < 0 || !ec || !out) return fail(c, GCMG_E_ARG, "bad argument");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        LevelView<double> v = view<double>(c, l, c->D64[l]);
        LevelView<double> vc = view<double>(c, l + 1, c->D64[l + 1]);
        launch_prolong<double>(v, vc, c->p.dim, ec, out, false, c->stream);
        check_launch();
        ck(cudaStreamSynchronize(c->stream), "sync");
        return GCMG_OK;
    })
}

gcmg_status gcmg_set_kernel_timing(gcmg_ctx *c, int kind) {
    if (!c || kind < -1 || kind > GCMG_KERNEL_BOUNDARY) return fail(c, GCMG_E_ARG, "bad kernel class");
    if (kind >= 0 && c->bz_units.empty())
        for (const HostLevel &L : c->H) c->bz_units.push_back(boundary_units(L));
    c->timing_kind = kind;
    c->events_used = 0;
    c->timed_bytes = 0.0;
    return GCMG_OK;
}

gcmg_status gcmg_kernel_timing(gcmg_ctx *c, int64_t *launches, double *total_ms) {
    double bytes = 0.0;
    return gcmg_kernel_timing_ex(c, launches, total_ms, &bytes);
}

gcmg_status gcmg_kernel_timing_ex(gcmg_ctx *c, int64_t *launches, double *total_ms, double *alg_bytes) {
    if (!c || !launches || !total_ms || !alg_bytes) return fail(c, GCMG_E_ARG, "null pointer");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        ck(cudaStreamSynchronize(c->stream), "sync");
        double tot = 0.0;
        for (size_t i = 0; i + 1 < c->events_used; i += 2) {
            float ms = 0.f;
            ck(cudaEventElapsedTime(&ms, c->events[i], c->events[i + 1]), "cudaEventElapsedTime");
            tot += ms;
        }
        *launches = (int64_t)(c->events_used / 2);
        *total_ms = tot;
        *alg_bytes = c->timed_bytes;
        c->events_used = 0;
        c->timed_bytes = 0.0;
        return GCMG_OK;
    })
}

int64_t gcmg_launch_counter(void) { return (int64_t)g_launches.load(); }

gcmg_status gcmg_junction_zone(const gcmg_ctx *c, int l, uint8_t *mask) {
    if (!valid_level(c, l) || !mask) return GCMG_E_ARG;
    const std::vector<uint8_t> z = junction_zone_mask(c->H[l], c->p.junction_radius);
    std::memcpy(mask, z.data(), z.size());
    return GCMG_OK;
}

gcmg_status gcmg_junction_solve_set(gcmg_ctx *c, int l, uint8_t *mask) {
    if (!valid_level(c, l) || !mask) return fail(c, GCMG_E_ARG, "bad level or pointer");
    GCMG_GUARD(c, {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        ensure_junction_solve(c);
        const HostLevel &L = c->H[l];
        std::memset(mask, 0, L.nn);
        for (int32_t p : L.js_node) mask[p] = 1;
        return GCMG_OK;
    })
}

}  // extern "C"
