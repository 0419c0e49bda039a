// Host-side geometry of the multigrid hierarchy: node classification, ghost
// equations, extra-sweep band, defect-extension wavefronts and the coarsest
// dense inverse.  Runs once per context; the per-cycle work is all on the GPU.
//
// Compiled without floating-point contraction so that x86 and Arm hosts build
// bit-identical records.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>

#include "gcmg_internal.h"

namespace gcmg {
namespace {

struct Idx {
    const HostLevel &L;
    void split(int64_t p, int j[3]) const {
        for (int a = 0; a < L.dim; a++) {
            j[a] = (int)(p / L.stride[a]);
            p -= (int64_t)j[a] * L.stride[a];
        }
    }
    int64_t join(const int j[3]) const {
        int64_t p = 0;
        for (int a = 0; a < L.dim; a++) p += (int64_t)j[a] * L.stride[a];
        return p;
    }
    bool inside_box(const int j[3]) const {
        for (int a = 0; a < L.dim; a++)
            if (j[a] < 0 || j[a] >= L.n) return false;
        return true;
    }
    bool on_edge(int64_t p) const {
        int j[3];
        split(p, j);
        for (int a = 0; a < L.dim; a++)
            if (j[a] == 0 || j[a] == L.n - 1) return true;
        return false;
    }
};

inline bool unknown(const HostLevel &L, int64_t p) {
    uint8_t k = L.type[p] & NODE_KIND;
    return k == NODE_IN || k == NODE_GHOST;
}

inline void central_grad(const HostLevel &L, int64_t p, double g[3]) {
    for (int a = 0; a < L.dim; a++)
        g[a] = (L.phi[p + L.stride[a]] - L.phi[p - L.stride[a]]) / (2.0 * L.h);
}

// Omega_h = {phi < 0}; ghosts: outside nodes with an inside axis neighbour.
void classify(HostLevel &L) {
    Idx I{L};
    L.type.assign(L.nn, NODE_OUT);
    L.n_in = 0;
    for (int64_t p = 0; p < L.nn; p++)
        if (L.phi[p] < 0.0) {
            if (I.on_edge(p)) throw GeomError{"an inside node lies on the box boundary"};
            L.type[p] = NODE_IN;
            L.n_in++;
        }
    L.ghost_node.clear();
    for (int64_t p = 0; p < L.nn; p++) {
        if (L.type[p] != NODE_OUT) continue;
        int j[3];
        I.split(p, j);
        bool g = false;
        for (int a = 0; a < L.dim && !g; a++)
            for (int s = -1; s <= 1 && !g; s += 2) {
                int k[3] = {j[0], j[1], j[2]};
                k[a] += s;
                if (I.inside_box(k) && L.type[I.join(k)] == NODE_IN) g = true;
            }
        if (g) {
            L.type[p] = NODE_GHOST;
            L.ghost_node.push_back((int32_t)p);
        }
    }
}

// One axis of a ghost stencil: node offsets, value and d/dx weights.
struct AxisRule {
    int m = 0;
    int off[3] = {0, 0, 0};
    double w[3] = {0, 0, 0}, dw[3] = {0, 0, 0};
};

// quadratic Lagrange basis on t in {0,1,2} for nodes at offsets base + k dir
AxisRule quad_rule(double h, int base, int dir, double t) {
    AxisRule r;
    r.m = 3;
    const double l[3] = {0.5 * (t - 1.0) * (t - 2.0), t * (2.0 - t), 0.5 * t * (t - 1.0)};
    const double dl[3] = {t - 1.5, 2.0 - 2.0 * t, t - 0.5};
    for (int k = 0; k < 3; k++) {
        r.off[k] = base + k * dir;
        r.w[k] = l[k];
        r.dw[k] = dl[k] / (dir * h);
    }
    return r;
}

AxisRule lin_rule(double h, int dir, double t) {
    AxisRule r;
    r.m = 2;
    r.off[0] = 0;
    r.off[1] = dir;
    r.w[0] = 1.0 - t;
    r.w[1] = t;
    r.dw[0] = -1.0 / (dir * h);
    r.dw[1] = 1.0 / (dir * h);
    return r;
}

struct Candidate {
    int nk = 0;
    int64_t node[KMAX];
    double val[KMAX];
    double grad[3][KMAX];
};

bool all_unknown(const HostLevel &L, const Candidate &c) {
    for (int k = 0; k < c.nk; k++)
        if (c.node[k] < 0 || !unknown(L, c.node[k])) return false;
    return true;
}

// tensor product of per-axis rules, slots in lexicographic order (axis 0 slowest)
void tensor(const HostLevel &L, const int jg[3], const AxisRule *ax, Candidate &c) {
    Idx I{L};
    const int d = L.dim;
    int cnt[3] = {1, 1, 1};
    for (int a = 0; a < d; a++) cnt[a] = ax[a].m;
    c.nk = 0;
    for (int k0 = 0; k0 < cnt[0]; k0++)
        for (int k1 = 0; k1 < cnt[1]; k1++)
            for (int k2 = 0; k2 < (d == 3 ? cnt[2] : 1); k2++) {
                const int kk[3] = {k0, k1, k2};
                int j[3] = {0, 0, 0};
                for (int a = 0; a < d; a++) j[a] = jg[a] + ax[a].off[kk[a]];
                const int s = c.nk++;
                c.node[s] = I.inside_box(j) ? I.join(j) : -1;
                double v = 1.0;
                for (int a = 0; a < d; a++) v *= ax[a].w[kk[a]];
                c.val[s] = v;
                for (int a = 0; a < d; a++) {
                    double g = ax[a].dw[kk[a]];
                    for (int b = 0; b < d; b++)
                        if (b != a) g *= ax[b].w[kk[b]];
                    c.grad[a][s] = g;
                }
            }
}

// Ghost equation of ghost q (Eqs. clpt, St_G, dir2d, neu2d; Remark 3).
// Readings shared with the paper-level description of the library:
//  * B = G - phi(G) grad_h phi / |grad_h phi|^2;
//  * s_a = sign of the offset -phi(G) g_a; a zero offset tries centred nodes
//    {-1,0,1} (quadratic only), then +1, then -1;
//  * stencils tried in order: quadratic 3^d, linear 2^d, corner (G and
//    G + s_a h e_a), two points along the first axis (direction -1 then +1)
//    whose neighbour of G is inside.
void ghost_equation(HostLevel &L, int64_t q) {
    Idx I{L};
    const int d = L.dim;
    const int64_t G = L.ghost_node[q];
    if (I.on_edge(G)) throw GeomError{"a ghost node lies on the box boundary"};
    int jg[3] = {0, 0, 0};
    I.split(G, jg);
    double g[3] = {0, 0, 0}, gg = 0.0;
    central_grad(L, G, g);
    for (int a = 0; a < d; a++) gg += g[a] * g[a];
    if (!(gg > 0.0)) throw GeomError{"zero level-set gradient at a ghost node"};
    const double ph = L.phi[G];
    double off[3] = {0, 0, 0};
    int sgn[3] = {0, 0, 0};
    std::vector<int> zero_axes;
    for (int a = 0; a < d; a++) {
        off[a] = -ph * g[a] / gg;
        const double sg = -ph * g[a];
        sgn[a] = sg > 0.0 ? 1 : (sg < 0.0 ? -1 : 0);
        L.B[q * d + a] = (L.origin[a] + jg[a] * L.h) + off[a];
        if (sgn[a] == 0) zero_axes.push_back(a);
    }
    const int nz = (int)zero_axes.size();
    Candidate c;
    int kind = -1;
    // quadratic: options per zero axis 0 centred, 1 +1, 2 -1
    int combos = 1;
    for (int z = 0; z < nz; z++) combos *= 3;
    for (int cb = 0; cb < combos && kind < 0; cb++) {
        AxisRule ax[3];
        int digits = cb, zi = nz - 1;
        int opt[3] = {0, 0, 0};
        for (; zi >= 0; zi--) { opt[zi] = digits % 3; digits /= 3; }
        int z = 0;
        for (int a = 0; a < d; a++) {
            if (sgn[a] != 0) {
                ax[a] = quad_rule(L.h, 0, sgn[a], off[a] / (sgn[a] * L.h));
            } else {
                const int o = opt[z++];
                ax[a] = (o == 0) ? quad_rule(L.h, -1, 1, 1.0) : quad_rule(L.h, 0, o == 1 ? 1 : -1, 0.0);
            }
        }
        tensor(L, jg, ax, c);
        if (all_unknown(L, c)) kind = STENCIL_QUAD;
    }
    // linear 2^d and corner: zero axes try +1 then -1
    for (int pass = 0; pass < 2 && kind < 0; pass++) {
        const int nc = 1 << nz;
        for (int cb = 0; cb < nc && kind < 0; cb++) {
            int dir[3] = {0, 0, 0};
            int z = 0;
            for (int a = 0; a < d; a++) {
                dir[a] = sgn[a];
                if (dir[a] == 0) { dir[a] = ((cb >> (nz - 1 - z)) & 1) ? -1 : 1; z++; }
            }
            if (pass == 0) {
                AxisRule ax[3];
                for (int a = 0; a < d; a++) ax[a] = lin_rule(L.h, dir[a], off[a] / (dir[a] * L.h));
                tensor(L, jg, ax, c);
                if (all_unknown(L, c)) kind = STENCIL_LIN;
            } else {
                c.nk = d + 1;
                c.node[0] = G;
                double tsum = 0.0;
                for (int a = 0; a < d; a++)
                    for (int s = 0; s <= d; s++) c.grad[a][s] = 0.0;
                for (int a = 0; a < d; a++) {
                    const double t = off[a] / (dir[a] * L.h);
                    int j[3] = {jg[0], jg[1], jg[2]};
                    j[a] += dir[a];
                    c.node[1 + a] = I.inside_box(j) ? I.join(j) : -1;
                    c.val[1 + a] = t;
                    tsum += t;
                    c.grad[a][1 + a] = 1.0 / (dir[a] * L.h);
                    c.grad[a][0] = -1.0 / (dir[a] * L.h);
                }
                c.val[0] = 1.0 - tsum;
                if (all_unknown(L, c)) kind = STENCIL_CORNER;
            }
        }
    }
    // two points along an axis towards an inside neighbour
    for (int a = 0; a < d && kind < 0; a++)
        for (int s = -1; s <= 1 && kind < 0; s += 2) {
            const int64_t P = G + s * L.stride[a];
            if ((L.type[P] & NODE_KIND) != NODE_IN) continue;
            const double t = off[a] / (s * L.h);
            c.nk = 2;
            c.node[0] = G;
            c.node[1] = P;
            c.val[0] = 1.0 - t;
            c.val[1] = t;
            for (int b = 0; b < d; b++) c.grad[b][0] = c.grad[b][1] = 0.0;
            c.grad[a][0] = -1.0 / (s * L.h);
            c.grad[a][1] = 1.0 / (s * L.h);
            kind = STENCIL_AXIS;
        }
    if (kind < 0) throw GeomError{"no usable ghost stencil"};
    // discrete normal: gradient of the interpolant of phi at B
    double gn[3] = {0, 0, 0}, norm2 = 0.0;
    for (int a = 0; a < d; a++) {
        for (int k = 0; k < c.nk; k++) gn[a] += c.grad[a][k] * L.phi[c.node[k]];
        norm2 += gn[a] * gn[a];
    }
    const double nrm = std::sqrt(norm2);
    if (!(nrm > 0.0)) throw GeomError{"degenerate discrete normal at a ghost node"};
    for (int a = 0; a < d; a++) L.nu[q * d + a] = gn[a] / nrm;
    L.scase[q] = (uint8_t)kind;
    for (int k = 0; k < KMAX; k++) {
        const int64_t o = q * KMAX + k;
        if (k < c.nk) {
            L.stn[o] = (int32_t)c.node[k];
            L.wD[o] = c.val[k];
            double w = 0.0;
            for (int a = 0; a < d; a++) w += L.nu[q * d + a] * c.grad[a][k];
            L.wN[o] = w;
        } else {
            L.stn[o] = (int32_t)G;
            L.wD[o] = 0.0;
            L.wN[o] = 0.0;
        }
    }
}

// Band of Sec. 3.2: inside nodes with -phi/|grad_h phi| <= delta.
void mark_band(HostLevel &L, double delta) {
    Idx I{L};
    L.band_red.clear();
    L.band_black.clear();
    for (int64_t p = 0; p < L.nn; p++) {
        if ((L.type[p] & NODE_KIND) != NODE_IN) continue;
        double g[3] = {0, 0, 0}, gg = 0.0;
        central_grad(L, p, g);
        for (int a = 0; a < L.dim; a++) gg += g[a] * g[a];
        if (!(gg > 0.0)) continue;
        if (L.phi[p] / std::sqrt(gg) >= -delta) {
            L.type[p] |= NODE_BAND;
            int j[3];
            I.split(p, j);
            int par = 0;
            for (int a = 0; a < L.dim; a++) par += j[a];
            ((par & 1) ? L.band_black : L.band_red).push_back((int32_t)p);
        }
    }
}

// Defect extension of Sec. 2.6 on fine level F: steady state of the upwind
// transport, r(P) = sum_a |n_a| r(Q_a) / sum_a |n_a| over Q_a = P - sgn(n_a) h e_a
// with phi(Q_a) < phi(P) (else the mean of the lower ghost / extended axis
// neighbours, else 0); the set is every outside non-ghost node next to a
// coarse ghost, closed under these dependencies.  Nodes are grouped into
// wavefronts: a node's sources all lie in earlier wavefronts (or are ghosts).
void build_extension(HostLevel &F, const HostLevel &C) {
    Idx I{F}, IC{C};
    const int d = F.dim;
    std::vector<uint8_t> in_set(F.nn, 0);
    std::vector<int64_t> work;
    for (int64_t q = 0; q < C.ng(); q++) {
        int J[3] = {0, 0, 0};
        IC.split(C.ghost_node[q], J);
        const int cube = d == 2 ? 9 : 27;
        for (int c = 0; c < cube; c++) {
            int j[3] = {0, 0, 0}, rem = c;
            for (int a = d - 1; a >= 0; a--) { j[a] = 2 * J[a] + rem % 3 - 1; rem /= 3; }
            if (!I.inside_box(j)) continue;
            const int64_t P = I.join(j);
            if (F.type[P] == NODE_OUT && !in_set[P]) { in_set[P] = 1; work.push_back(P); }
        }
    }
    for (size_t w = 0; w < work.size(); w++) {
        const int64_t P = work[w];
        if (I.on_edge(P)) throw GeomError{"the defect extension reaches the box boundary"};
        double g[3] = {0, 0, 0};
        central_grad(F, P, g);
        for (int a = 0; a < d; a++) {
            if (g[a] == 0.0) continue;
            const int64_t Q = P - (g[a] > 0.0 ? 1 : -1) * F.stride[a];
            if (F.phi[Q] < F.phi[P] && F.type[Q] == NODE_OUT && !in_set[Q]) {
                in_set[Q] = 1;
                work.push_back(Q);
            }
        }
    }
    // sources and weights of each node
    struct Ext {
        int64_t node;
        int cnt;
        int64_t src[EMAX];
        double w[EMAX];
        int wave;
    };
    std::vector<Ext> ext(work.size());
    std::vector<int32_t> slot(F.nn > 0 ? 0 : 0);
    std::sort(work.begin(), work.end());
    auto lower_usable = [&](int64_t P, int64_t Q) {
        return F.phi[Q] < F.phi[P] && ((F.type[Q] & NODE_KIND) == NODE_GHOST || in_set[Q]);
    };
    for (size_t e = 0; e < work.size(); e++) {
        const int64_t P = work[e];
        Ext &x = ext[e];
        x.node = P;
        x.cnt = 0;
        double g[3] = {0, 0, 0}, ws = 0.0;
        central_grad(F, P, g);
        for (int a = 0; a < d; a++) {
            if (g[a] == 0.0) continue;
            const int64_t Q = P - (g[a] > 0.0 ? 1 : -1) * F.stride[a];
            if (!lower_usable(P, Q)) continue;
            x.src[x.cnt] = Q;
            x.w[x.cnt] = std::fabs(g[a]);
            ws += std::fabs(g[a]);
            x.cnt++;
        }
        if (x.cnt > 0 && ws > 0.0) {
            for (int i = 0; i < x.cnt; i++) x.w[i] /= ws;
        } else {
            x.cnt = 0;
            for (int a = 0; a < d; a++)
                for (int s = -1; s <= 1; s += 2) {
                    const int64_t Q = P + s * F.stride[a];
                    if (lower_usable(P, Q)) x.src[x.cnt++] = Q;
                }
            for (int i = 0; i < x.cnt; i++) x.w[i] = 1.0 / x.cnt;
        }
    }
    // wavefront = 1 + max wavefront of extended sources (ghosts: 0); process
    // in increasing phi so sources are final before their dependants
    std::vector<size_t> order(work.size());
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const double pa = F.phi[ext[a].node], pb = F.phi[ext[b].node];
        return pa < pb || (pa == pb && ext[a].node < ext[b].node);
    });
    std::vector<int> wave_of(F.nn, 0);
    int nwave = 0;
    for (size_t oi : order) {
        Ext &x = ext[oi];
        int wv = 1;
        for (int i = 0; i < x.cnt; i++)
            if (in_set[x.src[i]]) wv = std::max(wv, wave_of[x.src[i]] + 1);
        x.wave = wv;
        wave_of[x.node] = wv;
        nwave = std::max(nwave, wv);
    }
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return ext[a].wave < ext[b].wave; });
    const size_t ne = work.size();
    F.ext_node.resize(ne);
    F.ext_cnt.resize(ne);
    F.ext_src.assign(ne * EMAX, 0);
    F.ext_w.assign(ne * EMAX, 0.0);
    F.ext_wave.assign(nwave + 1, 0);
    for (size_t i = 0; i < ne; i++) {
        const Ext &x = ext[order[i]];
        F.ext_node[i] = (int32_t)x.node;
        F.ext_cnt[i] = (uint8_t)x.cnt;
        for (int k = 0; k < x.cnt; k++) {
            F.ext_src[i * EMAX + k] = (int32_t)x.src[k];
            F.ext_w[i * EMAX + k] = x.w[k];
        }
        for (int k = x.cnt; k < EMAX; k++) F.ext_src[i * EMAX + k] = (int32_t)x.node;
        F.ext_wave[x.wave]++;
    }
    for (int w = 1; w <= nwave; w++) F.ext_wave[w] += F.ext_wave[w - 1];
    // ext_wave[w] now = number of nodes in waves <= w: offsets of wave w are [ext_wave[w-1], ext_wave[w])
}

}  // namespace

namespace {

// Appends one component to a local program: `upd` (sorted) are the nodes it
// updates, of which `wb` (sorted, a subset) are written back.
struct ProgramBuilder {
    HostLevel &L;
    LocalProgram &P;
    std::vector<int32_t> ghost_of;
    std::vector<int32_t> local;
    std::vector<int64_t> rd;
    explicit ProgramBuilder(HostLevel &lv, LocalProgram &pr) : L(lv), P(pr), ghost_of(lv.nn, -1), local(lv.nn, -1) {
        for (int64_t q = 0; q < L.ng(); q++) ghost_of[L.ghost_node[q]] = (int32_t)q;
    }
    // nodes read by the update of P (inside: axis neighbours; ghost: stencil)
    void reads(int64_t p, std::vector<int64_t> &out) const {
        out.clear();
        if ((L.type[p] & NODE_KIND) == NODE_IN) {
            for (int a = 0; a < L.dim; a++) {
                out.push_back(p - L.stride[a]);
                out.push_back(p + L.stride[a]);
            }
        } else {
            const int64_t q = ghost_of[p];
            const int cube = L.dim == 2 ? 9 : 27;
            for (int k = 0; k < cube; k++) out.push_back(L.stn[q * KMAX + k]);
        }
    }
    int parity(int64_t p) const {
        int par = 0;
        for (int a = 0; a < L.dim; a++) {
            par += (int)(p / L.stride[a]);
            p %= L.stride[a];
        }
        return par & 1;
    }
    // presweep (2D boundary blocks): the component also takes the relaxation's
    // interior red / black update over every inside node it reads (red over
    // those and the red neighbours of their black ones), with the values that
    // update reads staged after the base nodes
    void add(const std::vector<int64_t> &upd, const std::vector<int64_t> &wb, bool presweep = false) {
        std::vector<int64_t> nodes(wb);
        std::vector<uint8_t> in_wb_tmp;
        for (int64_t p : wb) local[p] = 0;
        for (int64_t p : upd)
            if (local[p] < 0) nodes.push_back(p);
        for (int64_t p : upd) local[p] = 0;
        std::vector<int64_t> halo;
        for (int64_t p : upd) {
            reads(p, rd);
            for (int64_t q : rd)
                if (local[q] < 0) halo.push_back(q);
        }
        std::sort(halo.begin(), halo.end());
        halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
        nodes.insert(nodes.end(), halo.begin(), halo.end());
        for (size_t i = 0; i < nodes.size(); i++) local[nodes[i]] = (int32_t)i;
        const size_t base = nodes.size();
        std::vector<int64_t> pre_red, pre_black;
        if (presweep) {
            auto inside = [&](int64_t p) { return (L.type[p] & NODE_KIND) == NODE_IN; };
            for (size_t i = 0; i < base; i++)
                if (inside(nodes[i])) (parity(nodes[i]) ? pre_black : pre_red).push_back(nodes[i]);
            std::vector<int64_t> more;   // red neighbours of the black ones, not staged yet
            for (int64_t p : pre_black) {
                reads(p, rd);
                for (int64_t q : rd)
                    if (inside(q) && local[q] < 0) more.push_back(q);
            }
            std::sort(more.begin(), more.end());
            more.erase(std::unique(more.begin(), more.end()), more.end());
            for (int64_t q : more) {
                local[q] = (int32_t)nodes.size();
                nodes.push_back(q);
                pre_red.push_back(q);
            }
            std::vector<int64_t> ring;   // values the updates read, not staged yet
            for (const std::vector<int64_t> *set : {&pre_red, &pre_black})
                for (int64_t p : *set) {
                    reads(p, rd);
                    for (int64_t q : rd)
                        if (local[q] < 0) ring.push_back(q);
                }
            std::sort(ring.begin(), ring.end());
            ring.erase(std::unique(ring.begin(), ring.end()), ring.end());
            for (int64_t q : ring) {
                local[q] = (int32_t)nodes.size();
                nodes.push_back(q);
            }
            for (const std::vector<int64_t> *set : {&pre_red, &pre_black})
                for (int64_t p : *set) {
                    P.pre_me.push_back(local[p]);
                    P.pre_glob.push_back((int32_t)p);
                    reads(p, rd);
                    for (int64_t q : rd) P.pre_nb.push_back(local[q]);
                }
        }
        P.pre_off.push_back((int32_t)P.pre_me.size());
        P.pre_red_cnt.push_back((int32_t)pre_red.size());
        for (int64_t p : nodes) P.lnode.push_back((int32_t)p);
        P.node_base.push_back((int32_t)base);
        P.node_off.push_back((int32_t)P.lnode.size());
        P.wb_cnt.push_back((int32_t)wb.size());
        int nred = 0, nint = 0, ngh = 0;
        for (int colour = 0; colour < 2; colour++)
            for (int64_t p : upd) {
                if ((L.type[p] & NODE_KIND) != NODE_IN || parity(p) != colour) continue;
                P.int_glob.push_back((int32_t)p);
                P.int_me.push_back(local[p]);
                reads(p, rd);
                for (int64_t q : rd) P.int_nb.push_back(local[q]);
                nint++;
                if (colour == 0) nred++;
            }
        for (int64_t p : upd) {
            if ((L.type[p] & NODE_KIND) != NODE_GHOST) continue;
            P.gh_me.push_back(local[p]);
            P.gh_q.push_back(ghost_of[p]);
            reads(p, rd);
            for (int64_t q : rd) P.gh_stn.push_back(local[q]);
            ngh++;
        }
        P.int_off.push_back((int32_t)P.int_me.size());
        P.red_cnt.push_back(nred);
        P.gh_off.push_back((int32_t)P.gh_me.size());
        P.max_nodes = std::max(P.max_nodes, (int)nodes.size());
        P.max_int = std::max(P.max_int, nint);
        P.max_gh = std::max(P.max_gh, ngh);
        P.max_pre = std::max(P.max_pre, P.pre_off.back() - P.pre_off[P.pre_off.size() - 2]);
        for (int64_t p : nodes) local[p] = -1;
    }
    // union lists of the updated nodes of all components (global fallback)
    void finish(const std::vector<int64_t> &all) {
        for (int64_t p : all) {
            if ((L.type[p] & NODE_KIND) == NODE_GHOST) P.zghost.push_back(ghost_of[p]);
            else (parity(p) ? P.zblack : P.zred).push_back((int32_t)p);
        }
    }
};

}  // namespace

// Junction zone: unknowns within radius h of a ghost whose 3^d neighbourhood
// holds a ghost of the other boundary type.  Split into components closed
// under the reads of their updates (inside node: axis neighbours; ghost: its
// stencil), so each can be relaxed on its own.
// Unknowns within radius h of a junction ghost: a ghost whose 3^d
// neighbourhood holds a ghost of the other boundary type.
static std::vector<uint8_t> junction_marks(const HostLevel &L, double radius, const std::vector<int32_t> &ghost_of) {
    Idx I{L};
    const int d = L.dim;
    std::vector<uint8_t> zone(L.nn, 0);
    const int R = (int)std::ceil(radius);
    const int cube = d == 2 ? 9 : 27;
    for (int64_t q = 0; q < L.ng(); q++) {
        int j[3] = {0, 0, 0};
        I.split(L.ghost_node[q], j);
        bool junction = false;
        for (int c = 0; c < cube && !junction; c++) {
            int k[3] = {0, 0, 0}, rem = c;
            for (int a = d - 1; a >= 0; a--) { k[a] = j[a] + rem % 3 - 1; rem /= 3; }
            if (!I.inside_box(k)) continue;
            const int32_t g2 = ghost_of[I.join(k)];
            if (g2 >= 0 && L.bc[g2] != L.bc[q]) junction = true;
        }
        if (!junction) continue;
        const int side = 2 * R + 1;
        const int total = d == 2 ? side * side : side * side * side;
        for (int c = 0; c < total; c++) {
            int k[3] = {0, 0, 0}, rem = c;
            double r2 = 0.0;
            for (int a = d - 1; a >= 0; a--) {
                const int o = rem % side - R;
                rem /= side;
                k[a] = j[a] + o;
                r2 += (double)o * o;
            }
            if (r2 > radius * radius || !I.inside_box(k)) continue;
            const int64_t P = I.join(k);
            if (unknown(L, P)) zone[P] = 1;
        }
    }
    return zone;
}

std::vector<int32_t> strips_for(const HostLevel &L, int rows) {
    const int sr = (L.n + rows - 1) / rows, sc = (L.n + STRIP_W - 1) / STRIP_W;
    std::vector<uint8_t> active((size_t)sr * sc, 0);
    for (int64_t p = 0; p < L.nn; p++) {
        const uint8_t k = L.type[p] & NODE_KIND;
        if (k == NODE_IN || k == NODE_GHOST) active[(size_t)(p / L.n / rows) * sc + (p % L.n) / STRIP_W] = 1;
    }
    std::vector<int32_t> out;
    for (int a = 0; a < sr; a++)
        for (int b = 0; b < sc; b++)
            if (active[(size_t)a * sc + b]) out.push_back((a << 16) | b);
    return out;
}

std::vector<uint8_t> junction_zone_mask(const HostLevel &L, double radius) {
    std::vector<int32_t> ghost_of(L.nn, -1);
    for (int64_t q = 0; q < L.ng(); q++) ghost_of[L.ghost_node[q]] = (int32_t)q;
    return junction_marks(L, radius, ghost_of);
}

// 3D, mu > 0 and a component of more than kJunctionBlockMin nodes: the zone
// is split instead into blocks of kJunctionBlock^3 nodes, each a component
// that updates every zone node within Chebyshev distance 4 mu of its block
// (the reach of mu sweeps: red 1, black 1, the ghosts' stencils 2) and writes
// back only the block's own zone nodes, so the result equals the global
// sweeps; the blocks overlap, so they write back through a separate grid.
constexpr int kJunctionBlock = 8, kJunctionBlockMin = 1500;

void build_junction(HostLevel &L, double radius, int mu) {
    LocalProgram prog;
    ProgramBuilder PB(L, prog);
    const std::vector<uint8_t> zone = junction_marks(L, radius, PB.ghost_of);
    std::vector<int64_t> zn;
    for (int64_t P = 0; P < L.nn; P++)
        if (zone[P]) zn.push_back(P);
    // union-find over zone nodes joined by reads
    std::vector<int32_t> zid(L.nn, -1);
    for (size_t i = 0; i < zn.size(); i++) zid[zn[i]] = (int32_t)i;
    std::vector<int32_t> parent(zn.size());
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int32_t x) {
        while (parent[x] != x) { parent[x] = parent[parent[x]]; x = parent[x]; }
        return x;
    };
    std::vector<int64_t> rd;
    for (size_t i = 0; i < zn.size(); i++) {
        PB.reads(zn[i], rd);
        for (int64_t Q : rd)
            if (zid[Q] >= 0) {
                const int32_t a = find((int32_t)i), b = find(zid[Q]);
                if (a != b) parent[std::max(a, b)] = std::min(a, b);
            }
    }
    std::vector<int32_t> comp_of_root(zn.size(), -1);
    std::vector<std::vector<int64_t>> comps;
    for (size_t i = 0; i < zn.size(); i++) {
        const int32_t r = find((int32_t)i);
        if (comp_of_root[r] < 0) { comp_of_root[r] = (int32_t)comps.size(); comps.emplace_back(); }
        comps[comp_of_root[r]].push_back(zn[i]);
    }
    size_t largest = 0;
    for (const auto &cz : comps) largest = std::max(largest, cz.size());
    if (L.dim == 3 && mu > 0 && largest > (size_t)kJunctionBlockMin) {
        const int n = L.n, B = kJunctionBlock, H = 4 * mu, nb = (n + B - 1) / B;
        std::vector<int> ci(zn.size()), cj(zn.size()), ck(zn.size());
        std::vector<std::vector<int64_t>> own((size_t)nb * nb * nb);
        std::vector<size_t> tiles;
        for (size_t z = 0; z < zn.size(); z++) {
            ci[z] = (int)(zn[z] / L.stride[0]);
            cj[z] = (int)((zn[z] / L.stride[1]) % n);
            ck[z] = (int)(zn[z] % n);
            const size_t t = ((size_t)(ci[z] / B) * nb + cj[z] / B) * nb + ck[z] / B;
            if (own[t].empty()) tiles.push_back(t);
            own[t].push_back(zn[z]);
        }
        std::sort(tiles.begin(), tiles.end());
        std::vector<int64_t> upd;
        for (size_t t : tiles) {
            const int t0 = (int)(t / ((size_t)nb * nb)) * B, t1 = (int)((t / nb) % nb) * B, t2 = (int)(t % nb) * B;
            upd.clear();
            for (size_t z = 0; z < zn.size(); z++)
                if (ci[z] >= t0 - H && ci[z] < t0 + B + H && cj[z] >= t1 - H && cj[z] < t1 + B + H &&
                    ck[z] >= t2 - H && ck[z] < t2 + B + H)
                    upd.push_back(zn[z]);
            PB.add(upd, own[t]);
        }
        prog.blocked = true;
    } else {
        for (const auto &cz : comps) PB.add(cz, cz);
    }
    PB.finish(zn);
    if (L.dim == 3) prog.zred_src = red_sources(L, prog.zred);
    L.junction = std::move(prog);
}

// Boundary blocks (2D): each block x block tile holding band nodes or ghosts
// becomes a component that updates every band node and ghost within
// Chebyshev distance 2 + 4 lambda of the tile (the reach of one ghost sweep
// plus lambda red / black / ghost sweeps) and writes back only the tile's
// own, so the result equals the global sweeps.
void build_boundary_blocks(HostLevel &L, int lambda, int block) {
    LocalProgram prog;
    ProgramBuilder PB(L, prog);
    const int n = L.n;
    const int H = 2 + 4 * lambda;
    const int nb = (n + block - 1) / block;
    auto updated = [&](int64_t p) {
        const uint8_t t = L.type[p];
        return (t & NODE_KIND) == NODE_GHOST || ((t & NODE_KIND) == NODE_IN && (t & NODE_BAND));
    };
    std::vector<int64_t> all;
    for (int bi = 0; bi < nb; bi++)
        for (int bj = 0; bj < nb; bj++) {
            std::vector<int64_t> wb, upd;
            const int i0 = bi * block, j0 = bj * block;
            for (int i = i0; i < std::min(n, i0 + block); i++)
                for (int j = j0; j < std::min(n, j0 + block); j++) {
                    const int64_t p = (int64_t)i * n + j;
                    if (updated(p)) wb.push_back(p);
                }
            if (wb.empty()) continue;
            for (int i = std::max(0, i0 - H); i < std::min(n, i0 + block + H); i++)
                for (int j = std::max(0, j0 - H); j < std::min(n, j0 + block + H); j++) {
                    const int64_t p = (int64_t)i * n + j;
                    if (updated(p)) upd.push_back(p);
                }
            PB.add(upd, wb, true);
            all.insert(all.end(), wb.begin(), wb.end());
        }
    std::sort(all.begin(), all.end());
    PB.finish(all);
    L.boundary = std::move(prog);
}

bool partial_transfer_weights(const HostLevel &F, int64_t p, bool interior, double *wt) {
    const int d = F.dim;
    const int cube = d == 2 ? 9 : 27, nbox = d == 2 ? 16 : 64;
    // interval codes per axis: 0 [-1,1], 1 [-1,0], 2 [0,1], 3 [0,0]
    static const int LO[4] = {-1, -1, 0, 0}, HI[4] = {1, 0, 1, 0};
    static const double W[4][3] = {{0.25, 0.5, 0.25}, {0.5, 0.5, 0.0}, {0.0, 0.5, 0.5}, {0.0, 1.0, 0.0}};
    bool member[27];
    for (int c = 0; c < cube; c++) {
        int rem = c;
        int64_t P = p;
        for (int a = d - 1; a >= 0; a--) { P += (int64_t)(rem % 3 - 1) * F.stride[a]; rem /= 3; }
        const uint8_t k = F.type[P] & NODE_KIND;
        member[c] = interior ? (k == NODE_IN) : (k != NODE_IN);
        wt[c] = 0.0;
    }
    int best = 0, count = 0;
    for (int pass = 0; pass < 2; pass++)
        for (int b = 0; b < nbox; b++) {
            int iv[3] = {0, 0, 0}, size = 1;
            for (int a = 0; a < d; a++) { iv[a] = (b >> (2 * a)) & 3; size *= HI[iv[a]] - LO[iv[a]] + 1; }
            bool ok = true;
            for (int c = 0; c < cube && ok; c++) {
                int rem = c;
                bool inside = true;
                for (int a = d - 1; a >= 0; a--) {
                    const int o = rem % 3 - 1;
                    rem /= 3;
                    if (o < LO[iv[a]] || o > HI[iv[a]]) inside = false;
                }
                if (inside && !member[c]) ok = false;
            }
            if (!ok) continue;
            if (pass == 0) {
                if (size > best) { best = size; count = 0; }
                if (size == best) count++;
            } else if (size == best) {
                for (int c = 0; c < cube; c++) {
                    int rem = c;
                    double w = 1.0;
                    for (int a = d - 1; a >= 0; a--) { w *= W[iv[a]][rem % 3]; rem /= 3; }
                    wt[c] += w / count;
                }
            }
        }
    return count > 0;
}

// Composes the extension of F (wavefront order: sources first) with the
// partial transfer over D_h - Omega_h at every ghost of C.
static void build_ghost_transfer(HostLevel &F, const HostLevel &C) {
    const int d = F.dim;
    const int cube = d == 2 ? 9 : 27;
    std::vector<int32_t> ghost_of(F.nn, -1), ext_of(F.nn, -1);
    for (int64_t q = 0; q < F.ng(); q++) ghost_of[F.ghost_node[q]] = (int32_t)q;
    for (size_t e = 0; e < F.ext_node.size(); e++) ext_of[F.ext_node[e]] = (int32_t)e;
    // each extension node as a combination of ghost defects
    std::vector<std::vector<std::pair<int32_t, double>>> expand(F.ext_node.size());
    for (size_t e = 0; e < F.ext_node.size(); e++) {
        std::vector<std::pair<int32_t, double>> acc;
        for (int k = 0; k < F.ext_cnt[e]; k++) {
            const int64_t src = F.ext_src[e * EMAX + k];
            const double w = F.ext_w[e * EMAX + k];
            if (ghost_of[src] >= 0) acc.emplace_back(ghost_of[src], w);
            else
                for (const auto &t : expand[ext_of[src]]) acc.emplace_back(t.first, w * t.second);
        }
        std::sort(acc.begin(), acc.end());
        std::vector<std::pair<int32_t, double>> merged;
        for (const auto &t : acc) {
            if (!merged.empty() && merged.back().first == t.first) merged.back().second += t.second;
            else merged.push_back(t);
        }
        expand[e].swap(merged);
    }
    F.gt_ptr.assign(1, 0);
    F.gt_col.clear();
    F.gt_val.clear();
    for (int64_t q = 0; q < C.ng(); q++) {
        int64_t rem = C.ghost_node[q], p = 0;
        for (int a = 0; a < d; a++) {
            const int64_t J = rem / C.stride[a];
            rem -= J * C.stride[a];
            p += 2 * J * F.stride[a];
        }
        double wt[27];
        std::vector<std::pair<int32_t, double>> acc;
        if (partial_transfer_weights(F, p, false, wt)) {
            for (int c = 0; c < cube; c++) {
                if (wt[c] == 0.0) continue;
                int r2 = c;
                int64_t P = p;
                for (int a = d - 1; a >= 0; a--) { P += (int64_t)(r2 % 3 - 1) * F.stride[a]; r2 /= 3; }
                if (ghost_of[P] >= 0) acc.emplace_back(ghost_of[P], wt[c]);
                else if (ext_of[P] >= 0)
                    for (const auto &t : expand[ext_of[P]]) acc.emplace_back(t.first, wt[c] * t.second);
            }
        }
        std::sort(acc.begin(), acc.end());
        for (size_t i = 0; i < acc.size(); i++) {
            if (i > 0 && acc[i].first == acc[i - 1].first) { F.gt_val.back() += acc[i].second; continue; }
            F.gt_col.push_back(acc[i].first);
            F.gt_val.push_back(acc[i].second);
        }
        F.gt_ptr.push_back((int32_t)F.gt_col.size());
    }
}

// Work items of the 3D fused sweep: for each ZM_TY x ZM_TX tile of the
// (axis 1, axis 2) plane, the runs of planes (axis 0) in which the tile holds
// an inside node or a ghost (runs closer than 3 planes merged), cut into
// pieces of at most ZM_SEG planes.  Items never overlap, so every unknown is
// written by exactly one CTA.
static std::vector<int32_t> plane_items(const HostLevel &L, int TY, int TX, int seg) {
    const int n = L.n, ty = (n + TY - 1) / TY, tx = (n + TX - 1) / TX;
    std::vector<uint8_t> act((size_t)ty * tx * n, 0);
    for (int64_t p = 0; p < L.nn; p++) {
        const uint8_t k = L.type[p] & NODE_KIND;
        if (k != NODE_IN && k != NODE_GHOST) continue;
        const int64_t i = p / ((int64_t)n * n), j = (p / n) % n, c = p % n;
        act[((size_t)(j / TY) * tx + c / TX) * n + i] = 1;
    }
    std::vector<int32_t> items;
    for (int t = 0; t < ty * tx; t++) {
        const uint8_t *a = &act[(size_t)t * n];
        int i = 0;
        while (i < n) {
            if (!a[i]) { i++; continue; }
            int end = i + 1;   // [i, end): a run, gaps of up to 2 idle planes merged
            for (int k = end; k < n; k++) {
                if (a[k]) end = k + 1;
                else if (k - end >= 2) break;
            }
            for (int s0 = i; s0 < end; s0 += seg) {
                items.push_back(((t / tx) << 16) | (t % tx));
                items.push_back((s0 << 16) | std::min(end, s0 + seg));
            }
            i = end;
        }
    }
    // launch order: by first plane, then tile (neighbouring tiles run side by
    // side and share their halo reads in L2)
    std::vector<size_t> ord(items.size() / 2);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) {
        const int ax = items[2 * x + 1] >> 16, ay = items[2 * y + 1] >> 16;
        return ax != ay ? ax < ay : items[2 * x] < items[2 * y];
    });
    std::vector<int32_t> sorted;
    sorted.reserve(items.size());
    for (size_t k : ord) {
        sorted.push_back(items[2 * k]);
        sorted.push_back(items[2 * k + 1]);
    }
    return sorted;
}

static void build_zmarch_items(HostLevel &L) {
    const int n = L.n;
    L.zm = plane_items(L, ZM_TY, ZM_TX, ZM_SEG);
    L.sr = plane_items(L, SR_TY, SR_W, SR_SEG);
    // inside-node masks of every item's planes first - 1 .. end (the tile
    // with a 1-node halo; nodes outside the box are not inside)
    L.zm_moff.clear();
    L.zm_mask.clear();
    int64_t planes = 0;
    for (size_t k = 0; k < L.zm.size(); k += 2) {
        L.zm_moff.push_back((int32_t)planes);
        const int a = L.zm[k + 1] >> 16, b = L.zm[k + 1] & 0xffff;
        planes += b - a + 2;
    }
    L.zm_mask.assign((size_t)planes * ZM_MPLANE, 0u);
    for (size_t k = 0; k < L.zm.size(); k += 2) {
        const int r0 = (L.zm[k] >> 16) * ZM_TY, c0 = (L.zm[k] & 0xffff) * ZM_TX;
        const int a = L.zm[k + 1] >> 16, b = L.zm[k + 1] & 0xffff;
        uint32_t *m = &L.zm_mask[(size_t)L.zm_moff[k / 2] * ZM_MPLANE];
        for (int i = a - 1; i <= b; i++, m += ZM_MPLANE) {
            if (i < 0 || i >= n) continue;
            for (int ry = 0; ry < ZM_TY + 2; ry++) {
                const int gj = r0 - 1 + ry;
                if (gj < 0 || gj >= n) continue;
                for (int rx = 0; rx < ZM_TX + 2; rx++) {
                    const int gk = c0 - 1 + rx;
                    if (gk < 0 || gk >= n) continue;
                    if ((L.type[((int64_t)i * n + gj) * n + gk] & NODE_KIND) == NODE_IN)
                        m[ry * ZM_MROW + (rx >> 5)] |= 1u << (rx & 31);
                }
            }
        }
    }
}

std::vector<int32_t> red_sources(const HostLevel &L, const std::vector<int32_t> &list) {
    const size_t m = list.size();
    std::vector<int32_t> src(6 * m);
    const int64_t off[6] = {-1, 1, -L.stride[0], L.stride[0], -L.stride[1], L.stride[1]};
    for (size_t i = 0; i < m; i++)
        for (int k = 0; k < 6; k++) {
            const int64_t q = (int64_t)list[i] + off[k];
            int32_t v = (int32_t)q;
            if ((L.type[q] & NODE_KIND) == NODE_GHOST) {
                const auto it = std::lower_bound(L.ghost_node.begin(), L.ghost_node.end(), (int32_t)q);
                v = -1 - (int32_t)(it - L.ghost_node.begin());
            }
            src[(size_t)k * m + i] = v;
        }
    return src;
}

// Row-span sweep items.  A row block is SP_J consecutive rows (axis 1); per
// plane its span is the union of its rows' unknown spans.  The planes where
// that span is not empty form runs (gaps of up to 2 idle planes merged), cut
// into pieces of at most seg planes; each piece covers the union of its
// planes' spans [kmin, kmax] with windows of 32 C nodes whose owned parts
// (the inner 32 C - 2 nodes) tile it: k0 = kmin - 1 + m (32 C - 2).  Items
// never overlap, so every unknown is written by exactly one CTA.
static void span_items_for(const HostLevel &L, int C, int seg, std::vector<int32_t> &out) {
    const int n = L.n, W = 32 * C - 2, nb = (n + SP_J - 1) / SP_J;
    std::vector<int> lo(n), hi(n);
    out.clear();
    for (int jb = 0; jb < nb; jb++) {
        for (int i = 0; i < n; i++) {
            int l = n, h = -1;
            for (int j = jb * SP_J; j < std::min(n, jb * SP_J + SP_J); j++) {
                const uint32_t sp = (uint32_t)L.sp_rows[2 * ((size_t)i * n + j)];
                const int sl = (int)(sp & 0xffffu), sh = (int)(sp >> 16);
                if (sl <= sh) {
                    l = std::min(l, sl);
                    h = std::max(h, sh);
                }
            }
            lo[i] = l;
            hi[i] = h;
        }
        int i = 0;
        while (i < n) {
            if (lo[i] > hi[i]) { i++; continue; }
            int end = i + 1;
            for (int k = end; k < n; k++) {
                if (lo[k] <= hi[k]) end = k + 1;
                else if (k - end >= 2) break;
            }
            for (int s0 = i; s0 < end; s0 += seg) {
                const int s1 = std::min(end, s0 + seg);
                int kmin = n, kmax = -1;
                for (int p = s0; p < s1; p++)
                    if (lo[p] <= hi[p]) {
                        kmin = std::min(kmin, lo[p]);
                        kmax = std::max(kmax, hi[p]);
                    }
                for (int k0 = kmin - 1; k0 + 1 <= kmax; k0 += W) {
                    out.push_back(jb);
                    out.push_back(k0);
                    out.push_back(s0);
                    out.push_back(s1);
                }
            }
            i = end;
        }
    }
}

// Work of the one-colour row sweep: every run of consecutive inside nodes of
// a row (i, j), cut into segments of at most 64 nodes, in increasing node
// order.
static void build_row_segments(HostLevel &L) {
    const int n = L.n;
    L.sp_list.clear();
    for (int64_t r = 0; r < (int64_t)n * n; r++) {
        const uint8_t *t = &L.type[(size_t)r * n];
        int k = 0;
        while (k < n) {
            if ((t[k] & NODE_KIND) != NODE_IN) { k++; continue; }
            int e = k;
            while (e + 1 < n && (t[e + 1] & NODE_KIND) == NODE_IN) e++;
            for (int k0 = k; k0 <= e; k0 += 64) {
                L.sp_list.push_back((int32_t)r);
                L.sp_list.push_back((int32_t)((uint32_t)k0 | ((uint32_t)std::min(e, k0 + 63) << 16)));
            }
            k = e + 1;
        }
    }
}

bool build_span_items(HostLevel &L, int C, int seg) {
    L.sp.clear();
    L.sp_rows.clear();
    L.sp_cols = 0;
    if (L.dim != 3 || L.n > 0xfffe) return false;
    const int n = L.n;
    seg = seg <= 0 ? SP_SEG : std::min(seg, SP_SEG);   // the CTA stages the metadata of SP_SEG + 4 planes
    const int32_t EMPTY = 0xffff;
    L.sp_rows.assign((size_t)2 * n * n, EMPTY);
    for (int64_t r = 0; r < (int64_t)n * n; r++) {
        const uint8_t *t = &L.type[(size_t)r * n];
        int lo = n, hi = -1, ilo = n, ihi = -1, cnt = 0;
        for (int k = 0; k < n; k++) {
            const int kind = t[k] & NODE_KIND;
            if (kind == NODE_IN || kind == NODE_GHOST) {
                lo = std::min(lo, k);
                hi = k;
            }
            if (kind == NODE_IN) {
                ilo = std::min(ilo, k);
                ihi = k;
                cnt++;
            }
        }
        if (cnt > 0 && cnt != ihi - ilo + 1) {   // inside nodes not one interval
            L.sp_rows.clear();
            return false;
        }
        if (hi >= lo) L.sp_rows[2 * r] = (int32_t)((uint32_t)lo | ((uint32_t)hi << 16));
        if (ihi >= ilo) L.sp_rows[2 * r + 1] = (int32_t)((uint32_t)ilo | ((uint32_t)ihi << 16));
    }
    // C: the fewest lane-node steps, counting a warp's fixed work per plane
    // (metadata, barrier, loop) as 1.25 columns and an item's pipeline fill
    // as 4 planes
    int best = C;
    if (best < SP_CMIN || best > SP_CMAX) {
        double bcost = 0.0;
        std::vector<int32_t> it;
        for (int cc = SP_CMIN; cc <= SP_CMAX; cc++) {
            span_items_for(L, cc, seg, it);
            double cost = 0.0;
            for (size_t q = 0; q < it.size(); q += 4) cost += (double)(it[q + 3] - it[q + 2] + 4) * (1.25 + cc);
            if (best < SP_CMIN || best > SP_CMAX || cost < bcost) {
                best = cc;
                bcost = cost;
            }
        }
    }
    std::vector<int32_t> items;
    span_items_for(L, best, seg, items);
    // launch order: by first plane, then row block, then window (neighbouring
    // blocks run side by side and share their halo rows in L2)
    const size_t m = items.size() / 4;
    std::vector<size_t> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) {
        if (items[4 * x + 2] != items[4 * y + 2]) return items[4 * x + 2] < items[4 * y + 2];
        if (items[4 * x] != items[4 * y]) return items[4 * x] < items[4 * y];
        return items[4 * x + 1] < items[4 * y + 1];
    });
    L.sp.reserve(items.size());
    for (size_t k : ord)
        for (int e = 0; e < 4; e++) L.sp.push_back(items[4 * k + e]);
    L.sp_cols = best;
    return true;
}

// The partial transfer's weights at fine image p over the inside set, in T,
// with the device's operations in its order: the 3^3 members, the largest
// boxes inside them (codes per axis 0 [-1,1], 1 [-1,0], 2 [0,1], 3 [0,0]; box
// b has code (b >> 2 a) & 3 on axis a), then per member the sum over those
// boxes, in increasing b, of the product over the axes of the 1D weights,
// divided by their number.  Zero for non-members and when no box fits.
template <typename T>
static void partial_weights_t(const HostLevel &F, int64_t p, T *w) {
    static const int LO[4] = {-1, -1, 0, 0}, HI[4] = {1, 0, 1, 0};
    auto w1d = [](int iv, int o) -> T {
        switch (iv) {
            case 0: return o == 0 ? (T)0.5 : (T)0.25;
            case 1: return o == 1 ? (T)0 : (T)0.5;
            case 2: return o == -1 ? (T)0 : (T)0.5;
            default: return o == 0 ? (T)1 : (T)0;
        }
    };
    unsigned member = 0;
    int off[27][3];
    for (int c = 0; c < 27; c++) {
        int rem = c;
        int64_t q = p;
        for (int a = 2; a >= 0; a--) {
            off[c][a] = rem % 3 - 1;
            rem /= 3;
            q += off[c][a] * F.stride[a];
        }
        if ((F.type[q] & NODE_KIND) == NODE_IN) member |= 1u << c;
    }
    int best = 0, count = 0;
    uint64_t bestset = 0;
    for (int b = 0; b < 64; b++) {
        unsigned m = 0;
        for (int c = 0; c < 27; c++) {
            bool in = true;
            for (int a = 0; a < 3; a++) {
                const int iv = (b >> (2 * a)) & 3;
                if (off[c][a] < LO[iv] || off[c][a] > HI[iv]) in = false;
            }
            if (in) m |= 1u << c;
        }
        if (m & ~member) continue;
        const int sz = __builtin_popcount(m);
        if (sz > best) { best = sz; count = 1; bestset = (uint64_t)1 << b; }
        else if (sz == best) { count++; bestset |= (uint64_t)1 << b; }
    }
    for (int c = 0; c < 27; c++) {
        w[c] = (T)0;
        if (count == 0 || !((member >> c) & 1u)) continue;
        T wc = 0;
        for (int b = 0; b < 64; b++) {
            if (!((bestset >> b) & 1)) continue;
            T wb = 1;
            for (int a = 0; a < 3; a++) wb *= w1d((b >> (2 * a)) & 3, off[c][a]);
            wc += wb;
        }
        wc /= (T)count;
        w[c] = wc;
    }
}

void build_hierarchy(int dim, int n, int n_coarse, const double *phi, double delta_over_h,
                     std::vector<HostLevel> &levels, double h0, const double *origin) {
    if (!(h0 > 0.0)) h0 = 2.0 / (n - 1);
    levels.clear();
    int nl = 1;
    for (int m = n; m > n_coarse; m = (m - 1) / 2 + 1) nl++;
    for (int l = 0; l < nl; l++) {
        HostLevel L;
        L.dim = dim;
        L.n = (n - 1) / (1 << l) + 1;
        L.h = h0 * (double)(1 << l);
        for (int a = 0; a < 3; a++) L.origin[a] = origin ? origin[a] : -1.0;
        L.nn = 1;
        for (int a = 0; a < dim; a++) L.nn *= L.n;
        L.stride[dim - 1] = 1;
        for (int a = dim - 2; a >= 0; a--) L.stride[a] = L.stride[a + 1] * L.n;
        L.phi.resize(L.nn);
        const int64_t step = (int64_t)1 << l;
        Idx I{L};
        for (int64_t p = 0; p < L.nn; p++) {
            int j[3] = {0, 0, 0};
            I.split(p, j);
            int64_t fi = 0;
            for (int a = 0; a < dim; a++) fi = fi * n + j[a] * step;
            L.phi[p] = phi[fi];
        }
        classify(L);
        const int64_t ng = L.ng();
        L.B.assign(ng * dim, 0.0);
        L.nu.assign(ng * dim, 0.0);
        L.scase.assign(ng, 0);
        L.stn.assign(ng * KMAX, 0);
        L.wD.assign(ng * KMAX, 0.0);
        L.wN.assign(ng * KMAX, 0.0);
        L.bc.assign(ng, 0);
        for (int64_t q = 0; q < ng; q++) ghost_equation(L, q);
        mark_band(L, delta_over_h * L.h);
        if (dim == 3) {
            L.band_red_src = red_sources(L, L.band_red);
            // ghost stencils that are boxes: slot s = (k0 m + k1) m + k2 at
            // node 0 + k0 D0 + k1 D1 + k2 D2, D_a = +-stride_a (checked slot
            // by slot; the 8-slot boxes pad with the ghost itself)
            L.gcode.assign(ng, 0);
            L.gbase.assign(ng, 0);
            for (int64_t q = 0; q < ng; q++) {
                const int32_t *st = &L.stn[q * KMAX];
                for (int m = 3; m >= 2; m--) {
                    const int64_t D2 = (int64_t)st[1] - st[0], D1 = (int64_t)st[m] - st[0],
                                  D0 = (int64_t)st[m * m] - st[0];
                    if (std::llabs(D2) != 1 || std::llabs(D1) != L.stride[1] || std::llabs(D0) != L.stride[0])
                        continue;
                    bool ok = true;
                    for (int sl = 0; sl < KMAX && ok; sl++) {
                        int64_t want = L.ghost_node[q];
                        if (sl < m * m * m) want = st[0] + (sl / (m * m)) * D0 + ((sl / m) % m) * D1 + (sl % m) * D2;
                        if (st[sl] != want) ok = false;
                    }
                    if (!ok) continue;
                    L.gcode[q] = (uint8_t)(m | (D0 < 0 ? 4 : 0) | (D1 < 0 ? 8 : 0) | (D2 < 0 ? 16 : 0));
                    L.gbase[q] = st[0];
                    break;
                }
            }
        }
        if (dim == 2) {
            const int tr = (L.n + TILE_R - 1) / TILE_R, tc = (L.n + TILE_C - 1) / TILE_C;
            std::vector<uint8_t> active((size_t)tr * tc, 0);
            // tiles holding inside nodes or ghosts (the sweep writes the one
            // and carries the other into the other buffer)
            for (int64_t p = 0; p < L.nn; p++)
                if ((L.type[p] & NODE_KIND) == NODE_IN || (L.type[p] & NODE_KIND) == NODE_GHOST)
                    active[(p / L.n) / TILE_R * tc + (p % L.n) / TILE_C] = 1;
            for (int a = 0; a < tr; a++)
                for (int b = 0; b < tc; b++)
                    if (active[(size_t)a * tc + b]) L.tiles.push_back((a << 16) | b);
        } else if (L.nn < ((int64_t)1 << 31)) {
            build_zmarch_items(L);
            build_span_items(L);
            if (L.n <= 0xfffe) build_row_segments(L);
            // active chunks: CHUNK-node runs of a row holding an inside node or a ghost
            for (int64_t row = 0; row < L.nn; row += L.n)
                for (int z0 = 0; z0 < L.n; z0 += CHUNK) {
                    const int len = std::min(CHUNK, L.n - z0);
                    bool act = false;
                    for (int z = z0; z < z0 + len && !act; z++) {
                        const uint8_t k = L.type[row + z] & NODE_KIND;
                        act = k == NODE_IN || k == NODE_GHOST;
                    }
                    if (act) {   // bit 7: parity of the row's (i0 + i1), for the colour of a node
                        const int64_t r = row / L.n, i0 = r / L.n, i1 = r % L.n;
                        L.chunk.push_back((int32_t)(row + z0));
                        L.chunk_len.push_back((uint8_t)(len | (((i0 + i1) & 1) << 7)));
                    }
                }
        }
        levels.push_back(std::move(L));
    }
    for (int l = 0; l + 1 < nl; l++) {
        build_extension(levels[l], levels[l + 1]);
        build_ghost_transfer(levels[l], levels[l + 1]);
        if (dim == 3) {
            HostLevel &F = levels[l];
            const HostLevel &C = levels[l + 1];
            F.partial_coarse.clear();
            for (int64_t i = 0; i < C.nn; i++) {
                if ((C.type[i] & NODE_KIND) != NODE_IN) continue;
                const int64_t ci = i / C.stride[0], cj = (i / C.stride[1]) % C.n, ck = i % C.n;
                const int64_t p = 2 * ci * F.stride[0] + 2 * cj * F.stride[1] + 2 * ck;
                bool full = true;
                for (int a = -1; a <= 1 && full; a++)
                    for (int b = -1; b <= 1 && full; b++)
                        for (int c2 = -1; c2 <= 1 && full; c2++)
                            if ((F.type[p + a * F.stride[0] + b * F.stride[1] + c2] & NODE_KIND) != NODE_IN) full = false;
                if (!full) F.partial_coarse.push_back((int32_t)i);
            }
            const size_t m = F.partial_coarse.size();
            F.partial_wf.assign(27 * m, 0.0f);
            F.partial_wd.assign(27 * m, 0.0);
            for (size_t t = 0; t < m; t++) {
                const int64_t i = F.partial_coarse[t];
                const int64_t ci = i / C.stride[0], cj = (i / C.stride[1]) % C.n, ck = i % C.n;
                const int64_t p = 2 * ci * F.stride[0] + 2 * cj * F.stride[1] + 2 * ck;
                float wf[27];
                double wd[27];
                partial_weights_t<float>(F, p, wf);
                partial_weights_t<double>(F, p, wd);
                for (int c = 0; c < 27; c++) {
                    F.partial_wf[(size_t)c * m + t] = wf[c];
                    F.partial_wd[(size_t)c * m + t] = wd[c];
                }
            }
        }
    }
    number_coarse_unknowns(levels.back());   // the inverse is built before the first solve
}

// Unknowns of the coarsest level (inside nodes and ghosts in node order) with
// their ghost numbers; independent of the boundary types.
void number_coarse_unknowns(HostLevel &L) {
    L.unk_node.clear();
    L.unk_ghost.clear();
    std::vector<int32_t> ghost_of(L.nn, -1);
    for (int64_t q = 0; q < L.ng(); q++) ghost_of[L.ghost_node[q]] = (int32_t)q;
    for (int64_t p = 0; p < L.nn; p++)
        if (unknown(L, p)) {
            L.unk_node.push_back((int32_t)p);
            L.unk_ghost.push_back(ghost_of[p]);
        }
    L.ainv_dirty = true;
}

// Dense inverse of the coarsest system (Eq. discr with the level's bc):
// Gauss-Jordan elimination with partial pivoting on [A | I].
namespace {

// Inverse of an m x m system given row by row as (column, value) pairs, by
// an LU factorisation with partial pivoting confined to the band of the
// matrix, then m triangular solves.  Unknowns numbered in node order couple
// within about one grid row, so this costs O(m bw^2 + m^2 bw) rather than
// the O(m^3) of eliminating the full matrix.  X: row major, m x m.
using Rows = std::vector<std::vector<std::pair<int64_t, double>>>;

void invert_rows(int64_t m, const Rows &rows, std::vector<double> &X, const char *singular) {
    std::vector<double> A((size_t)(m * m), 0.0);
    int64_t bl = 0, bu = 0;
    for (int64_t i = 0; i < m; i++)
        for (const auto &cv : rows[i]) {
            A[i * m + cv.first] += cv.second;
            bl = std::max(bl, i - cv.first);
            bu = std::max(bu, cv.first - i);
        }
    const int64_t ub = bu + bl;   // upper bandwidth once rows have been swapped
    std::vector<int64_t> piv(m);
    for (int64_t c = 0; c < m; c++) {
        const int64_t last = std::min(m - 1, c + bl);
        int64_t p = c;
        for (int64_t i = c + 1; i <= last; i++)
            if (std::fabs(A[i * m + c]) > std::fabs(A[p * m + c])) p = i;
        if (!(std::fabs(A[p * m + c]) > 0.0)) throw GeomError{singular};
        piv[c] = p;
        // the interchange moves the U part only; the multipliers already
        // stored stay where they are and the solves apply the interchanges
        // one elimination step at a time, in the same order
        const int64_t j1 = std::min(m - 1, c + ub);
        if (p != c)
            for (int64_t jj = c; jj <= j1; jj++) std::swap(A[c * m + jj], A[p * m + jj]);
        const double inv = 1.0 / A[c * m + c];
        for (int64_t i = c + 1; i <= last; i++) {
            const double f = A[i * m + c] * inv;
            A[i * m + c] = f;
            if (f == 0.0) continue;
            for (int64_t jj = c + 1; jj <= j1; jj++) A[i * m + jj] -= f * A[c * m + jj];
        }
    }
    X.assign((size_t)(m * m), 0.0);
    std::vector<double> b(m);
    for (int64_t col = 0; col < m; col++) {
        std::fill(b.begin(), b.end(), 0.0);
        b[col] = 1.0;
        for (int64_t c = 0; c < m; c++) {
            if (piv[c] != c) std::swap(b[c], b[piv[c]]);
            const double bc = b[c];
            if (bc == 0.0) continue;
            const int64_t last = std::min(m - 1, c + bl);
            for (int64_t i = c + 1; i <= last; i++) b[i] -= A[i * m + c] * bc;
        }
        for (int64_t c = m - 1; c >= 0; c--) {
            double t = b[c];
            const int64_t j1 = std::min(m - 1, c + ub);
            for (int64_t jj = c + 1; jj <= j1; jj++) t -= A[c * m + jj] * b[jj];
            b[c] = t / A[c * m + c];
        }
        for (int64_t i = 0; i < m; i++) X[i * m + col] = b[i];
    }
}

// The equation of unknown p (inside: -Lap_h; ghost q: its boundary condition
// with the current type) over the columns id[] gives; nodes without a column
// (id < 0) are held fixed and left out.
void equation_row(const HostLevel &L, int64_t p, int32_t q, const std::vector<int64_t> &id,
                  std::vector<std::pair<int64_t, double>> &row) {
    row.clear();
    if (q < 0) {
        const double ih2 = 1.0 / (L.h * L.h);
        row.emplace_back(id[p], 2.0 * L.dim * ih2);
        for (int a = 0; a < L.dim; a++)
            for (int sg = -1; sg <= 1; sg += 2) {
                const int64_t P = p + sg * L.stride[a];
                if (id[P] >= 0) row.emplace_back(id[P], -ih2);
            }
    } else {
        const double *w = (L.bc[q] ? L.wN.data() : L.wD.data()) + (int64_t)q * KMAX;
        for (int k = 0; k < KMAX; k++) {
            const int64_t P = L.stn[(int64_t)q * KMAX + k];
            if (w[k] != 0.0 && id[P] >= 0) row.emplace_back(id[P], w[k]);
        }
    }
}

}  // namespace

void build_coarse_inverse(HostLevel &L) {
    std::vector<int64_t> id(L.nn, -1);
    for (size_t i = 0; i < L.unk_node.size(); i++) id[L.unk_node[i]] = (int64_t)i;
    const int64_t m = (int64_t)L.unk_node.size();
    Rows rows(m);
    for (int64_t i = 0; i < m; i++) equation_row(L, L.unk_node[i], L.unk_ghost[i], id, rows[i]);
    invert_rows(m, rows, L.Ainv, "singular coarsest-level system");
    L.ainv_dirty = false;
}

void build_junction_solve(HostLevel &L, double radius) {
    std::vector<int32_t> ghost_of(L.nn, -1);
    for (int64_t q = 0; q < L.ng(); q++) ghost_of[L.ghost_node[q]] = (int32_t)q;
    std::vector<uint8_t> in = junction_marks(L, radius, ghost_of);
    // grow by the stencils of the zone's ghosts (unused slots name the ghost)
    const std::vector<uint8_t> zone = in;
    for (int64_t q = 0; q < L.ng(); q++)
        if (zone[L.ghost_node[q]])
            for (int k = 0; k < KMAX; k++) in[L.stn[q * KMAX + k]] = 1;
    // strip ghosts whose stencil leaves the set, until none does
    for (bool changed = true; changed;) {
        changed = false;
        for (int64_t q = 0; q < L.ng(); q++) {
            const int64_t G = L.ghost_node[q];
            if (!in[G]) continue;
            for (int k = 0; k < KMAX; k++)
                if (!in[L.stn[q * KMAX + k]]) { in[G] = 0; changed = true; break; }
        }
    }
    // components: unknowns joined by the couplings of their equations
    std::vector<int64_t> nodes;
    for (int64_t P = 0; P < L.nn; P++)
        if (in[P]) nodes.push_back(P);
    std::vector<int64_t> id(L.nn, -1);
    for (size_t i = 0; i < nodes.size(); i++) id[nodes[i]] = (int64_t)i;
    std::vector<int64_t> parent(nodes.size());
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int64_t x) {
        while (parent[x] != x) { parent[x] = parent[parent[x]]; x = parent[x]; }
        return x;
    };
    std::vector<std::pair<int64_t, double>> row;
    for (size_t i = 0; i < nodes.size(); i++) {
        equation_row(L, nodes[i], ghost_of[nodes[i]], id, row);
        for (const auto &cv : row) {
            const int64_t a = find((int64_t)i), b = find(cv.first);
            if (a != b) parent[std::max(a, b)] = std::min(a, b);
        }
    }
    std::vector<int64_t> comp_of_root(nodes.size(), -1);
    std::vector<std::vector<int64_t>> comps;
    for (size_t i = 0; i < nodes.size(); i++) {
        const int64_t r = find((int64_t)i);
        if (comp_of_root[r] < 0) { comp_of_root[r] = (int64_t)comps.size(); comps.emplace_back(); }
        comps[comp_of_root[r]].push_back(nodes[i]);
    }
    L.js_off.assign(1, 0);
    L.js_aoff.assign(1, 0);
    L.js_node.clear();
    L.js_ghost.clear();
    L.js_inv.clear();
    std::vector<int64_t> lid(L.nn, -1);
    std::vector<double> X;
    for (const auto &cz : comps) {
        const int64_t m = (int64_t)cz.size();
        if (m > JS_MAX) throw GeomError{"junction zone component larger than " + std::to_string(JS_MAX)};
        for (int64_t i = 0; i < m; i++) lid[cz[i]] = i;
        Rows rows(m);
        for (int64_t i = 0; i < m; i++) equation_row(L, cz[i], ghost_of[cz[i]], lid, rows[i]);
        invert_rows(m, rows, X, "singular junction-zone system");
        for (int64_t i = 0; i < m; i++) {
            L.js_node.push_back((int32_t)cz[i]);
            L.js_ghost.push_back(ghost_of[cz[i]]);
            lid[cz[i]] = -1;
        }
        L.js_inv.insert(L.js_inv.end(), X.begin(), X.end());
        L.js_off.push_back((int32_t)L.js_node.size());
        L.js_aoff.push_back((int64_t)L.js_inv.size());
    }
}

}  // namespace gcmg
