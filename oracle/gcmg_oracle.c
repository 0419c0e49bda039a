/*
 * gcmg_oracle.c -- plain FP64 CPU oracle for the ghost-cell multigrid of
 * Coco & Russo, "A Finite Difference Ghost-cell Multigrid approach for
 * Poisson Equation with mixed Boundary Conditions in Arbitrary Domain"
 * (arXiv 1111.0983).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA library.  Only the tests, the package smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header or table with
 * the CUDA path and must never be linked into it.
 *
 * Everything here is written for a reader checking it against the paper by
 * eye: full-box loops, no blocking, no fusion, no reordering beyond what the
 * paper states.  Each function names the section / equation it follows.
 * Readings of passages the paper leaves open are marked "Reading:".
 *
 * Grid (Sec. 2.3, "Relaxation operator"): d = 2 or 3, n = N+1 nodes per axis,
 * h = 2/N, node j has coordinate x_a = -1 + j_a h.  Arrays are C ordered with
 * axis 0 (x) slowest, so increasing linear index is the paper's lexicographic
 * order (x slowest, Sec. 2.4 GS-LEX).
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fPIC -shared (no FMA
 * contraction, so x86 and Arm hosts round identically), with -fopenmp where
 * the compiler has it.  OpenMP only splits loops whose iterations are
 * independent (one colour of a red-black sweep, the Jacobi ghost update, the
 * defect, the restriction, the interpolation, the band marks), so the
 * results are bitwise the same for any number of threads; orc_set_threads
 * sets the count (1: serial).
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#define ORC_PARALLEL_FOR _Pragma("omp parallel for schedule(static)")
#else
#define ORC_PARALLEL_FOR
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXD 3
#define MAXK 27

enum { T_EXT = 0, T_INT = 1, T_GHOST = 2 };
enum { BC_D = 0, BC_N = 1 };
enum { ST_QUAD = 0, ST_LIN = 1, ST_CORNER = 2, ST_AXIS = 3 };
enum { ORC_OK = 0, ORC_E_ARG = 1, ORC_E_GEOM = 2, ORC_E_NOCONV = 3, ORC_E_SINGULAR = 4 };

typedef struct {
    int nu1, nu2;          /* pre / post relaxations (TGCS steps 2 and 8) */
    int lambda;            /* extra boundary sweeps after each relaxation (Sec. 3.2) */
    int gamma;             /* 1 = V-cycle, 2 = W-cycle (Remarks 1-2 of Sec. 1) */
    int mode;              /* 0 = red-black interior + Jacobi ghosts, 1 = GS-LEX (Sec. 2.4) */
    int extra_once;        /* 1: the lambda sweeps follow the whole nu-sweep phase only */
    double delta_over_h;   /* band width delta / h (Sec. 3.2 uses 3) */
    double c_dirichlet;    /* mu_D dt (Sec. 2.3 uses 0.9) */
    double c_neumann_factor; /* mu_N dt = factor * 2h / (3 sqrt(d)) (Sec. 2.3 uses 0.9) */
    int junction_sweeps;   /* mu_J: local sweeps near Dirichlet/Neumann junctions (0: none) */
    double junction_radius;/* R_J: junction zone radius, in units of h of each level */
    int junction_solve;    /* 1: solve the zone's equations exactly instead of mu_J sweeps */
    int smoother;          /* 0: the paper's relaxation; 1: its Kaczmarz comparison (Sec. 3.3,
                              "Comparison with the Kaczmarz and the block relaxations") */
} orc_params;

typedef struct {
    int dim, n;
    double h;
    int64_t nn;
    int64_t st[MAXD];      /* strides */
    double *phi;
    uint8_t *type;
    uint8_t *band;
    uint8_t *jzone;        /* unknowns of the junction zone (NULL: none) */
    int64_t jn;            /* exact zone solve: number of zone unknowns, */
    int64_t *jnode;        /* their nodes (increasing index) */
    double *jLU;           /* and the LU factors of their equations (jn x jn) */
    int64_t *jpiv;
    /* ghost records, in increasing node index */
    int64_t ng;
    int64_t *gnode;
    int32_t *gid;          /* node -> ghost number, -1 elsewhere */
    double *B, *nu, *tloc; /* ng*dim */
    int8_t *sdir;          /* ng*dim: s_a in {-1,0,+1} (0: B_a == G_a) */
    uint8_t *gcase;
    int32_t *nk;
    int64_t *stn;          /* ng*MAXK stencil nodes */
    double *wD, *wN;       /* ng*MAXK Dirichlet / Neumann weights */
    uint8_t *bc;           /* ng */
    double *c;             /* ng */
    /* grid functions */
    double *u, *f, *r, *g, *gtmp;
    /* defect extension used before restricting this level's defect */
    int64_t ne;
    int64_t *enode;
    int32_t *ensrc;        /* per extension node: number of sources */
    int64_t *esrc;         /* ne*2*MAXD */
    double *ew;            /* ne*2*MAXD */
    /* coarsest level: dense LU of the assembled system */
    int64_t nunk;
    int64_t *unk;          /* unknown -> node */
    double *LU;
    int64_t *piv;
} Level;

typedef struct {
    int dim, nlev, status;
    orc_params p;
    Level *L;
    char err[256];
} Oracle;

/* ------------------------------------------------------------------ utils */

static void idx_to_j(const Level *L, int64_t idx, int j[MAXD]) {
    for (int a = 0; a < L->dim; a++) {
        j[a] = (int)(idx / L->st[a]);
        idx -= (int64_t)j[a] * L->st[a];
    }
}

static int64_t j_to_idx(const Level *L, const int j[MAXD]) {
    int64_t idx = 0;
    for (int a = 0; a < L->dim; a++) idx += (int64_t)j[a] * L->st[a];
    return idx;
}

static int j_in_box(const Level *L, const int j[MAXD]) {
    for (int a = 0; a < L->dim; a++)
        if (j[a] < 0 || j[a] >= L->n) return 0;
    return 1;
}

static int is_unknown(const Level *L, int64_t idx) {
    return L->type[idx] == T_INT || L->type[idx] == T_GHOST;
}

static int parity(const Level *L, int64_t idx) {
    int j[MAXD], s = 0;
    idx_to_j(L, idx, j);
    for (int a = 0; a < L->dim; a++) s += j[a];
    return s & 1;
}

static double coord(const Level *L, int ja) { return -1.0 + (double)ja * L->h; }

/* central-difference gradient of phi at node idx (interior of the box) */
static void grad_phi(const Level *L, int64_t idx, double g[MAXD]) {
    for (int a = 0; a < L->dim; a++)
        g[a] = (L->phi[idx + L->st[a]] - L->phi[idx - L->st[a]]) / (2.0 * L->h);
}

static int on_box_edge(const Level *L, int64_t idx) {
    int j[MAXD];
    idx_to_j(L, idx, j);
    for (int a = 0; a < L->dim; a++)
        if (j[a] == 0 || j[a] == L->n - 1) return 1;
    return 0;
}

/* ------------------------------------------------- classification (Sec 2.3)
 * Omega_h: nodes with phi < 0 (Omega = {phi < 0}).  Ghost: a node outside
 * Omega with an axis neighbour (distance h) inside Omega.
 */
static int classify(Oracle *O, Level *L) {
    for (int64_t i = 0; i < L->nn; i++) L->type[i] = (L->phi[i] < 0.0) ? T_INT : T_EXT;
    for (int64_t i = 0; i < L->nn; i++) {
        if (L->type[i] != T_INT) continue;
        if (on_box_edge(L, i)) {
            O->status = ORC_E_GEOM;
            strcpy(O->err, "interior node on the box boundary");
            return -1;
        }
    }
    int64_t ng = 0;
    for (int64_t i = 0; i < L->nn; i++) {
        if (L->type[i] != T_EXT) continue;
        int j[MAXD];
        idx_to_j(L, i, j);
        int ghost = 0;
        for (int a = 0; a < L->dim && !ghost; a++)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                int jj[MAXD];
                memcpy(jj, j, sizeof(jj));
                jj[a] += sgn;
                if (j_in_box(L, jj) && L->phi[j_to_idx(L, jj)] < 0.0) ghost = 1;
            }
        if (ghost) { L->type[i] = T_GHOST; ng++; }
    }
    L->ng = ng;
    return 0;
}

/* --------------------------------------------- ghost equations (Sec. 2.3)
 * 1D Lagrange basis on nodes t = 0, 1, 2 and its derivative in t.
 */
static void lagr3(double t, double w[3], double dw[3]) {
    w[0] = (t - 1.0) * (t - 2.0) / 2.0;
    w[1] = t * (2.0 - t);
    w[2] = t * (t - 1.0) / 2.0;
    dw[0] = (2.0 * t - 3.0) / 2.0;
    dw[1] = 2.0 - 2.0 * t;
    dw[2] = (2.0 * t - 1.0) / 2.0;
}

typedef struct {
    int m;
    int off[3];
    double w[3];   /* value weights */
    double dw[3];  /* d/dx weights */
} Axis1D;

typedef struct {
    int nk;
    int64_t node[MAXK];
    double wD[MAXK];
    double gr[MAXD][MAXK]; /* gradient weights per axis */
} Stencil;

static int stencil_ok(const Level *L, const int jg[MAXD], const Stencil *S) {
    (void)jg;
    for (int k = 0; k < S->nk; k++)
        if (S->node[k] < 0 || !is_unknown(L, S->node[k])) return 0;
    return 1;
}

/* tensor product of per-axis 1D rules; node k runs lexicographically with
 * axis 0 slowest.  Nodes leaving the box are marked -1. */
static void tensor_stencil(const Level *L, const int jg[MAXD], const Axis1D ax[MAXD], Stencil *S) {
    int d = L->dim, k = 0;
    int kk[MAXD] = {0, 0, 0};
    int total = 1;
    for (int a = 0; a < d; a++) total *= ax[a].m;
    for (int c = 0; c < total; c++) {
        int rem = c;
        for (int a = d - 1; a >= 0; a--) { kk[a] = rem % ax[a].m; rem /= ax[a].m; }
        int jj[MAXD];
        for (int a = 0; a < d; a++) jj[a] = jg[a] + ax[a].off[kk[a]];
        S->node[k] = j_in_box(L, jj) ? j_to_idx(L, jj) : -1;
        double w = 1.0;
        for (int a = 0; a < d; a++) w *= ax[a].w[kk[a]];
        S->wD[k] = w;
        for (int a = 0; a < d; a++) {
            double gw = ax[a].dw[kk[a]];
            for (int b = 0; b < d; b++)
                if (b != a) gw *= ax[b].w[kk[b]];
            S->gr[a][k] = gw;
        }
        k++;
    }
    S->nk = k;
}

/* quadratic rule along one axis.  s = +-1: upwind nodes 0, s, 2s with the
 * evaluation point at t = delta/(s h) (Eq. St_G).  centred: nodes -1, 0, 1 with
 * the point on the middle node (Reading for sgn(0)). */
static void axis_quad(double h, int s, int centred, double delta, Axis1D *A) {
    double w[3], dw[3];
    A->m = 3;
    if (centred) {
        lagr3(1.0, w, dw);
        for (int k = 0; k < 3; k++) { A->off[k] = k - 1; A->w[k] = w[k]; A->dw[k] = dw[k] / h; }
    } else {
        double t = delta / ((double)s * h);
        lagr3(t, w, dw);
        for (int k = 0; k < 3; k++) {
            A->off[k] = k * s;
            A->w[k] = w[k];
            A->dw[k] = dw[k] / ((double)s * h);
        }
    }
}

static void axis_lin(double h, int s, double delta, Axis1D *A) {
    double t = delta / ((double)s * h);
    A->m = 2;
    A->off[0] = 0; A->off[1] = s;
    A->w[0] = 1.0 - t; A->w[1] = t;
    A->dw[0] = -1.0 / ((double)s * h);
    A->dw[1] = 1.0 / ((double)s * h);
}

/* Builds the ghost equation of ghost number q: closest point B (Eq. clpt),
 * upwind stencil (Eq. St_G), reduced stencils (Remark 3), Dirichlet weights
 * (Eq. dir2d / discrBC) and Neumann weights with the discrete normal
 * grad L[phi] / |grad L[phi]| at B (Eq. neu2d / discrBC).
 *
 * Reading (clpt): B = G - phi(G) grad_h phi / |grad_h phi|^2, i.e. the paper's
 * G - n phi(G) with the extra 1/|grad phi| of a non-distance level set.
 * Reading (sgn 0): s_a = sgn(B_a - G_a) is taken from the exact sign of the
 * offset -phi(G) g_a; a zero offset uses centred nodes, else +1, then -1.
 * Reading (Remark 3): first of quadratic 3^d, linear 2^d, corner (d+1 nodes),
 * two-point axis stencil whose nodes all lie in Omega_h u Gamma_h.
 */
static int build_ghost(Oracle *O, Level *L, int64_t q) {
    int d = L->dim;
    int64_t G = L->gnode[q];
    int jg[MAXD];
    idx_to_j(L, G, jg);
    if (on_box_edge(L, G)) {
        O->status = ORC_E_GEOM;
        strcpy(O->err, "ghost node on the box boundary");
        return -1;
    }
    double gphi[MAXD], gg = 0.0;
    grad_phi(L, G, gphi);
    for (int a = 0; a < d; a++) gg += gphi[a] * gphi[a];
    if (!(gg > 0.0)) {
        O->status = ORC_E_GEOM;
        strcpy(O->err, "zero level-set gradient at a ghost");
        return -1;
    }
    double phiG = L->phi[G];
    double delta[MAXD];
    int s[MAXD];
    for (int a = 0; a < d; a++) {
        delta[a] = -phiG * gphi[a] / gg;
        double sg = -phiG * gphi[a];
        s[a] = (sg > 0.0) ? 1 : ((sg < 0.0) ? -1 : 0);
        L->B[q * d + a] = coord(L, jg[a]) + delta[a];
        L->sdir[q * d + a] = (int8_t)s[a];
    }
    int nz = 0; /* number of axes with a zero offset */
    for (int a = 0; a < d; a++)
        if (s[a] == 0) nz++;

    Stencil S;
    int found = 0, scase = -1;
    int sused[MAXD];
    /* (1) quadratic, zero axes try centred, +1, -1 */
    {
        int ncomb = 1;
        for (int z = 0; z < nz; z++) ncomb *= 3;
        for (int c = 0; c < ncomb && !found; c++) {
            int opt[MAXD] = {0, 0, 0}, rem = c;
            for (int z = nz - 1; z >= 0; z--) { opt[z] = rem % 3; rem /= 3; }
            Axis1D ax[MAXD];
            int zi = 0;
            for (int a = 0; a < d; a++) {
                if (s[a] != 0) { axis_quad(L->h, s[a], 0, delta[a], &ax[a]); sused[a] = s[a]; }
                else {
                    int o = opt[zi++];
                    if (o == 0) { axis_quad(L->h, 1, 1, 0.0, &ax[a]); sused[a] = 0; }
                    else { int ss = (o == 1) ? 1 : -1; axis_quad(L->h, ss, 0, 0.0, &ax[a]); sused[a] = ss; }
                }
            }
            tensor_stencil(L, jg, ax, &S);
            if (stencil_ok(L, jg, &S)) { found = 1; scase = ST_QUAD; }
        }
    }
    /* (2) linear 2^d, zero axes +1 then -1 */
    if (!found) {
        int ncomb = 1 << nz;
        for (int c = 0; c < ncomb && !found; c++) {
            Axis1D ax[MAXD];
            int zi = 0;
            for (int a = 0; a < d; a++) {
                int ss = s[a];
                if (ss == 0) { ss = ((c >> (nz - 1 - zi)) & 1) ? -1 : 1; zi++; }
                axis_lin(L->h, ss, delta[a], &ax[a]);
                sused[a] = ss;
            }
            tensor_stencil(L, jg, ax, &S);
            if (stencil_ok(L, jg, &S)) { found = 1; scase = ST_LIN; }
        }
    }
    /* (3) corner: G and G + s_a h e_a, linear interpolation */
    if (!found) {
        int ncomb = 1 << nz;
        for (int c = 0; c < ncomb && !found; c++) {
            int ss[MAXD], zi = 0;
            for (int a = 0; a < d; a++) {
                ss[a] = s[a];
                if (ss[a] == 0) { ss[a] = ((c >> (nz - 1 - zi)) & 1) ? -1 : 1; zi++; }
            }
            S.nk = d + 1;
            S.node[0] = G;
            double tsum = 0.0;
            for (int a = 0; a < d; a++) {
                double t = delta[a] / ((double)ss[a] * L->h);
                int jj[MAXD];
                memcpy(jj, jg, sizeof(jj));
                jj[a] += ss[a];
                S.node[1 + a] = j_in_box(L, jj) ? j_to_idx(L, jj) : -1;
                S.wD[1 + a] = t;
                tsum += t;
                for (int b = 0; b < d; b++) S.gr[b][1 + a] = 0.0;
                S.gr[a][1 + a] = 1.0 / ((double)ss[a] * L->h);
                S.gr[a][0] = -1.0 / ((double)ss[a] * L->h);
            }
            S.wD[0] = 1.0 - tsum;
            if (stencil_ok(L, jg, &S)) {
                found = 1; scase = ST_CORNER;
                for (int a = 0; a < d; a++) sused[a] = ss[a];
            }
        }
    }
    /* (4) two points along the first axis (a = 0.., direction -1 then +1)
     * whose neighbour of G is inside Omega_h */
    if (!found) {
        for (int a = 0; a < d && !found; a++)
            for (int sg = -1; sg <= 1 && !found; sg += 2) {
                int jj[MAXD];
                memcpy(jj, jg, sizeof(jj));
                jj[a] += sg;
                int64_t P = j_to_idx(L, jj);
                if (L->type[P] != T_INT) continue;
                double t = delta[a] / ((double)sg * L->h);
                S.nk = 2;
                S.node[0] = G; S.node[1] = P;
                S.wD[0] = 1.0 - t; S.wD[1] = t;
                for (int b = 0; b < d; b++) { S.gr[b][0] = 0.0; S.gr[b][1] = 0.0; }
                S.gr[a][0] = -1.0 / ((double)sg * L->h);
                S.gr[a][1] = 1.0 / ((double)sg * L->h);
                for (int b = 0; b < d; b++) sused[b] = 0;
                sused[a] = sg;
                found = 1; scase = ST_AXIS;
            }
    }
    if (!found) {
        O->status = ORC_E_GEOM;
        strcpy(O->err, "no usable ghost stencil");
        return -1;
    }
    /* discrete normal: gradient of the interpolant of phi at B */
    double gn[MAXD], nrm = 0.0;
    for (int a = 0; a < d; a++) {
        gn[a] = 0.0;
        for (int k = 0; k < S.nk; k++) gn[a] += S.gr[a][k] * L->phi[S.node[k]];
        nrm += gn[a] * gn[a];
    }
    nrm = sqrt(nrm);
    if (!(nrm > 0.0)) {
        O->status = ORC_E_GEOM;
        strcpy(O->err, "degenerate discrete normal at a ghost");
        return -1;
    }
    for (int a = 0; a < d; a++) L->nu[q * d + a] = gn[a] / nrm;
    L->nk[q] = S.nk;
    L->gcase[q] = (uint8_t)scase;
    for (int k = 0; k < MAXK; k++) {
        int64_t o = q * MAXK + k;
        if (k < S.nk) {
            L->stn[o] = S.node[k];
            L->wD[o] = S.wD[k];
            double wn = 0.0;
            for (int a = 0; a < d; a++) wn += L->nu[q * d + a] * S.gr[a][k];
            L->wN[o] = wn;
        } else {
            L->stn[o] = G;
            L->wD[o] = 0.0;
            L->wN[o] = 0.0;
        }
    }
    for (int a = 0; a < d; a++) {
        double t;
        if (sused[a] == 0) t = (scase == ST_QUAD) ? 1.0 : 0.0;
        else t = delta[a] / ((double)sused[a] * L->h);
        L->tloc[q * d + a] = t;
        L->sdir[q * d + a] = (int8_t)sused[a];
    }
    return 0;
}

/* ------------------------------------------- band of Sec. 3.2 (extra sweeps)
 * Interior nodes within delta of the boundary.  Reading: the distance of an
 * interior node P is estimated by -phi(P)/|grad_h phi(P)|.
 */
static void build_band(Level *L, double delta) {
    ORC_PARALLEL_FOR
    for (int64_t i = 0; i < L->nn; i++) {
        L->band[i] = 0;
        if (L->type[i] != T_INT) continue;
        double g[MAXD], gg = 0.0;
        grad_phi(L, i, g);
        for (int a = 0; a < L->dim; a++) gg += g[a] * g[a];
        double dist = (gg > 0.0) ? L->phi[i] / sqrt(gg) : -INFINITY;
        if (dist >= -delta) L->band[i] = 1;
    }
}

/* --------------------------------------------- defect extension (Sec. 2.6)
 * The fine defect is extended outside Omega_h constant along the normal, so
 * that coarse ghost points which are not fine ghosts receive a value.
 * Reading: the steady state of the upwind iteration (exp),
 *   r(P) = sum_a |n_a| r(Q_a) / sum_a |n_a|,  Q_a = P - sgn(n_a) h e_a,
 * evaluated in increasing-phi order (the Gauss-Seidel ordering by distance
 * the paper suggests).  A neighbour Q_a is used only when phi(Q_a) < phi(P);
 * with no usable upwind neighbour, the mean of the ghost / earlier extended
 * axis neighbours is used, else 0.  The extension set is every exterior
 * non-ghost fine node of the 3^d neighbourhood of a coarse ghost, closed under
 * those upwind dependencies.
 */
typedef struct { double phi; int64_t idx; } PhiIdx;

static int cmp_phiidx(const void *x, const void *y) {
    const PhiIdx *a = (const PhiIdx *)x, *b = (const PhiIdx *)y;
    if (a->phi < b->phi) return -1;
    if (a->phi > b->phi) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

static int build_extension(Oracle *O, Level *F, const Level *C) {
    int d = F->dim;
    uint8_t *inE = (uint8_t *)calloc((size_t)F->nn, 1);
    int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)F->nn);
    int64_t sp = 0, ne = 0;
    for (int64_t X = 0; X < C->nn; X++) {
        if (C->type[X] != T_GHOST) continue;
        int J[MAXD];
        idx_to_j(C, X, J);
        int total = 1;
        for (int a = 0; a < d; a++) total *= 3;
        for (int c = 0; c < total; c++) {
            int jj[MAXD], rem = c;
            for (int a = d - 1; a >= 0; a--) { jj[a] = 2 * J[a] + (rem % 3) - 1; rem /= 3; }
            if (!j_in_box(F, jj)) continue;
            int64_t P = j_to_idx(F, jj);
            if (F->type[P] == T_EXT && !inE[P]) { inE[P] = 1; stack[sp++] = P; ne++; }
        }
    }
    while (sp > 0) {
        int64_t P = stack[--sp];
        if (on_box_edge(F, P)) {
            O->status = ORC_E_GEOM;
            strcpy(O->err, "defect extension reaches the box boundary");
            free(inE); free(stack);
            return -1;
        }
        double g[MAXD];
        grad_phi(F, P, g);
        for (int a = 0; a < d; a++) {
            if (g[a] == 0.0) continue;
            int64_t Q = P - ((g[a] > 0.0) ? 1 : -1) * F->st[a];
            if (F->phi[Q] < F->phi[P] && F->type[Q] == T_EXT && !inE[Q]) {
                inE[Q] = 1; stack[sp++] = Q; ne++;
            }
        }
    }
    PhiIdx *ord = (PhiIdx *)malloc(sizeof(PhiIdx) * (size_t)(ne > 0 ? ne : 1));
    int64_t k = 0;
    for (int64_t P = 0; P < F->nn; P++)
        if (inE[P]) { ord[k].phi = F->phi[P]; ord[k].idx = P; k++; }
    qsort(ord, (size_t)ne, sizeof(PhiIdx), cmp_phiidx);
    F->ne = ne;
    F->enode = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ne + 1));
    F->ensrc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne + 1));
    F->esrc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ne + 1) * 2 * MAXD);
    F->ew = (double *)malloc(sizeof(double) * (size_t)(ne + 1) * 2 * MAXD);
    for (int64_t e = 0; e < ne; e++) {
        int64_t P = ord[e].idx;
        F->enode[e] = P;
        double g[MAXD], wsum = 0.0;
        int m = 0;
        grad_phi(F, P, g);
        for (int a = 0; a < d; a++) {
            if (g[a] == 0.0) continue;
            int64_t Q = P - ((g[a] > 0.0) ? 1 : -1) * F->st[a];
            if (!(F->phi[Q] < F->phi[P])) continue;
            if (!(F->type[Q] == T_GHOST || inE[Q])) continue;
            F->esrc[e * 2 * MAXD + m] = Q;
            F->ew[e * 2 * MAXD + m] = fabs(g[a]);
            wsum += fabs(g[a]);
            m++;
        }
        if (m > 0 && wsum > 0.0) {
            for (int i = 0; i < m; i++) F->ew[e * 2 * MAXD + i] /= wsum;
        } else {
            m = 0;
            for (int a = 0; a < d; a++)
                for (int sg = -1; sg <= 1; sg += 2) {
                    int64_t Q = P + sg * F->st[a];
                    if (!(F->phi[Q] < F->phi[P])) continue;
                    if (!(F->type[Q] == T_GHOST || inE[Q])) continue;
                    F->esrc[e * 2 * MAXD + m] = Q;
                    m++;
                }
            for (int i = 0; i < m; i++) F->ew[e * 2 * MAXD + i] = 1.0 / (double)m;
        }
        F->ensrc[e] = m;
    }
    free(ord); free(inE); free(stack);
    return 0;
}

static void apply_extension(const Level *F, double *r) {
    for (int64_t e = 0; e < F->ne; e++) {
        double v = 0.0;
        for (int i = 0; i < F->ensrc[e]; i++)
            v += F->ew[e * 2 * MAXD + i] * r[F->esrc[e * 2 * MAXD + i]];
        r[F->enode[e]] = v;
    }
}

/* ------------------------------------------------ relaxation (Sec. 2.3-2.4)
 * Interior: Gauss-Seidel form of Eq. (jac2d), u_P = (h^2 f_P + sum nbrs)/(2d).
 * Ghost: Eqs. (dir2d)/(neu2d), u_G += c (g_G - L_G u).
 */
static double ghost_operator(const Level *L, int64_t q, const double *u) {
    const double *w = (L->bc[q] == BC_D) ? L->wD : L->wN;
    double s = 0.0;
    for (int k = 0; k < L->nk[q]; k++) s += w[q * MAXK + k] * u[L->stn[q * MAXK + k]];
    return s;
}

static void interior_update(Level *L, int64_t i) {
    double s = L->h * L->h * L->f[i];
    for (int a = 0; a < L->dim; a++) s += L->u[i + L->st[a]] + L->u[i - L->st[a]];
    L->u[i] = s / (2.0 * L->dim);
}

/* red (even sum of indices) then black half sweep; band_only restricts to band */
static void rb_sweep(Level *L, int band_only) {
    for (int color = 0; color < 2; color++) {
        ORC_PARALLEL_FOR
        for (int64_t i = 0; i < L->nn; i++) {
            if (L->type[i] != T_INT) continue;
            if (band_only && !L->band[i]) continue;
            if (parity(L, i) != color) continue;
            interior_update(L, i);
        }
    }
}

/* simultaneous (Jacobi) update of all ghosts from the current values */
static void ghost_jacobi(Level *L) {
    ORC_PARALLEL_FOR
    for (int64_t q = 0; q < L->ng; q++)
        L->gtmp[q] = L->u[L->gnode[q]] + L->c[q] * (L->g[q] - ghost_operator(L, q, L->u));
    ORC_PARALLEL_FOR
    for (int64_t q = 0; q < L->ng; q++) L->u[L->gnode[q]] = L->gtmp[q];
}

/* GS-LEX over Omega_h u Gamma_h (band_only: band u Gamma_h), in place */
static void lex_sweep(Level *L, int band_only) {
    for (int64_t i = 0; i < L->nn; i++) {
        if (L->type[i] == T_INT) {
            if (band_only && !L->band[i]) continue;
            interior_update(L, i);
        } else if (L->type[i] == T_GHOST) {
            int64_t q = L->gid[i];
            L->u[i] += L->c[q] * (L->g[q] - ghost_operator(L, q, L->u));
        }
    }
}

static void base_relax(Oracle *O, Level *L) {
    if (O->p.mode == 1) lex_sweep(L, 0);
    else { rb_sweep(L, 0); ghost_jacobi(L); }
}

/* Junction relaxation (an addition to the paper's smoother; none gives the
 * paper's method).  Where Dirichlet and Neumann ghosts meet, the error of the
 * mixed problem is singular and the boundary extra sweeps of Sec. 3.2 do not
 * reach it, so the cycle's factor grows as h shrinks.  Following the same
 * rationale (relax more where the error decays slowly), the unknowns within
 * R_J h of a ghost whose 3^d neighbourhood holds a ghost of the other type
 * are relaxed again after every relaxation on every level, either by mu_J
 * sweeps (red, black, then Jacobi on the ghosts; zone_sweep) or by solving
 * their equations exactly (zone_solve, below). */
static void zone_sweep(Level *L) {
    for (int color = 0; color < 2; color++) {
        ORC_PARALLEL_FOR
        for (int64_t i = 0; i < L->nn; i++)
            if (L->type[i] == T_INT && L->jzone[i] && parity(L, i) == color) interior_update(L, i);
    }
    ORC_PARALLEL_FOR
    for (int64_t q = 0; q < L->ng; q++)
        if (L->jzone[L->gnode[q]]) L->gtmp[q] = L->u[L->gnode[q]] + L->c[q] * (L->g[q] - ghost_operator(L, q, L->u));
    ORC_PARALLEL_FOR
    for (int64_t q = 0; q < L->ng; q++)
        if (L->jzone[L->gnode[q]]) L->u[L->gnode[q]] = L->gtmp[q];
}

/* marks unknowns within radius (in h) of a junction ghost: a ghost whose
 * 3^d neighbourhood holds a ghost of the other bc type */
static void build_jzone(Level *L, double radius) {
    int d = L->dim;
    if (!L->jzone) L->jzone = (uint8_t *)calloc((size_t)L->nn, 1);
    memset(L->jzone, 0, (size_t)L->nn);
    int R = (int)ceil(radius);
    for (int64_t q = 0; q < L->ng; q++) {
        int64_t G = L->gnode[q];
        int j[MAXD]; idx_to_j(L, G, j);
        int junction = 0;
        int total = 1; for (int a = 0; a < d; a++) total *= 3;
        for (int c = 0; c < total; c++) {
            int jj[MAXD], rem = c;
            for (int a = d - 1; a >= 0; a--) { jj[a] = j[a] + rem % 3 - 1; rem /= 3; }
            if (!j_in_box(L, jj)) continue;
            int64_t P = j_to_idx(L, jj);
            if (L->type[P] == T_GHOST && L->bc[L->gid[P]] != L->bc[q]) junction = 1;
        }
        if (!junction) continue;
        int side = 2 * R + 1, tot = 1; for (int a = 0; a < d; a++) tot *= side;
        for (int c = 0; c < tot; c++) {
            int jj[MAXD], rem = c; double r2 = 0;
            for (int a = d - 1; a >= 0; a--) { int o = rem % side - R; rem /= side; jj[a] = j[a] + o; r2 += (double)o * o; }
            if (r2 > radius * radius || !j_in_box(L, jj)) continue;
            int64_t P = j_to_idx(L, jj);
            if (is_unknown(L, P)) L->jzone[P] = 1;
        }
    }
}

/* Exact junction-zone solve (the alternative to the mu_J sweeps): the
 * equations of the zone's unknowns, with every value outside the zone held
 * fixed, are solved exactly, i.e. u_Z += A_ZZ^{-1} r_Z with r the defect.
 * A block (Schwarz) step of the same system; unlike the sweeps it cannot
 * grow a local mode, e.g. next to a Dirichlet ghost whose own weight in its
 * condition is almost zero. */
static int lu_factor(double *A, int64_t n, int64_t *piv);
static void lu_solve(const double *A, int64_t n, const int64_t *piv, double *b);

static double row_defect(const Level *L, int64_t i, const double *u) {
    if (L->type[i] == T_INT) {
        double lap = -2.0 * L->dim * u[i];
        for (int a = 0; a < L->dim; a++) lap += u[i + L->st[a]] + u[i - L->st[a]];
        return L->f[i] + lap / (L->h * L->h);
    }
    int64_t q = L->gid[i];
    return L->g[q] - ghost_operator(L, q, u);
}

static int build_jsolve(Level *L) {
    free(L->jnode); free(L->jLU); free(L->jpiv);
    L->jnode = NULL; L->jLU = NULL; L->jpiv = NULL; L->jn = 0;
    /* the solved set: the zone grown by the stencils of its ghosts, then
     * stripped (repeatedly) of every ghost whose stencil leaves it, so that
     * each ghost row is complete: a row cut off from the node that carries
     * most of its weight would leave A_ZZ nearly singular */
    uint8_t *in = (uint8_t *)malloc((size_t)L->nn);
    memcpy(in, L->jzone, (size_t)L->nn);
    for (int64_t q = 0; q < L->ng; q++)
            if (L->jzone[L->gnode[q]])
                for (int m = 0; m < L->nk[q]; m++) in[L->stn[q * MAXK + m]] = 1;
    for (int changed = 1; changed;) {
        changed = 0;
        for (int64_t q = 0; q < L->ng; q++) {
            int64_t G = L->gnode[q];
            if (!in[G]) continue;
            for (int m = 0; m < L->nk[q]; m++)
                if (!in[L->stn[q * MAXK + m]]) { in[G] = 0; changed = 1; break; }
        }
    }
    int64_t n = 0;
    for (int64_t i = 0; i < L->nn; i++) n += in[i] ? 1 : 0;
    if (n == 0) { free(in); return 0; }
    int64_t *loc = (int64_t *)malloc(sizeof(int64_t) * (size_t)L->nn);
    L->jnode = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    L->jLU = (double *)calloc((size_t)(n * n), sizeof(double));
    L->jpiv = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t k = 0;
    for (int64_t i = 0; i < L->nn; i++) {
        loc[i] = in[i] ? k : -1;
        if (in[i]) L->jnode[k++] = i;
    }
    free(in);
    L->jn = n;
    double ih2 = 1.0 / (L->h * L->h);
    for (int64_t r = 0; r < n; r++) {
        int64_t i = L->jnode[r];
        double *row = L->jLU + r * n;
        if (L->type[i] == T_INT) {   /* -Delta_h */
            row[r] += 2.0 * L->dim * ih2;
            for (int a = 0; a < L->dim; a++)
                for (int sg = -1; sg <= 1; sg += 2) {
                    int64_t P = i + sg * L->st[a];
                    if (loc[P] >= 0) row[loc[P]] -= ih2;
                }
        } else {                     /* L_h of the ghost's condition */
            int64_t q = L->gid[i];
            const double *w = (L->bc[q] == BC_D) ? L->wD : L->wN;
            for (int m = 0; m < L->nk[q]; m++) {
                int64_t P = L->stn[q * MAXK + m];
                if (loc[P] >= 0) row[loc[P]] += w[q * MAXK + m];
            }
        }
    }
    free(loc);
    return lu_factor(L->jLU, n, L->jpiv);
}

static void zone_solve(Level *L) {
    double *b = (double *)malloc(sizeof(double) * (size_t)L->jn);
    for (int64_t k = 0; k < L->jn; k++) b[k] = row_defect(L, L->jnode[k], L->u);
    lu_solve(L->jLU, L->jn, L->jpiv, b);
    for (int64_t k = 0; k < L->jn; k++) L->u[L->jnode[k]] += b[k];
    free(b);
}

static void junction_relax(Oracle *O, Level *L) {
    if (!L->jzone) return;
    if (O->p.junction_solve) {
        if (L->jn) zone_solve(L);
    } else {
        for (int m = 0; m < O->p.junction_sweeps; m++) zone_sweep(L);
    }
}

/* lambda extra sweeps on Gamma_h and the band (Sec. 3.2) */
static void extra_sweeps(Oracle *O, Level *L) {
    for (int k = 0; k < O->p.lambda; k++) {
        if (O->p.mode == 1) lex_sweep(L, 1);
        else { rb_sweep(L, 1); ghost_jacobi(L); }
    }
}

/* ----------------------------------------- Kaczmarz comparison smoother
 * Sec. 3.3, "Comparison with the Kaczmarz and the block relaxations": a
 * Gauss-Seidel sweep over the inside nodes, then lambda Kaczmarz sweeps over
 * the set J of the ghost equations and the inside equations within delta of
 * the boundary (the band).  A Kaczmarz step on row j of L u = b moves u along
 * the row: u += (b_j - <l_j, u>) / ||l_j||^2 l_j.
 * Rows: an inside node i, scaled by h^2 (the step does not depend on a row's
 * scale): 2d u_i - sum of its 2d neighbours = h^2 f_i; a ghost q: its
 * boundary equation, sum_k w_k u_k = g_q.
 * Reading: the paper leaves the order of J open ("for j in J").  The order
 * taken: colour c(i) = sum_a (j_a mod 5) 5^a of the row's node, colours in
 * increasing c, nodes in increasing index within a colour.  A row's support
 * lies within 2 nodes of its node on every axis, so two rows of one colour
 * (5 or more apart on some axis) share no unknown: within a colour the order
 * does not change the result, and the colours can be swept in parallel. */
static int kaczmarz_colour(const Level *L, int64_t i) {
    int j[MAXD];
    idx_to_j(L, i, j);
    int c = 0, m = 1;
    for (int a = 0; a < L->dim; a++) { c += (j[a] % 5) * m; m *= 5; }
    return c;
}

/* one Kaczmarz step on the row of node i (an inside band node or a ghost);
 * sums in the order written, each product rounded on its own */
static void kaczmarz_row(Level *L, int64_t i) {
    double *u = L->u;
    if (L->type[i] == T_INT) {
        const int d = L->dim;
        double s = 0.0;
        for (int a = 0; a < d; a++) s += u[i + L->st[a]] + u[i - L->st[a]];
        const double r = (L->h * L->h * L->f[i] + s) - 2.0 * d * u[i];
        const double t = r / (double)(4 * d * d + 2 * d);
        u[i] += 2.0 * d * t;
        for (int a = 0; a < d; a++) { u[i + L->st[a]] -= t; u[i - L->st[a]] -= t; }
    } else if (L->type[i] == T_GHOST) {
        const int64_t q = L->gid[i];
        const double *w = (L->bc[q] == BC_D) ? L->wD : L->wN;
        double s = 0.0, n2 = 0.0;
        for (int k = 0; k < L->nk[q]; k++) {
            s += w[q * MAXK + k] * u[L->stn[q * MAXK + k]];
            n2 += w[q * MAXK + k] * w[q * MAXK + k];
        }
        const double t = (L->g[q] - s) / n2;
        for (int k = 0; k < L->nk[q]; k++) u[L->stn[q * MAXK + k]] += t * w[q * MAXK + k];
    }
}

static int in_kaczmarz_set(const Level *L, int64_t i) {
    return (L->type[i] == T_INT && L->band[i]) || L->type[i] == T_GHOST;
}

static void kaczmarz_sweep(Level *L) {
    const int ncol = L->dim == 2 ? 25 : 125;
    for (int c = 0; c < ncol; c++)
        for (int64_t i = 0; i < L->nn; i++)
            if (in_kaczmarz_set(L, i) && kaczmarz_colour(L, i) == c) kaczmarz_row(L, i);
}

static void kaczmarz_relax(Oracle *O, Level *L, int with_extra) {
    rb_sweep(L, 0);
    const int sweeps = with_extra ? O->p.lambda : 1;
    for (int m = 0; m < sweeps; m++) kaczmarz_sweep(L);
}

static void smooth(Oracle *O, Level *L, int nu) {
    if (O->p.smoother == 1) {
        for (int k = 0; k < nu; k++) kaczmarz_relax(O, L, 1);
        return;
    }
    for (int k = 0; k < nu; k++) {
        base_relax(O, L);
        if (!O->p.extra_once) extra_sweeps(O, L);
        if (O->p.junction_sweeps || O->p.junction_solve) junction_relax(O, L);
    }
    if (O->p.extra_once && nu > 0) extra_sweeps(O, L);
}

/* ------------------------------------------------ defect (TGCS step 3)
 * r = f + Delta_h u on Omega_h, r = g - L_h u on Gamma_h, 0 elsewhere.
 */
static void defect(const Level *L, const double *u, double *r) {
    ORC_PARALLEL_FOR
    for (int64_t i = 0; i < L->nn; i++) {
        if (L->type[i] == T_INT) {
            double lap = -2.0 * L->dim * u[i];
            for (int a = 0; a < L->dim; a++) lap += u[i + L->st[a]] + u[i - L->st[a]];
            r[i] = L->f[i] + lap / (L->h * L->h);
        } else if (L->type[i] == T_GHOST) {
            int64_t q = L->gid[i];
            r[i] = L->g[q] - ghost_operator(L, q, u);
        } else {
            r[i] = 0.0;
        }
    }
}

static double max_abs_unknowns(const Level *L, const double *r) {
    double m = 0.0;
    for (int64_t i = 0; i < L->nn; i++)
        if (is_unknown(L, i)) {
            double v = fabs(r[i]);
            if (v != v) return v;
            if (v > m) m = v;
        }
    return m;
}

/* ---------------------------------------------- restriction (Sec. 2.5)
 * Partial grid transfer at coarse node X over the fine set I: among boxes
 * T = prod_a [alpha_a, beta_a], alpha in {-1,0}, beta in {0,1}, whose fine
 * nodes all lie in I, the largest ones are used, with the tensor-product
 * weights of the 1D rules (restI)/(restL)/(restR) (injection for 1-wide
 * axes).  Reading: equally large boxes are averaged.
 * Composite operator: I = Omega_h at coarse interior nodes, I = D_h - Omega_h
 * at coarse ghosts.
 */
static double w1d(int alpha, int beta, int o) {
    /* weights of offset o in {-1,0,1} for interval [alpha, beta] */
    if (alpha == -1 && beta == 1) return (o == 0) ? 0.5 : 0.25;
    if (alpha == -1 && beta == 0) return (o == 1) ? 0.0 : 0.5;
    if (alpha == 0 && beta == 1) return (o == -1) ? 0.0 : 0.5;
    return (o == 0) ? 1.0 : 0.0; /* [0,0] */
}

static int in_set(const Level *F, int64_t P, int interior_set) {
    return interior_set ? (F->type[P] == T_INT) : (F->type[P] != T_INT);
}

/* fills wt[3^d] (offsets lexicographic, axis 0 slowest); returns 0 if no box */
static int partial_weights(const Level *F, const int jf[MAXD], int interior_set, double wt[MAXK]) {
    int d = F->dim;
    int nb = 1, nnb = 1;
    for (int a = 0; a < d; a++) { nb *= 4; nnb *= 3; }
    int member[MAXK];
    for (int c = 0; c < nnb; c++) {
        int jj[MAXD], rem = c;
        for (int a = d - 1; a >= 0; a--) { jj[a] = jf[a] + (rem % 3) - 1; rem /= 3; }
        member[c] = j_in_box(F, jj) && in_set(F, j_to_idx(F, jj), interior_set);
    }
    static const int AL[4] = {-1, -1, 0, 0}, BE[4] = {1, 0, 1, 0};
    int best = 0, count = 0;
    for (int c = 0; c < nnb; c++) wt[c] = 0.0;
    for (int b = 0; b < nb; b++) {
        int iv[MAXD], rem = b, size = 1;
        for (int a = d - 1; a >= 0; a--) { iv[a] = rem % 4; rem /= 4; }
        for (int a = 0; a < d; a++) size *= BE[iv[a]] - AL[iv[a]] + 1;
        int ok = 1;
        for (int c = 0; c < nnb && ok; c++) {
            int r2 = c, inside = 1;
            for (int a = d - 1; a >= 0; a--) {
                int o = (r2 % 3) - 1; r2 /= 3;
                if (o < AL[iv[a]] || o > BE[iv[a]]) inside = 0;
            }
            if (inside && !member[c]) ok = 0;
        }
        if (!ok) continue;
        if (size > best) {
            best = size; count = 0;
            for (int c = 0; c < nnb; c++) wt[c] = 0.0;
        }
        if (size == best) {
            count++;
            for (int c = 0; c < nnb; c++) {
                int r2 = c;
                double w = 1.0;
                for (int a = d - 1; a >= 0; a--) {
                    int o = (r2 % 3) - 1; r2 /= 3;
                    w *= w1d(AL[iv[a]], BE[iv[a]], o);
                }
                wt[c] += w;
            }
        }
    }
    if (count == 0) return 0;
    for (int c = 0; c < nnb; c++) wt[c] /= (double)count;
    return 1;
}

static double partial_transfer(const Level *F, const int jf[MAXD], int interior_set, const double *r) {
    double wt[MAXK];
    if (!partial_weights(F, jf, interior_set, wt)) return 0.0;
    int d = F->dim, nnb = 1;
    for (int a = 0; a < d; a++) nnb *= 3;
    double v = 0.0;
    for (int c = 0; c < nnb; c++) {
        if (wt[c] == 0.0) continue;
        int jj[MAXD], rem = c;
        for (int a = d - 1; a >= 0; a--) { jj[a] = jf[a] + (rem % 3) - 1; rem /= 3; }
        v += wt[c] * r[j_to_idx(F, jj)];
    }
    return v;
}

static void restrict_defect(const Level *F, Level *C, const double *r, double *fc, double *gc) {
    ORC_PARALLEL_FOR
    for (int64_t X = 0; X < C->nn; X++) {
        int J[MAXD], jf[MAXD];
        idx_to_j(C, X, J);
        for (int a = 0; a < C->dim; a++) jf[a] = 2 * J[a];
        if (C->type[X] == T_INT) fc[X] = partial_transfer(F, jf, 1, r);
        else {
            fc[X] = 0.0;
            if (C->type[X] == T_GHOST) gc[C->gid[X]] = partial_transfer(F, jf, 0, r);
        }
    }
}

/* -------------------------------------------- interpolation (Sec. 2.6)
 * Bilinear / trilinear interpolation onto Omega_h u Gamma_h.  Reading: coarse
 * parents outside Omega_2h u Gamma_2h are dropped and the remaining weights
 * renormalised (no parent: zero correction).
 */
static double prolong_at(const Level *F, const Level *C, int64_t P, const double *e) {
    int d = F->dim, j[MAXD];
    idx_to_j(F, P, j);
    int lo[MAXD], m[MAXD], total = 1;
    for (int a = 0; a < d; a++) {
        lo[a] = j[a] / 2;
        m[a] = (j[a] % 2) ? 2 : 1;
        total *= m[a];
    }
    double num = 0.0, den = 0.0;
    for (int c = 0; c < total; c++) {
        int J[MAXD], rem = c;
        double w = 1.0;
        for (int a = d - 1; a >= 0; a--) {
            int k = rem % m[a]; rem /= m[a];
            J[a] = lo[a] + k;
            w *= (m[a] == 2) ? 0.5 : 1.0;
        }
        int64_t X = j_to_idx(C, J);
        if (!is_unknown(C, X)) continue;
        num += w * e[X];
        den += w;
    }
    return (den > 0.0) ? num / den : 0.0;
}

static void prolong_correct(Level *F, const Level *C) {
    ORC_PARALLEL_FOR
    for (int64_t P = 0; P < F->nn; P++)
        if (is_unknown(F, P)) F->u[P] += prolong_at(F, C, P, C->u);
}

/* ---------------------------------- discrete system (Eq. discr, discrBC) */
static int64_t assemble(const Level *L, int64_t *rows, int64_t *cols, double *vals, int64_t *unk_of_node) {
    int64_t nu = 0, nnz = 0;
    for (int64_t i = 0; i < L->nn; i++) unk_of_node[i] = is_unknown(L, i) ? nu++ : -1;
    for (int64_t i = 0; i < L->nn; i++) {
        if (L->type[i] == T_INT) {
            double ih2 = 1.0 / (L->h * L->h);
            if (rows) { rows[nnz] = unk_of_node[i]; cols[nnz] = unk_of_node[i]; vals[nnz] = 2.0 * L->dim * ih2; }
            nnz++;
            for (int a = 0; a < L->dim; a++)
                for (int sg = -1; sg <= 1; sg += 2) {
                    if (rows) { rows[nnz] = unk_of_node[i]; cols[nnz] = unk_of_node[i + sg * L->st[a]]; vals[nnz] = -ih2; }
                    nnz++;
                }
        } else if (L->type[i] == T_GHOST) {
            int64_t q = L->gid[i];
            const double *w = (L->bc[q] == BC_D) ? L->wD : L->wN;
            for (int k = 0; k < L->nk[q]; k++) {
                if (rows) { rows[nnz] = unk_of_node[i]; cols[nnz] = unk_of_node[L->stn[q * MAXK + k]]; vals[nnz] = w[q * MAXK + k]; }
                nnz++;
            }
        }
    }
    return nnz;
}

/* dense LU with partial pivoting, row-major n x n */
static int lu_factor(double *A, int64_t n, int64_t *piv) {
    for (int64_t k = 0; k < n; k++) {
        int64_t p = k;
        double best = fabs(A[k * n + k]);
        for (int64_t i = k + 1; i < n; i++)
            if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); p = i; }
        if (!(best > 0.0)) return -1;
        piv[k] = p;
        if (p != k)
            for (int64_t j = 0; j < n; j++) { double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t; }
        for (int64_t i = k + 1; i < n; i++) {
            double l = A[i * n + k] / A[k * n + k];
            A[i * n + k] = l;
            if (l != 0.0)
                for (int64_t j = k + 1; j < n; j++) A[i * n + j] -= l * A[k * n + j];
        }
    }
    return 0;
}

static void lu_solve(const double *A, int64_t n, const int64_t *piv, double *b) {
    /* rows were swapped whole during the factorisation: permute b first */
    for (int64_t k = 0; k < n; k++) {
        int64_t p = piv[k];
        if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
    for (int64_t k = 0; k < n; k++)
        for (int64_t i = k + 1; i < n; i++) b[i] -= A[i * n + k] * b[k];
    for (int64_t k = n - 1; k >= 0; k--) {
        double s = b[k];
        for (int64_t j = k + 1; j < n; j++) s -= A[k * n + j] * b[j];
        b[k] = s / A[k * n + k];
    }
}

static int factor_coarsest(Oracle *O, Level *L) {
    int64_t *uon = (int64_t *)malloc(sizeof(int64_t) * (size_t)L->nn);
    int64_t nnz = assemble(L, NULL, NULL, NULL, uon);
    int64_t *rows = (int64_t *)malloc(sizeof(int64_t) * (size_t)nnz);
    int64_t *cols = (int64_t *)malloc(sizeof(int64_t) * (size_t)nnz);
    double *vals = (double *)malloc(sizeof(double) * (size_t)nnz);
    assemble(L, rows, cols, vals, uon);
    int64_t n = 0;
    for (int64_t i = 0; i < L->nn; i++) if (uon[i] >= 0) n++;
    L->nunk = n;
    L->unk = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < L->nn; i++) if (uon[i] >= 0) L->unk[uon[i]] = i;
    L->LU = (double *)calloc((size_t)(n * n + 1), sizeof(double));
    L->piv = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t k = 0; k < nnz; k++) L->LU[rows[k] * n + cols[k]] += vals[k];
    int rc = lu_factor(L->LU, n, L->piv);
    free(uon); free(rows); free(cols); free(vals);
    if (rc != 0) {
        O->status = ORC_E_SINGULAR;
        strcpy(O->err, "singular coarsest-level system");
        return -1;
    }
    return 0;
}

static void coarse_solve(Level *L) {
    double *b = (double *)malloc(sizeof(double) * (size_t)(L->nunk + 1));
    for (int64_t k = 0; k < L->nunk; k++) {
        int64_t i = L->unk[k];
        b[k] = (L->type[i] == T_INT) ? L->f[i] : L->g[L->gid[i]];
    }
    lu_solve(L->LU, L->nunk, L->piv, b);
    for (int64_t i = 0; i < L->nn; i++) L->u[i] = 0.0;
    for (int64_t k = 0; k < L->nunk; k++) L->u[L->unk[k]] = b[k];
    free(b);
}

/* --------------------------------------------------- cycle (TGCS, Sec 2.4)
 * Steps: relax nu1 times, defect, restrict (after extension), solve the
 * coarse residual problem recursively gamma times from zero (exactly on the
 * coarsest grid), interpolate and correct, relax nu2 times.
 */
static void cycle(Oracle *O, int l) {
    Level *L = &O->L[l];
    if (l == O->nlev - 1) { coarse_solve(L); return; }
    Level *C = &O->L[l + 1];
    smooth(O, L, O->p.nu1);
    defect(L, L->u, L->r);
    apply_extension(L, L->r);
    restrict_defect(L, C, L->r, C->f, C->g);
    for (int64_t i = 0; i < C->nn; i++) C->u[i] = 0.0;
    int gam = (l + 1 == O->nlev - 1) ? 1 : O->p.gamma;
    for (int k = 0; k < gam; k++) cycle(O, l + 1);
    prolong_correct(L, C);
    smooth(O, L, O->p.nu2);
}

/* ------------------------------------- reinitialisation (Eq. sdf, Sec. 2.1)
 * phi_t = sgn(phi0) (1 - |grad phi|) from phi = phi0, explicit steps of
 * dt = h / d.  Reading: the paper fixes neither the discretisation nor the
 * number of steps ("a few"); the form taken is the one of the reinitialisation
 * reference it cites (Russo & Smereka): Godunov upwinding of |grad phi| with
 * the sign of phi0 and, at nodes with an axis neighbour across the zero set
 * of phi0, the subcell fix that moves phi towards h phi0 / Delta phi0 (Delta
 * phi0 the largest centred or one-sided difference of phi0 over the axes), so
 * that the zero set stays where phi0 puts it.  Outside the box a node's own
 * value is used (one-sided differences vanish there). */
static double sgn(double x) { return (x > 0.0) - (x < 0.0); }

static void reinit_step(int dim, int n, const double *p0, const double *p, double *q) {
    const double h = 2.0 / (n - 1), dt = h / dim;
    int64_t st[MAXD], nn = 1;
    for (int a = dim - 1; a >= 0; a--) { st[a] = nn; nn *= n; }
    for (int64_t i = 0; i < nn; i++) {
        int j[MAXD];
        int64_t rem = i;
        for (int a = 0; a < dim; a++) { j[a] = (int)(rem / st[a]); rem -= (int64_t)j[a] * st[a]; }
        const double s = sgn(p0[i]);
        int near = 0;
        double dmax = 0.0, g = 0.0;
        for (int a = 0; a < dim; a++) {
            const int64_t im = j[a] > 0 ? i - st[a] : i, ip = j[a] < n - 1 ? i + st[a] : i;
            if (p0[im] * p0[i] < 0.0 || p0[ip] * p0[i] < 0.0) near = 1;
            double d = fabs(p0[ip] - p0[im]) / 2.0;
            if (fabs(p0[ip] - p0[i]) > d) d = fabs(p0[ip] - p0[i]);
            if (fabs(p0[i] - p0[im]) > d) d = fabs(p0[i] - p0[im]);
            if (d > dmax) dmax = d;
            const double bm = (p[i] - p[im]) / h, fw = (p[ip] - p[i]) / h;   /* backward, forward */
            double u2, v2;
            if (s > 0.0) {
                u2 = bm > 0.0 ? bm * bm : 0.0;
                v2 = fw < 0.0 ? fw * fw : 0.0;
            } else {
                u2 = bm < 0.0 ? bm * bm : 0.0;
                v2 = fw > 0.0 ? fw * fw : 0.0;
            }
            g += u2 > v2 ? u2 : v2;
        }
        if (s == 0.0) q[i] = p[i];
        else if (near && dmax > 0.0) q[i] = p[i] - dt / h * (s * fabs(p[i]) - h * p0[i] / dmax);
        else q[i] = p[i] - dt * s * (sqrt(g) - 1.0);
    }
}

/* phi after `steps` steps from phi0 (n^dim nodes of the box [-1,1]^dim) */
void orc_reinit(int dim, int n, const double *phi0, int steps, double *phi) {
    int64_t nn = 1;
    for (int a = 0; a < dim; a++) nn *= n;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)nn);
    memcpy(phi, phi0, sizeof(double) * (size_t)nn);
    for (int k = 0; k < steps; k++) {
        reinit_step(dim, n, phi0, phi, tmp);
        memcpy(phi, tmp, sizeof(double) * (size_t)nn);
    }
    free(tmp);
}

/* ------------------------------------------------------------ public API */

static void free_level(Level *L) {
    free(L->phi); free(L->type); free(L->band); free(L->jzone); free(L->jnode); free(L->jLU); free(L->jpiv); free(L->gnode); free(L->gid);
    free(L->B); free(L->nu); free(L->tloc); free(L->sdir); free(L->gcase); free(L->nk);
    free(L->stn); free(L->wD); free(L->wN); free(L->bc); free(L->c);
    free(L->u); free(L->f); free(L->r); free(L->g); free(L->gtmp);
    free(L->enode); free(L->ensrc); free(L->esrc); free(L->ew);
    free(L->unk); free(L->LU); free(L->piv);
}

void orc_destroy(void *h) {
    Oracle *O = (Oracle *)h;
    if (!O) return;
    for (int l = 0; l < O->nlev; l++) free_level(&O->L[l]);
    free(O->L);
    free(O);
}

/* threads of the loops marked ORC_PARALLEL_FOR (1: serial); returns the
 * count in effect (always 1 without OpenMP) */
int orc_set_threads(int k) {
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
    return omp_get_max_threads();
#else
    (void)k;
    return 1;
#endif
}

int orc_status(void *h) { return ((Oracle *)h)->status; }
const char *orc_error(void *h) { return ((Oracle *)h)->err; }
int orc_num_levels(void *h) { return ((Oracle *)h)->nlev; }
int orc_level_n(void *h, int l) { return ((Oracle *)h)->L[l].n; }
double orc_level_h(void *h, int l) { return ((Oracle *)h)->L[l].h; }
int64_t orc_num_ghosts(void *h, int l) { return ((Oracle *)h)->L[l].ng; }
int64_t orc_num_ext(void *h, int l) { return ((Oracle *)h)->L[l].ne; }
int64_t orc_num_coarse_unknowns(void *h) { Oracle *O = (Oracle *)h; return O->L[O->nlev - 1].nunk; }

/* Builds every level from the fine level set phi (n^dim values).  Coarse
 * levels take phi at their nodes (coarse nodes are fine nodes); the coarse
 * operators are rediscretised (Sec. 1.3, Remark 3).  Returns NULL only on
 * allocation failure; check orc_status. */
void *orc_create(int dim, int n, int n_coarse, const double *phi, const orc_params *p) {
    Oracle *O = (Oracle *)calloc(1, sizeof(Oracle));
    if (!O) return NULL;
    O->dim = dim;
    O->p = *p;
    if (dim < 2 || dim > 3 || n < 5 || n_coarse < 3 || ((n - 1) % (n_coarse - 1)) != 0) {
        O->status = ORC_E_ARG;
        strcpy(O->err, "bad grid sizes");
        return O;
    }
    if (p->smoother < 0 || p->smoother > 1) {
        O->status = ORC_E_ARG;
        strcpy(O->err, "bad smoother");
        return O;
    }
    int nlev = 1, m = n;
    while (m > n_coarse) {
        if ((m - 1) % 2) { O->status = ORC_E_ARG; strcpy(O->err, "n-1 not a power-of-two multiple of n_coarse-1"); return O; }
        m = (m - 1) / 2 + 1;
        nlev++;
    }
    if (m != n_coarse) { O->status = ORC_E_ARG; strcpy(O->err, "bad coarse size"); return O; }
    O->nlev = nlev;
    O->L = (Level *)calloc((size_t)nlev, sizeof(Level));
    for (int l = 0; l < nlev; l++) {
        Level *L = &O->L[l];
        L->dim = dim;
        L->n = (n - 1) / (1 << l) + 1;
        L->h = 2.0 / (double)(L->n - 1);
        L->nn = 1;
        for (int a = 0; a < dim; a++) L->nn *= L->n;
        L->st[dim - 1] = 1;
        for (int a = dim - 2; a >= 0; a--) L->st[a] = L->st[a + 1] * L->n;
        L->phi = (double *)malloc(sizeof(double) * (size_t)L->nn);
        /* phi injected from the fine level */
        int step = 1 << l;
        for (int64_t i = 0; i < L->nn; i++) {
            int j[MAXD];
            idx_to_j(L, i, j);
            int64_t fi = 0, fst = 1;
            for (int a = dim - 1; a >= 0; a--) { fi += (int64_t)j[a] * step * fst; fst *= n; }
            L->phi[i] = phi[fi];
        }
        L->type = (uint8_t *)malloc((size_t)L->nn);
        L->band = (uint8_t *)malloc((size_t)L->nn);
        L->u = (double *)calloc((size_t)L->nn, sizeof(double));
        L->f = (double *)calloc((size_t)L->nn, sizeof(double));
        L->r = (double *)calloc((size_t)L->nn, sizeof(double));
        if (classify(O, L)) return O;
        int64_t ng = L->ng;
        L->gnode = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ng + 1));
        L->gid = (int32_t *)malloc(sizeof(int32_t) * (size_t)L->nn);
        int64_t q = 0;
        for (int64_t i = 0; i < L->nn; i++) {
            L->gid[i] = -1;
            if (L->type[i] == T_GHOST) { L->gnode[q] = i; L->gid[i] = (int32_t)q; q++; }
        }
        L->B = (double *)calloc((size_t)(ng + 1) * dim, sizeof(double));
        L->nu = (double *)calloc((size_t)(ng + 1) * dim, sizeof(double));
        L->tloc = (double *)calloc((size_t)(ng + 1) * dim, sizeof(double));
        L->sdir = (int8_t *)calloc((size_t)(ng + 1) * dim, 1);
        L->gcase = (uint8_t *)calloc((size_t)(ng + 1), 1);
        L->nk = (int32_t *)calloc((size_t)(ng + 1), sizeof(int32_t));
        L->stn = (int64_t *)calloc((size_t)(ng + 1) * MAXK, sizeof(int64_t));
        L->wD = (double *)calloc((size_t)(ng + 1) * MAXK, sizeof(double));
        L->wN = (double *)calloc((size_t)(ng + 1) * MAXK, sizeof(double));
        L->bc = (uint8_t *)calloc((size_t)(ng + 1), 1);
        L->c = (double *)calloc((size_t)(ng + 1), sizeof(double));
        L->g = (double *)calloc((size_t)(ng + 1), sizeof(double));
        L->gtmp = (double *)calloc((size_t)(ng + 1), sizeof(double));
        for (q = 0; q < ng; q++) {
            if (build_ghost(O, L, q)) return O;
            L->c[q] = p->c_dirichlet;
        }
        build_band(L, p->delta_over_h * L->h);
    }
    /* all-Dirichlet until orc_set_bc is called for the coarsest level */
    if (factor_coarsest(O, &O->L[nlev - 1])) return O;
    for (int l = 0; l + 1 < nlev; l++)
        if (build_extension(O, &O->L[l], &O->L[l + 1])) return O;
    return O;
}

/* Boundary-condition type per ghost of level l (0 = Dirichlet, 1 = Neumann);
 * sets the relaxation coefficients mu_D dt or mu_N dt of Sec. 2.3.
 * Reading: in 3D mu_N dt = factor * 2h / (3 sqrt(3)) (the 2D CFL bound with
 * sqrt(2) replaced by sqrt(d)). */
void orc_set_bc(void *h, int l, const uint8_t *bc) {
    Oracle *O = (Oracle *)h;
    Level *L = &O->L[l];
    for (int64_t q = 0; q < L->ng; q++) {
        L->bc[q] = bc[q] ? BC_N : BC_D;
        L->c[q] = (L->bc[q] == BC_D) ? O->p.c_dirichlet
                                     : O->p.c_neumann_factor * 2.0 * L->h / (3.0 * sqrt((double)L->dim));
    }
    build_jzone(L, O->p.junction_radius);
    if (O->p.junction_solve && build_jsolve(L) != 0) {
        O->status = ORC_E_SINGULAR;
        strcpy(O->err, "singular junction-zone system");
    }
    if (l == O->nlev - 1) {
        free(L->unk); free(L->LU); free(L->piv);
        L->unk = NULL; L->LU = NULL; L->piv = NULL;
        factor_coarsest(O, L);
    }
}

/* f on the fine grid (values at Omega_h are used), g per fine ghost */
void orc_set_rhs(void *h, const double *f, const double *g) {
    Oracle *O = (Oracle *)h;
    Level *L = &O->L[0];
    for (int64_t i = 0; i < L->nn; i++) L->f[i] = (L->type[i] == T_INT) ? f[i] : 0.0;
    for (int64_t q = 0; q < L->ng; q++) L->g[q] = g[q];
}

/* f and g of level l: the problem's data sampled on that level (f at its
 * nodes, g at its ghosts' boundary points); used by orc_fmg */
void orc_set_rhs_level(void *h, int l, const double *f, const double *g) {
    Oracle *O = (Oracle *)h;
    Level *L = &O->L[l];
    for (int64_t i = 0; i < L->nn; i++) L->f[i] = (L->type[i] == T_INT) ? f[i] : 0.0;
    for (int64_t q = 0; q < L->ng; q++) L->g[q] = g[q];
}

/* Full multigrid (nested iteration; the paper notes it derives from the
 * V-cycle, Sec. 2.4): the coarsest level's problem solved exactly, then on
 * each finer level l in turn its solution started from the interpolation
 * (Sec. 2.6) of level l+1's and improved by nu cycles with level l as the
 * finest.  Every level's f and g must have been set (orc_set_rhs_level);
 * the cycles at level l overwrite the f and g of the coarser levels, which
 * are not needed again.  u: the fine-grid result. */
void orc_fmg(void *h, int nu, double *u) {
    Oracle *O = (Oracle *)h;
    coarse_solve(&O->L[O->nlev - 1]);
    for (int l = O->nlev - 2; l >= 0; l--) {
        Level *F = &O->L[l];
        const Level *C = &O->L[l + 1];
        for (int64_t P = 0; P < F->nn; P++) F->u[P] = is_unknown(F, P) ? prolong_at(F, C, P, C->u) : 0.0;
        for (int k = 0; k < nu; k++) cycle(O, l);
    }
    memcpy(u, O->L[0].u, sizeof(double) * (size_t)O->L[0].nn);
}

void orc_get_types(void *h, int l, uint8_t *out) {
    Level *L = &((Oracle *)h)->L[l];
    memcpy(out, L->type, (size_t)L->nn);
}

void orc_get_jzone(void *h, int l, uint8_t *out) {
    Level *L = &((Oracle *)h)->L[l];
    if (L->jzone) memcpy(out, L->jzone, (size_t)L->nn);
    else memset(out, 0, (size_t)L->nn);
}

/* nodes whose equations the exact junction solve of level l solves (mask) */
void orc_get_jsolve(void *h, int l, uint8_t *out) {
    Level *L = &((Oracle *)h)->L[l];
    memset(out, 0, (size_t)L->nn);
    for (int64_t k = 0; k < L->jn; k++) out[L->jnode[k]] = 1;
}

void orc_get_band(void *h, int l, uint8_t *out) {
    Level *L = &((Oracle *)h)->L[l];
    memcpy(out, L->band, (size_t)L->nn);
}

void orc_get_ghosts(void *h, int l, int64_t *node, double *B, double *nu, double *t, int8_t *s,
                    uint8_t *scase, int32_t *nk, int64_t *stn, double *wD, double *wN) {
    Level *L = &((Oracle *)h)->L[l];
    int64_t ng = L->ng;
    int d = L->dim;
    if (node) memcpy(node, L->gnode, sizeof(int64_t) * (size_t)ng);
    if (B) memcpy(B, L->B, sizeof(double) * (size_t)ng * d);
    if (nu) memcpy(nu, L->nu, sizeof(double) * (size_t)ng * d);
    if (t) memcpy(t, L->tloc, sizeof(double) * (size_t)ng * d);
    if (s) memcpy(s, L->sdir, (size_t)ng * d);
    if (scase) memcpy(scase, L->gcase, (size_t)ng);
    if (nk) memcpy(nk, L->nk, sizeof(int32_t) * (size_t)ng);
    if (stn) memcpy(stn, L->stn, sizeof(int64_t) * (size_t)ng * MAXK);
    if (wD) memcpy(wD, L->wD, sizeof(double) * (size_t)ng * MAXK);
    if (wN) memcpy(wN, L->wN, sizeof(double) * (size_t)ng * MAXK);
}

void orc_get_ext(void *h, int l, int64_t *enode, int32_t *nsrc, int64_t *src, double *w) {
    Level *L = &((Oracle *)h)->L[l];
    if (enode) memcpy(enode, L->enode, sizeof(int64_t) * (size_t)L->ne);
    if (nsrc) memcpy(nsrc, L->ensrc, sizeof(int32_t) * (size_t)L->ne);
    if (src) memcpy(src, L->esrc, sizeof(int64_t) * (size_t)L->ne * 2 * MAXD);
    if (w) memcpy(w, L->ew, sizeof(double) * (size_t)L->ne * 2 * MAXD);
}

/* Defect of u (fine grid values) at level l with that level's f, g. */
double orc_defect(void *h, int l, const double *u, double *r) {
    Level *L = &((Oracle *)h)->L[l];
    defect(L, u, r);
    return max_abs_unknowns(L, r);
}

/* Extension applied in place to a grid function r of level l */
void orc_extend(void *h, int l, double *r) { apply_extension(&((Oracle *)h)->L[l], r); }

/* Composite restriction of a fine grid function r (level l) to level l+1:
 * fc (coarse grid, interior nodes) and gc (per coarse ghost). */
void orc_restrict(void *h, int l, const double *r, double *fc, double *gc) {
    Oracle *O = (Oracle *)h;
    restrict_defect(&O->L[l], &O->L[l + 1], r, fc, gc);
}

/* Weights of the partial transfer at coarse node X of level l+1 */
int orc_restrict_weights(void *h, int l, int64_t X, int interior_set, double *wt) {
    Oracle *O = (Oracle *)h;
    const Level *C = &O->L[l + 1];
    int J[MAXD], jf[MAXD];
    idx_to_j(C, X, J);
    for (int a = 0; a < C->dim; a++) jf[a] = 2 * J[a];
    return partial_weights(&O->L[l], jf, interior_set, wt);
}

/* Interpolation of a coarse grid function e (level l+1) onto level l:
 * out = I e on Omega_h u Gamma_h, 0 elsewhere. */
void orc_prolong(void *h, int l, const double *e, double *out) {
    Oracle *O = (Oracle *)h;
    const Level *F = &O->L[l], *C = &O->L[l + 1];
    for (int64_t P = 0; P < F->nn; P++) out[P] = is_unknown(F, P) ? prolong_at(F, C, P, e) : 0.0;
}

/* One relaxation of u in place at level l: the base sweep, then (with_extra)
 * the lambda band sweeps and the junction sweeps */
void orc_relax(void *h, int l, double *u, const double *f, const double *g, int with_extra) {
    Oracle *O = (Oracle *)h;
    Level *L = &O->L[l];
    memcpy(L->u, u, sizeof(double) * (size_t)L->nn);
    for (int64_t i = 0; i < L->nn; i++) L->f[i] = (L->type[i] == T_INT) ? f[i] : 0.0;
    memcpy(L->g, g, sizeof(double) * (size_t)L->ng);
    if (O->p.smoother == 1) {
        kaczmarz_relax(O, L, with_extra);
        memcpy(u, L->u, sizeof(double) * (size_t)L->nn);
        return;
    }
    base_relax(O, L);
    if (with_extra) {
        extra_sweeps(O, L);
        if (O->p.junction_sweeps || O->p.junction_solve) junction_relax(O, L);
    }
    memcpy(u, L->u, sizeof(double) * (size_t)L->nn);
}

/* One Kaczmarz step (Sec. 3.3) on the row of node i of level l, applied to u
 * in place, with the level's right-hand side f, g (inside f at inside nodes). */
void orc_kaczmarz_row(void *h, int l, int64_t i, double *u, const double *f, const double *g) {
    Level *L = &((Oracle *)h)->L[l];
    memcpy(L->u, u, sizeof(double) * (size_t)L->nn);
    for (int64_t k = 0; k < L->nn; k++) L->f[k] = (L->type[k] == T_INT) ? f[k] : 0.0;
    memcpy(L->g, g, sizeof(double) * (size_t)L->ng);
    kaczmarz_row(L, i);
    memcpy(u, L->u, sizeof(double) * (size_t)L->nn);
}

/* Number of nonzeros of the level-l system; with non-NULL arrays, fills the
 * COO triplets over unknowns numbered in increasing node index. */
int64_t orc_assemble(void *h, int l, int64_t *rows, int64_t *cols, double *vals, int64_t *unk_of_node) {
    Level *L = &((Oracle *)h)->L[l];
    int64_t *tmp = unk_of_node ? unk_of_node : (int64_t *)malloc(sizeof(int64_t) * (size_t)L->nn);
    int64_t nnz = assemble(L, rows, cols, vals, tmp);
    if (!unk_of_node) free(tmp);
    return nnz;
}

/* Multigrid solve from the initial guess u (fine grid, in/out).  norms[m] =
 * max-norm defect over Omega_h u Gamma_h after m cycles (norms[0]: initial).
 * Stops when norms[m] <= rtol * norms[0] or after max_cycles.  Returns the
 * number of cycles done; *status: 0 converged, ORC_E_NOCONV otherwise. */
int orc_solve(void *h, double *u, double rtol, int max_cycles, double *norms, int *status) {
    Oracle *O = (Oracle *)h;
    Level *L = &O->L[0];
    for (int64_t i = 0; i < L->nn; i++) L->u[i] = is_unknown(L, i) ? u[i] : 0.0;
    double n0 = orc_defect(h, 0, L->u, L->r);
    norms[0] = n0;
    int m = 0;
    *status = ORC_E_NOCONV;
    if (n0 == 0.0) { *status = ORC_OK; }
    else {
        while (m < max_cycles) {
            cycle(O, 0);
            m++;
            double nm = orc_defect(h, 0, L->u, L->r);
            norms[m] = nm;
            if (nm != nm) break;
            if (nm <= rtol * n0) { *status = ORC_OK; break; }
        }
    }
    memcpy(u, L->u, sizeof(double) * (size_t)L->nn);
    return m;
}
