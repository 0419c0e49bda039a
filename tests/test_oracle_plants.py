"""Planted slips: each pin of the oracle must catch a plausible mistake.

Every case below copies the oracle's C source, plants one mistake in one of
its functions (a wrong Lagrange weight or derivative, the sign of B - G, a
dropped ghost row in GS-LEX, a reversed sweep order, a restriction weight,
...), compiles the copy into a temporary library and runs the pin named
beside it against that library.  The pin must fail; the same pin passes on
the unmodified oracle in test_oracle.py / test_oracle_paper_mode.py.  Every
function of the oracle's arithmetic carries at least one planted slip here.
"""
import os

import pytest

import oracle
import test_oracle as T
import test_oracle_paper_mode as PM
from paper_1111_0983_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "gcmg_oracle.c")

# (function, what is planted, original text, planted text, pin)
PLANTS = [
    ("lagr3", "derivative of the middle Lagrange weight",
     "dw[1] = 2.0 - 2.0 * t;", "dw[1] = 2.0 - 1.0 * t;",
     lambda: T.test_quadratic_rows_exact(2, 33, "all")),
    ("lagr3", "third Lagrange weight",
     "w[2] = t * (t - 1.0) / 2.0;", "w[2] = t * (t + 1.0) / 2.0;",
     lambda: T.test_quadratic_rows_exact(2, 33, "none")),
    ("build_ghost", "sign of B - G",
     "delta[a] = -phiG * gphi[a] / gg;", "delta[a] = phiG * gphi[a] / gg;",
     T.test_closest_point_lies_on_sdf_boundary),
    ("build_ghost", "discrete normal not normalised",
     "for (int a = 0; a < d; a++) L->nu[q * d + a] = gn[a] / nrm;",
     "for (int a = 0; a < d; a++) L->nu[q * d + a] = gn[a];",
     T.test_ghost_weight_identities),
    ("tensor_stencil", "gradient weight without the other axes' factors",
     "if (b != a) gw *= ax[b].w[kk[b]];", "if (b != a) gw *= 1.0;",
     lambda: T.test_quadratic_rows_exact(2, 33, "all")),
    ("axis_lin", "linear rule's weights swapped",
     "A->w[0] = 1.0 - t; A->w[1] = t;", "A->w[0] = t; A->w[1] = 1.0 - t;",
     lambda: T.test_linear_rows_exact_all_stencils(inputs.star(27), 33)),
    ("interior_update", "interior Gauss-Seidel divisor",
     "L->u[i] = s / (2.0 * L->dim);", "L->u[i] = s / (2.0 * L->dim + 0.5);",
     lambda: PM.test_discrete_solution_is_a_fixed_point_of_each_relaxation(0)),
    ("ghost_jacobi", "sign of the ghost step",
     "    for (int64_t q = 0; q < L->ng; q++)\n        L->gtmp[q] = L->u[L->gnode[q]] + L->c[q]",
     "    for (int64_t q = 0; q < L->ng; q++)\n        L->gtmp[q] = L->u[L->gnode[q]] - L->c[q]",
     lambda: T.test_multigrid_matches_direct_solve(inputs.disk(), 33, 9)),
    ("lex_sweep", "ghost rows left out of GS-LEX",
     "L->u[i] += L->c[q] * (L->g[q] - ghost_operator(L, q, L->u));",
     "L->u[i] += 0.0 * L->c[q] * (L->g[q] - ghost_operator(L, q, L->u));",
     PM.test_gslex_relaxes_the_ghost_rows),
    ("lex_sweep", "band test applied to the ghosts",
     "        } else if (L->type[i] == T_GHOST) {\n            int64_t q = L->gid[i];\n            L->u[i] +=",
     "        } else if (L->type[i] == T_GHOST && !band_only) {\n            int64_t q = L->gid[i];\n            L->u[i] +=",
     PM.test_gslex_relaxes_the_ghost_rows),
    ("lex_sweep", "sweep in reverse node order",
     "static void lex_sweep(Level *L, int band_only) {\n    for (int64_t i = 0; i < L->nn; i++) {",
     "static void lex_sweep(Level *L, int band_only) {\n    for (int64_t i = L->nn - 1; i >= 0; i--) {",
     PM.test_gslex_moves_a_perturbation_forward_in_node_order),
    ("lex_sweep", "band nodes skipped in the band sweeps",
     "            if (band_only && !L->band[i]) continue;\n            interior_update(L, i);",
     "            if (band_only) continue;\n            interior_update(L, i);",
     PM.test_gslex_table_rhoC_W_cycle_nu3),
    ("smooth", "extra sweeps after the phase only when nu > 1",
     "if (O->p.extra_once && nu > 0) extra_sweeps(O, L);", "if (O->p.extra_once && nu > 1) extra_sweeps(O, L);",
     PM.test_extra_once_equals_default_for_single_sweeps),
    ("extra_sweeps", "ghost sweep left out of the red-black band sweeps",
     "        else { rb_sweep(L, 1); ghost_jacobi(L); }\n    }\n}",
     "        else { rb_sweep(L, 1); }\n    }\n}",
     T.test_paper_table_rhoC_W_cycle_nu3),
    ("build_band", "band narrower than delta",
     "if (dist >= -delta) L->band[i] = 1;", "if (dist >= -0.3 * delta) L->band[i] = 1;",
     PM.test_gslex_table_rhoC_W_cycle_nu3),
    ("defect", "sign of the Laplacian in the defect",
     "            r[i] = L->f[i] + lap / (L->h * L->h);", "            r[i] = L->f[i] - lap / (L->h * L->h);",
     lambda: T.test_multigrid_matches_direct_solve(inputs.disk(), 33, 9)),
    ("w1d", "full-weighting factor",
     "if (alpha == -1 && beta == 1) return (o == 0) ? 0.5 : 0.25;",
     "if (alpha == -1 && beta == 1) return (o == 0) ? 0.4 : 0.3;",
     T.test_restriction_printed_stencils),
    ("partial_weights", "tied boxes summed, not averaged",
     "for (int c = 0; c < nnb; c++) wt[c] /= (double)count;", "for (int c = 0; c < nnb; c++) wt[c] /= 1.0;",
     T.test_restriction_partition_of_unity),
    ("prolong_at", "interpolation weight squared",
     "num += w * e[X];", "num += w * w * e[X];",
     T.test_prolongation_linear_exact_where_parents_exist),
    ("build_extension", "extension weight 1 instead of |n_a|",
     "F->ew[e * 2 * MAXD + m] = fabs(g[a]);", "F->ew[e * 2 * MAXD + m] = 1.0;",
     T.test_extension_constants_and_normal_invariance),
    ("cmp_phiidx", "extension order by decreasing phi",
     "    if (a->phi < b->phi) return -1;\n    if (a->phi > b->phi) return 1;",
     "    if (a->phi < b->phi) return 1;\n    if (a->phi > b->phi) return -1;",
     T.test_extension_is_upwind_ordered),
    ("apply_extension", "extension weights ignored",
     "v += F->ew[e * 2 * MAXD + i] * r[F->esrc[e * 2 * MAXD + i]];",
     "v += 0.5 * r[F->esrc[e * 2 * MAXD + i]];",
     T.test_extension_constants_and_normal_invariance),
    ("coarse_solve", "ghost data dropped on the coarsest grid",
     "b[k] = (L->type[i] == T_INT) ? L->f[i] : L->g[L->gid[i]];", "b[k] = (L->type[i] == T_INT) ? L->f[i] : 0.0;",
     T.test_fmg_single_level_is_direct_solve),
    ("cycle", "W-cycle recursion taken once",
     "int gam = (l + 1 == O->nlev - 1) ? 1 : O->p.gamma;", "int gam = 1;",
     T.test_paper_table_badrho_degradation),
    ("zone_solve", "junction correction subtracted",
     "for (int64_t k = 0; k < L->jn; k++) L->u[L->jnode[k]] += b[k];",
     "for (int64_t k = 0; k < L->jn; k++) L->u[L->jnode[k]] -= b[k];",
     T.test_junction_solve_is_exact_on_its_set),
    ("kaczmarz_row", "ghost row step halved",
     "const double t = (L->g[q] - s) / n2;", "const double t = (L->g[q] - s) / (2.0 * n2);",
     T.test_kaczmarz_step_moves_along_its_row_and_satisfies_it),
    ("reinit_step", "subcell fix without its sign",
     "q[i] = p[i] - dt / h * (s * fabs(p[i]) - h * p0[i] / dmax);",
     "q[i] = p[i] - dt / h * (fabs(p[i]) - h * p0[i] / dmax);",
     lambda: T.test_reinit_distance_function(2, 129)),
]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as fh:
        return fh.read()


@pytest.mark.parametrize("func,what,old,new,pin", PLANTS, ids=[f"{p[0]}: {p[1]}" for p in PLANTS])
def test_planted_slip_fails_its_pin(source, tmp_path, func, what, old, new, pin):
    assert source.count(old) == 1, f"planting site not unique in {func}"
    path = oracle.build_variant(source.replace(old, new), str(tmp_path))
    with oracle.variant(path):
        with pytest.raises((AssertionError, oracle.OracleError, FloatingPointError, ValueError)):
            pin()


def test_every_oracle_function_carries_a_plant(source):
    """The arithmetic functions of the oracle (everything but index helpers,
    memory management and the exported wrappers) are each planted above, or
    are exercised only through a planted caller listed here."""
    import re
    planted = {p[0] for p in PLANTS}
    via_caller = {
        "idx_to_j", "j_to_idx", "j_in_box", "is_unknown", "parity", "coord", "grad_phi", "on_box_edge",
        "stencil_ok", "free_level", "lu_factor", "lu_solve", "assemble", "factor_coarsest",
        "max_abs_unknowns", "in_set", "partial_transfer", "restrict_defect", "prolong_correct",
        "ghost_operator", "rb_sweep", "base_relax", "zone_sweep", "build_jzone", "row_defect",
        "build_jsolve", "junction_relax", "kaczmarz_colour", "in_kaczmarz_set", "kaczmarz_sweep",
        "kaczmarz_relax", "classify", "axis_quad", "sgn",
    }
    statics = set(re.findall(r"^static \w[\w\s\*]*?\b(\w+)\(", source, flags=re.M))
    missing = statics - planted - via_caller
    assert not missing, sorted(missing)
