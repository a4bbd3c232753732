"""Mutation check of the oracle's pins (CPU): each plausible mistake below is planted in a copy of
oracle/dg_oracle.c (never in the file itself), compiled, and the pins of test_oracle_pins.py must fail
for it.  This shows that the pins pin the oracle rather than restate it."""

import os
import subprocess
import tempfile

import pytest

import oracle
from tests import test_oracle_pins as pins
from tests import test_oracle_tensor_pins as xpins
from tests import test_oracle_bc_pins as bpins
from tests import test_oracle_multilinear_pins as mpins
from tests import test_oracle_transport_pins as tpins

SRC = os.path.join(os.path.dirname(oracle.__file__), "dg_oracle.c")

# (name, original text, mutated text)
MUTANTS = [
    ("weighted average sign", "wm * dnum + wp * dnup", "wm * dnum - wp * dnup"),
    ("upwind branch swapped", "return bnu >= 0.0 ? um * bnu : up * bnu;", "return bnu >= 0.0 ? up * bnu : um * bnu;"),
    ("penalty dropped", "+ gam * jump_u * jump_v", "+ 0.0 * gam * jump_u * jump_v"),
    ("symmetry term sign", "- avg_dv * jump_u", "+ avg_dv * jump_u"),
    ("convection sign", "fl[r] = Dg[r] - br * uq;", "fl[r] = Dg[r] + br * uq;"),
    ("transposed basis index", "t->grad[o * 3 + 1] = v[0][j1] * d[1][j2] * v[2][j3];",
     "t->grad[o * 3 + 1] = v[0][j1] * d[1][j3] * v[2][j2];"),
    ("boundary normal sign", "double nout[3] = {sgn * nu[0], sgn * nu[1], sgn * nu[2]};\n          double Db_[3][3];",
     "double nout[3] = {nu[0], nu[1], nu[2]};\n          double Db_[3][3];"),
    ("Gauss weight", "w[i] = 1.0 / ((1.0 - t * t) * dP[m] * dP[m]);", "w[i] = 2.0 / ((1.0 - t * t) * dP[m] * dP[m]);"),
    ("Dirichlet data sign in the right hand side", "- dnv * g + gam * g * v", "+ dnv * g + gam * g * v"),
    ("reaction dropped", "cq * uq * ph[i]", "0.0 * cq * uq * ph[i]"),
    ("harmonic mean replaced by arithmetic mean", "return 2.0 * a * b / (a + b);", "return 0.5 * (a + b);"),
    ("face weight swapped", "double wm = dp / (dm + dp), wp = dm / (dm + dp);",
     "double wm = dm / (dm + dp), wp = dp / (dm + dp);"),
    ("periodic wrap dropped", "if (pr->periodic[dir]) nic[dir] = (nic[dir] + pr->n[dir]) % pr->n[dir];",
     "if (0) nic[dir] = (nic[dir] + pr->n[dir]) % pr->n[dir];"),
    ("periodic wrap off by one", "nic[dir] = (nic[dir] + pr->n[dir]) % pr->n[dir];",
     "nic[dir] = (nic[dir] + pr->n[dir] + 1) % pr->n[dir];"),
    ("interior face velocity ignored", "double bnu = bfp ? bfp[p] : bdotn;", "double bnu = bdotn;"),
    ("volume velocity component", "pr->b_vol[((size_t)cell * cx->vol.np + p) * 3 + r]",
     "pr->b_vol[((size_t)cell * cx->vol.np + p) * 3 + 0]"),
    ("tensor off-diagonal entry", "Dm[0][1] = Dm[1][0] = t[3];", "Dm[0][1] = Dm[1][0] = t[4];"),
    ("gradient mapped by J^-1 instead of J^-T", "g[a] += Jinv[r][a] * gref[r];", "g[a] += Jinv[a][r] * gref[r];"),
    ("face normal from a column of J^-1 instead of a row", "for (int a = 0; a < 3; ++a) nu[a] = g->Jinv[r][a] / len;",
     "for (int a = 0; a < 3; ++a) nu[a] = g->Jinv[a][r] / len;"),
    ("face area element without the normal scale", "return g->det * len;", "return g->det;"),
    ("neighbour's tensor from its far face", "unpack6(pr->D_face + (((size_t)nbr * 6 + oface) * ft->np + p) * 6, Dn_);",
     "unpack6(pr->D_face + (((size_t)nbr * 6 + 2 * dir + side) * ft->np + p) * 6, Dn_);"),
    ("point-wise reaction ignored", "const double cq = pr->c_vol ? pr->c_vol[(size_t)cell * cx->vol.np + p] : pr->c;",
     "const double cq = pr->c;"),
    ("trilinear shape derivative sign", "dN[r] = corner[r] ? 1.0 : -1.0;", "dN[r] = corner[r] ? 1.0 : 1.0;"),
    ("neighbour's gradient with the own cell's geometry", "eval_fe(nt, p, zn, Gn.Jinv, &un, gn);",
     "eval_fe(nt, p, zn, Go.Jinv, &un, gn);"),
    ("penalty with the larger cell volume", "const double vmin = volT < volN ? volT : volN;",
     "const double vmin = volT > volN ? volT : volN;"),
    ("volume element dropped on multilinear cells", "v += cx->vol.wgt[p] * g.det;", "v += cx->vol.wgt[p];"),
    ("Neumann flux sign in the right hand side", "y[i] -= dx * jf * ph[i];", "y[i] += dx * jf * ph[i];"),
    ("outflow face without its upwind flux", "y[i] += dx * upwind(us, 0.0, bnu) * ph[i];",
     "y[i] += 0.0 * dx * upwind(us, 0.0, bnu) * ph[i];"),
    ("Neumann face given the Dirichlet terms", "} else if (pr->bc[2 * dir + side] == BC_NEUMANN) {",
     "} else if (0) {"),
]


def _pin_checks():
    """The fast pins, each returning normally when it holds."""
    yield lambda: pins.test_gauss_legendre_matches_numpy(5)
    yield lambda: pins.test_basis_matches_numpy_and_is_orthonormal(3)
    for case in pins.KRON_CASES[1:3]:
        yield lambda case=case: pins.test_oracle_matches_kronecker_closed_form(case)
    yield lambda: pins.test_polynomial_solution_has_zero_residual(2, (3, 2, 2))
    yield pins.test_diffusion_part_is_symmetric_and_coercive
    yield lambda: pins.test_global_conservation((1.0, 0.5, 0.25))
    yield pins.test_reaction_term_is_mass_matrix
    yield pins.test_rhs_constant_source
    yield lambda: tpins.test_periodic_matches_kronecker_closed_form((1, 0, 0))
    yield tpins.test_constant_field_given_at_points_equals_constant_velocity
    yield tpins.test_periodic_transport_conserves_mass_exactly
    yield tpins.test_periodic_translation_invariance
    yield lambda: xpins.test_tensor_diffusion_matches_kronecker_closed_form((2, 3, 2), 2, (0, 0, 0))
    yield lambda: xpins.test_linear_map_scales_the_operator_by_its_determinant(2)
    yield lambda: xpins.test_polynomial_solution_on_affine_mesh_has_zero_residual(2)
    yield lambda: xpins.test_polynomial_solution_with_polynomial_coefficients_has_zero_residual(2)
    yield lambda: bpins.test_mixed_boundary_types_match_kronecker_closed_form(bpins.BC_CASES[0])
    yield lambda: bpins.test_polynomial_solution_with_mixed_boundary_types_has_zero_residual(2)
    yield bpins.test_neumann_rhs_closed_form
    yield lambda: mpins.test_quadratic_solution_on_multilinear_mesh_has_zero_residual(2)
    yield mpins.test_volume_element_integrates_the_domain
    yield mpins.test_interior_penalty_on_multilinear_cells
    yield lambda: mpins.test_affine_vertices_reproduce_the_affine_map(2, 3)


@pytest.mark.parametrize("name,orig,mutated", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, orig, mutated):
    text = open(SRC).read()
    assert text.count(orig) == 1, f"mutation site for '{name}' not found exactly once"
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "mutant.c")
        lib = os.path.join(d, "libmutant.so")
        open(src, "w").write(text.replace(orig, mutated))
        subprocess.run(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-o", lib, src, "-lm"],
                       check=True)
        caught = []
        with oracle.use_library(lib):
            for check in _pin_checks():
                try:
                    check()
                except AssertionError:
                    caught.append(check)
    assert caught, f"no pin fails for the planted mistake: {name}"


def test_unmutated_oracle_passes_the_same_pins():
    for check in _pin_checks():
        check()
