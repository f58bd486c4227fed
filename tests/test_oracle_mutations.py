"""Planted mistakes in the oracle, each of which one of its pins must catch.

Every case takes one function of ``oracle/`` as it is written, changes one
expression into a plausible mistake (a dropped term or weight, a swapped
index, a transposed operand, a missing assembly or mask), and runs one pin
from the oracle's own test files against that mutant: the pin must fail.
The unmutated pins pass in their own files, so together this shows that the
pins constrain each of these parts of the oracle rather than merely agreeing
with it.  The mistakes are planted in the oracle on the CPU only; nothing
here touches the CUDA path.
"""

import importlib
import inspect
import os
import sys
import textwrap

import numpy as np
import pytest

from oracle import geometry, gll, mesh, numbering, operator, pressure, projection, schwarz, solver

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _pins(name):
    return importlib.import_module(name)


def _mutant(owner, name, old, new):
    """The function ``owner.name`` recompiled from its own source with the
    one occurrence of ``old`` replaced by ``new``, in its module's globals."""
    fn = inspect.unwrap(getattr(owner, name))
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, f"{name}: the planted snippet must occur exactly once"
    ns = dict(sys.modules[fn.__module__].__dict__)
    exec(compile(src.replace(old, new), f"<mutant of {fn.__module__}.{name}>", "exec"), ns)
    return ns[name]


# (id, owner, function, original text, mistake, other (owner, name) bindings of
#  the same function, pin module, pin call)
CASES = [
    # -- GLL basis (nodes, weights, D)
    ("legendre_recurrence_coefficient", gll, "legendre",
     "- k * p_prev) / (k + 1)", "- (k + 1) * p_prev) / (k + 1)", [],
     "test_oracle_gll", lambda t: t.test_closed_form_nodes_weights(3)),
    ("gll_weight_unsquared", gll, "nodes_weights",
     "pn * pn)", "pn)", [],
     "test_oracle_gll", lambda t: t.test_quadrature_exact_to_degree_2N_minus_1(4)),
    ("derivative_corner_entry", gll, "derivative_matrix",
     "D[0, 0] = -N * (N + 1) / 4.0", "D[0, 0] = -N * (N + 1) / 2.0", [],
     "test_oracle_gll", lambda t: t.test_derivative_exact_on_polynomials(5)),
    # -- geometric factors G = w detJ J^-1 J^-T and B
    ("metric_transposed", geometry, "factors",
     'np.einsum("...ba,...ca->...bc", Jinv, Jinv)', 'np.einsum("...ab,...ac->...bc", Jinv, Jinv)', [],
     "test_oracle_geometry", lambda t: t.test_sheared_element_factors()),
    ("metric_without_detJ", geometry, "factors",
     "scale = w3[None] * detJ", "scale = w3[None] * np.ones_like(detJ)", [],
     "test_oracle_geometry", lambda t: t.test_affine_box_factors_closed_form()),
    ("g4_takes_the_rt_entry", geometry, "factors",
     "G[:, 3] = scale * M[..., 0, 1]", "G[:, 3] = scale * M[..., 0, 2]", [],
     "test_oracle_geometry", lambda t: t.test_sheared_element_factors()),
    ("jacobian_transposed", geometry, "jacobian",
     "J[..., a, 0] = fr\n        J[..., a, 1] = fs\n        J[..., a, 2] = ft",
     "J[..., 0, a] = fr\n        J[..., 1, a] = fs\n        J[..., 2, a] = ft", [],
     "test_oracle_geometry", lambda t: t.test_sheared_element_factors()),
    # -- local operator (Alg. 1 + h2 B u)
    ("wr_cross_terms_swapped", operator, "ax_local",
     "wr = h1 * (g1 * ur + g4 * us + g5 * ut)", "wr = h1 * (g1 * ur + g5 * us + g4 * ut)", [(solver, "ax_local")],
     "test_oracle_operator", lambda t: t.test_constants_in_kernel_and_symmetry_on_curved_pipe()),
    ("back_contraction_with_D_not_DT", operator, "ax_local",
     'np.einsum("li,ekjl->ekji", D, wr)', 'np.einsum("il,ekjl->ekji", D, wr)', [(solver, "ax_local")],
     "test_oracle_operator", lambda t: t.test_constants_in_kernel_and_symmetry_on_curved_pipe()),
    ("mass_term_without_B", operator, "ax_local",
     "w = w + h2 * B * u", "w = w + h2 * u", [(solver, "ax_local")],
     "test_oracle_operator", lambda t: t.test_affine_element_matches_kronecker_matrix(3, 0.3, 2.5)),
    ("diagonal_cross_term_weight", operator, "local_diagonal",
     "2.0 * di * dj * g4", "1.0 * di * dj * g4", [(solver, "local_diagonal")],
     "test_oracle_operator", lambda t: t.test_local_diagonal_matches_unit_vectors_on_curved_element()),
]

CASES += [
    # -- numbering, QQ^T and the Dirichlet mask
    ("no_periodic_identification", numbering, "global_numbering",
     "if mesh.period is not None:", "if False:", [],
     "test_oracle_numbering", lambda t: t.test_pipe_counts_and_multiplicities(2, 1, 2, 3, True)),
    ("gather_overwrites_instead_of_summing", numbering, "gs",
     "np.add.at(s, glo, flat)", "s[glo] = flat", [],
     "test_oracle_numbering", lambda t: t.test_gs_pins()),
    ("face_1_is_the_j_face", numbering, "face_points",
     "sel[:, :, n - 1] = True", "sel[:, n - 1, :] = True", [],
     "test_oracle_numbering", lambda t: t.test_dirichlet_mask_pipe()),
    # -- assembled operator, Jacobi diagonal, PCG
    ("jacobi_diagonal_not_assembled", solver.Problem, "jacobi_inverse",
     "d = self.gs(local_diagonal(", "d = (local_diagonal(", [],
     "test_oracle_solver", lambda t: t.test_dense_spd_pcg_matches_cholesky(lambda: mesh.box(2, 2, 2, 3), 0.0)),
    ("inner_product_without_multiplicity", solver.Problem, "dot",
     "np.sum(a * b / self.mult)", "np.sum(a * b)", [],
     "test_oracle_solver",
     lambda t: t.test_pcg_iterates_minimise_the_energy_error_over_the_krylov_space(
         lambda: mesh.pipe(2, 1, 2, 3, L=2.0), 0.0)),
    ("cg_beta_inverted", solver, "pcg",
     "beta = rho_new / rho", "beta = rho / rho_new", [],
     "test_oracle_solver",
     lambda t: t.test_pcg_iterates_minimise_the_energy_error_over_the_krylov_space(
         lambda: mesh.pipe(2, 1, 2, 3, L=2.0), 0.0)),
    ("cg_step_with_r_dot_r", solver, "pcg",
     "alpha = rho / sigma", "alpha = prob.dot(r, r) / sigma", [],
     "test_oracle_solver",
     lambda t: t.test_pcg_iterates_minimise_the_energy_error_over_the_krylov_space(
         lambda: mesh.box(2, 2, 2, 3), 1.5)),
    ("cg_unpreconditioned_inside_the_loop", solver, "pcg",
     "        z = Minv * r\n        rho_new", "        z = r\n        rho_new", [],
     "test_oracle_solver",
     lambda t: t.test_pcg_iterates_minimise_the_energy_error_over_the_krylov_space(
         lambda: mesh.pipe(2, 1, 2, 3, L=2.0), 0.0)),
    ("refinement_correction_not_rescaled", solver, "pcg_mixed",
     "x = x + rnorm * d.astype(np.float64)", "x = x + d.astype(np.float64)", [],
     "test_oracle_solver", lambda t: t.test_mixed_precision_refinement(1e-5)),
    ("reliable_update_restarts_cg", solver, "pcg_mixed_reliable",
     "            rr_max = p32.dot(r, r)\n", "            rr_max = p32.dot(r, r)\n            p = 0 * p\n", [],
     "test_oracle_solver", lambda t: t.test_reliable_updates_keep_the_krylov_iterates(0.9)),
    ("reliable_update_increment_not_rescaled", solver, "pcg_mixed_reliable",
     "x = x + x32.astype(np.float64) / s\n            x32[:] = 0.0",
     "x = x + x32.astype(np.float64)\n            x32[:] = 0.0", [],
     "test_oracle_solver", lambda t: t.test_mixed_reliable_updates()),
    ("fp32_operator_unmasked", solver.Problem32, "A",
     "return self.mask * self.prob.gs(w)", "return self.prob.gs(w)", [],
     "test_oracle_solver", lambda t: t.test_mixed_precision_refinement(1e-5)),
    ("fp32_cg_beta_inverted", solver, "pcg32",
     "beta = np.float32(rho_new / rho)", "beta = np.float32(rho / rho_new)", [],
     "test_oracle_solver", lambda t: t.test_fp32_inner_pcg_iterates_follow_the_krylov_optimum()),
    # -- projection onto previous solutions
    ("projection_never_restarts", projection.Projection, "solve",
     "if len(self.X) >= self.max_vectors:", "if False:", [],
     "test_oracle_projection", lambda t: t.test_full_basis_restarts_from_the_newest_solution()),
    ("projection_basis_euclidean_orthogonal", projection.Projection, "_append",
     "beta = [P.dot(ax, v) for ax in self.AX]", "beta = [P.dot(x, v) for x in self.X]", [],
     "test_oracle_projection", lambda t: t.test_basis_is_a_orthonormal()),
    ("projection_coefficients_with_A", projection.Projection, "guess",
     "coef = [self.prob.dot(x, b) for x in self.X]", "coef = [self.prob.dot(self.prob.A(x), b) for x in self.X]", [],
     "test_oracle_projection", lambda t: t.test_guess_is_the_dense_a_orthogonal_projection()),
]

CASES += [
    # -- pressure operator E = D B^-1 D^T (Sec. 2, Eq. 5)
    ("adjugate_transposed", pressure, "div_factors",
     'np.einsum("ekjiba,kji->ebakji", adj, rho3)', 'np.einsum("ekjiab,kji->ebakji", adj, rho3)', [],
     "test_oracle_pressure", lambda t: t.test_divergence_of_coordinates_is_gl_volume_on_curved_pipe()),
    ("divergence_without_gl_weights", pressure, "div_factors",
     'np.einsum("ekjiba,kji->ebakji", adj, rho3)', 'np.einsum("ekjiba,kji->ebakji", adj, np.ones_like(rho3))', [],
     "test_oracle_pressure", lambda t: t.test_affine_element_matches_kronecker_divergence(4)),  # two GL points have unit weights
    ("gradient_directions_swapped", pressure, "grad_local",
     "mats = [(I.T, I.T, Dg.T), (I.T, Dg.T, I.T), (Dg.T, I.T, I.T)]",
     "mats = [(I.T, Dg.T, I.T), (I.T, I.T, Dg.T), (Dg.T, I.T, I.T)]", [],
     "test_oracle_pressure", lambda t: t.test_gradient_is_the_transpose_of_divergence()),
    ("inverse_mass_without_mask", pressure.Pressure, "minv",
     "return self.prob.mask * self.prob.gs(v) / self.Bg", "return self.prob.gs(v) / self.Bg", [],
     "test_oracle_pressure", lambda t: t.test_consistent_poisson_operator_has_only_the_constant_null_mode()),
    ("inverse_mass_unassembled", pressure.Pressure, "minv",
     "return self.prob.mask * self.prob.gs(v) / self.Bg", "return self.prob.mask * self.prob.gs(v / self.prob.B)", [],
     "test_oracle_pressure", lambda t: t.test_diagonal_is_the_dense_diagonal("pipe", 3)),
    ("pressure_diagonal_rows_not_squared", pressure.Pressure, "diagonal",
     "row * row", "row", [],
     "test_oracle_pressure", lambda t: t.test_diagonal_is_the_dense_diagonal("box", 3)),
    ("lagrange_derivative_sign", pressure, "lagrange_derivative",
     "1.0 / (x_nodes[l] - xq)", "1.0 / (xq - x_nodes[l])", [],
     "test_oracle_pressure", lambda t: t.test_interpolation_and_derivative_at_gl_points(6)),
    ("lagrange_basis_denominator_sign", gll, "lagrange_eval",
     "(t - xm) / (x_nodes[j] - xm)", "(t - xm) / (xm - x_nodes[j])", [],
     # N sign flips: the same polynomial at even N, so the pin runs at odd N
     "test_oracle_pressure", lambda t: t.test_interpolation_and_derivative_at_gl_points(3)),
    ("pressure_space_with_n_gl_points", pressure, "interpolation_matrices",
     "gl_nodes_weights(N - 1)", "gl_nodes_weights(N)", [],
     "test_oracle_pressure", lambda t: t.test_interpolation_and_derivative_at_gl_points(6)),
    # -- overlapping Schwarz local solves (Sec. 2, Eq. 6)
    ("element_lengths_r_and_s_swapped", schwarz, "element_lengths",
     "np.stack([lr, ls, lt], axis=1)", "np.stack([ls, lr, lt], axis=1)", [],
     "test_oracle_schwarz",
     lambda t: t.test_fdm_local_solve_is_the_exact_overlapping_subdomain_inverse_on_a_tensor_box(0.0)),
    ("face_neighbour_recorded_on_one_side", schwarz, "face_neighbours",
     "nb[e2, f2] = (e1, f1)", "nb[e2, f2] = (-1, -1)", [],
     "test_oracle_schwarz",
     lambda t: t.test_fdm_local_solve_is_the_exact_overlapping_subdomain_inverse_on_a_tensor_box(0.0)),
    ("fdm_extension_with_own_length", schwarz, "fdm_1d",
     "K[end, end] += (2.0 / ln) * Kref[N, N]", "K[end, end] += (2.0 / l) * Kref[N, N]", [],
     "test_oracle_schwarz",
     lambda t: t.test_fdm_local_solve_is_the_exact_overlapping_subdomain_inverse_on_a_tensor_box(0.0)),
    ("fdm_extension_without_mass", schwarz, "fdm_1d",
     "B[end, end] += (ln / 2.0) * w[N]", "B[end, end] += 0.0 * w[N]", [],
     "test_oracle_schwarz",
     lambda t: t.test_fdm_local_solve_is_the_exact_overlapping_subdomain_inverse_on_a_tensor_box(2.5)),
    ("pressure_cg_operator_not_projected", pressure, "cg",
     "w = P.E(p)\n        w = w - w.mean()\n", "w = P.E(p)\n", [],
     "test_oracle_pressure",
     lambda t: t.test_pressure_cg_matches_dense_solve_on_the_mean_free_space(lambda: mesh.pipe(2, 1, 3, 3, L=1.5))),
    ("pressure_cg_beta_inverted", pressure, "cg",
     "p = z + (rho_new / rho) * p", "p = z + (rho / rho_new) * p", [],
     "test_oracle_pressure", lambda t: t.test_pressure_cg_iterates_minimise_the_energy_error_over_the_krylov_space(False)),
    ("pressure_cg_step_with_r_dot_r", pressure, "cg",
     "alpha = rho / sigma", "alpha = np.sum(r * r) / sigma", [],
     "test_oracle_pressure", lambda t: t.test_pressure_cg_iterates_minimise_the_energy_error_over_the_krylov_space(True)),
    ("pressure_jacobi_not_projected", pressure, "cg",
     "return z - z.mean()", "return z", [],
     "test_oracle_pressure", lambda t: t.test_jacobi_cg_reaches_the_plain_solution_in_fewer_iterations()),
    ("schwarz_weight_on_one_side", schwarz.Schwarz, "apply",
     "self.prob.gs(W * self.local_solve(W * r))", "self.prob.gs(self.local_solve(W * r))", [],
     "test_oracle_schwarz",
     lambda t: t.test_preconditioner_is_symmetric_positive_definite(lambda: mesh.box(2, 2, 2, 3), False)),
    ("coarse_restriction_counts_copies", schwarz.Schwarz, "restrict",
     "r / self.prob.mult", "r", [],
     "test_oracle_schwarz",
     lambda t: t.test_preconditioner_is_symmetric_positive_definite(lambda: mesh.pipe(2, 1, 3, 3, L=1.5), True)),
    ("coarse_functions_i_and_k_swapped", schwarz.Schwarz, "_coarse_space",
     "fk[:, None, None] * fj[None, :, None] * fi[None, None, :]",
     "fi[:, None, None] * fj[None, :, None] * fk[None, None, :]", [],
     "test_oracle_schwarz", lambda t: t.test_coarse_functions_reproduce_trilinear_fields()),
    ("schwarz_cg_beta_inverted", schwarz, "pcg",
     "p = z + (rho_new / rho) * p", "p = z + (rho / rho_new) * p", [],
     "test_oracle_schwarz", lambda t: t.test_schwarz_pcg_iterates_minimise_the_energy_error_over_the_krylov_space()),
    ("fdm_local_solve_without_h2", schwarz.Schwarz, "local_solve",
     "+ lt[:, :, None, None]) + h2", "+ lt[:, :, None, None])", [],
     "test_oracle_schwarz",
     lambda t: t.test_fdm_local_solve_is_the_exact_overlapping_subdomain_inverse_on_a_tensor_box(2.5)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(case, monkeypatch):
    _, owner, name, old, new, others, pin_module, pin = case
    bad = _mutant(owner, name, old, new)
    monkeypatch.setattr(owner, name, bad)
    for o, n in others:
        monkeypatch.setattr(o, n, bad)
    with pytest.raises((AssertionError, np.linalg.LinAlgError)):
        pin(_pins(pin_module))


def test_every_planted_snippet_is_in_the_oracle():
    """The list above tracks the oracle's text: each planted mistake replaces
    an expression that occurs exactly once in its function."""
    for _, owner, name, old, _new, _o, _m, _p in CASES:
        src = inspect.getsource(inspect.unwrap(getattr(owner, name)))
        assert src.count(old) == 1, name
