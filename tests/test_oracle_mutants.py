"""Planted mistakes in the oracle: each mutant is a copy of the oracle's C
source with one plausible error (a dropped term, a wrong sign, factor, operand
or index), compiled on the CPU and swapped in for the real oracle while the pin
that targets it runs. The pin must fail on the mutant; the unchanged oracle
passes every pin (tests/test_oracle_pins.py). This shows the pins are tied to
what the paper and the mathematics fix, not to the oracle's own code."""
import inspect
import itertools
import os

import pytest

import oracle
import test_oracle_pins as pins

# (name, original source text, planted mistake, pins that must fail)
MUTANTS = [
    # kernel, neighbours, walls
    ("sigma_3d", "if (dim == 3) return 1.0 / (120.0 * ORC_PI * h * h * h);",
     "if (dim == 3) return 3.0 / (359.0 * ORC_PI * h * h * h);", ["test_kernel_integrates_to_one"]),
    ("minimum_image", "if (dx > halfL) dx = dx - L;", "if (dx > L) dx = dx - L;", ["test_neighbours_match_kdtree"]),
    ("cell_ring", "for (int dx = -1; dx <= 1; ++dx) {", "for (int dx = 0; dx <= 1; ++dx) {",
     ["test_cell_list_equals_bruteforce"]),
    ("wall_g_sign", "sg = sg + P->rho0 * gr * W;", "sg = sg - P->rho0 * gr * W;",
     ["test_wall_pressure_and_ghost_velocity"]),
    ("ghost_velocity", "vghost[w * dim + a] = 2.0 * vw[w * dim + a] - sv[a] / sw;",
     "vghost[w * dim + a] = vw[w * dim + a] - sv[a] / sw;", ["test_wall_pressure_and_ghost_velocity"]),
    # pair terms, Eqs. (dp-dtau-frozen-edac, mom-sph-frozen)
    ("divergence_c", "api = api + m * rho / rho * c * c * vij_gw;", "api = api + m * rho / rho * c * vij_gw;",
     ["test_divergence_term"]),
    ("edac_factor", "api = api + 4.0 * m / ((rho + rho) * rho) * nu_e", "api = api + 2.0 * m / ((rho + rho) * rho) * nu_e",
     ["test_edac_diffusion_term_and_denominator_reading"]),
    ("pressure_pj_sign", "double pres = p[i] / (rho * rho) + pj / (rho * rho) + pi_ij;",
     "double pres = p[i] / (rho * rho) - pj / (rho * rho) + pi_ij;", ["test_pressure_gradient_term"]),
    ("viscous_factor", "double visc = m * 4.0 * P->nu", "double visc = m * 2.0 * P->nu", ["test_viscous_term"]),
    # artificial viscosity, Eqs. (mom-av, av-phiij)
    ("av_switch", "if (vr < 0.0) {", "if (vr > 0.0) {", ["test_artificial_viscosity_structure"]),
    ("av_v_sum", "vr = vr + (vi[a] - vvis[a]) * d[a];", "vr = vr + (vi[a] + vvis[a]) * d[a];",
     ["test_artificial_viscosity_structure"]),
    ("av_no_h", "pi_ij = -P->alpha * h * c * phi / rho;", "pi_ij = -P->alpha * c * phi / rho;",
     ["test_artificial_viscosity_magnitude_against_its_continuum_limit"]),
    ("av_c_squared", "pi_ij = -P->alpha * h * c * phi / rho;", "pi_ij = -P->alpha * h * c * c * phi / rho;",
     ["test_artificial_viscosity_structure", "test_artificial_viscosity_magnitude_against_its_continuum_limit"]),
    ("av_no_rho", "pi_ij = -P->alpha * h * c * phi / rho;", "pi_ij = -P->alpha * h * c * phi;",
     ["test_artificial_viscosity_structure"]),
    ("av_sign", "pi_ij = -P->alpha * h * c * phi / rho;", "pi_ij = P->alpha * h * c * phi / rho;",
     ["test_artificial_viscosity_magnitude_against_its_continuum_limit"]),
    ("av_denominator", "double phi = vr / (r2 + P->eta * h * h);", "double phi = vr / (r2 + h * h);",
     ["test_artificial_viscosity_magnitude_against_its_continuum_limit"]),
    # shifting, Eqs. (shift-deltar, shift-correct)
    ("shift_missing_half", "-0.5 * h * h * dr[i * dim + a]", "-1.0 * h * h * dr[i * dim + a]",
     ["test_shifting_displacement_matches_its_continuum_limit"]),
    ("shift_sign", "-0.5 * h * h * dr[i * dim + a]", "0.5 * h * h * dr[i * dim + a]",
     ["test_shifting_is_zero_on_a_lattice_and_reduces_disorder",
      "test_shifting_displacement_matches_its_continuum_limit"]),
    ("shift_drop_one", "(1.0 + W / wdx)", "(W / wdx)", ["test_shifting_displacement_matches_its_continuum_limit"]),
    ("shift_drop_w", "(1.0 + W / wdx)", "(1.0)", ["test_shifting_displacement_matches_its_continuum_limit"]),
    ("shift_walls_left_out", "dr[i * dim + a] = dr[i * dim + a] + vol * (1.0 + W / wdx) * gw;",
     "if (j < nf) dr[i * dim + a] = dr[i * dim + a] + vol * (1.0 + W / wdx) * gw;",
     ["test_shifting_counts_wall_particles_in_the_displacement"]),
    ("taylor_p_sign", "p[i] = p[i] + dp;", "p[i] = p[i] - dp;", ["test_shifting_taylor_correction_carries_linear_fields"]),
    ("taylor_p_dropped", "p[i] = p[i] + dp;", "p[i] = p[i];", ["test_shifting_taylor_correction_carries_linear_fields"]),
    ("taylor_v_dropped", "v[i * dim + b] = v[i * dim + b] + dvb;", "v[i * dim + b] = v[i * dim + b];",
     ["test_shifting_taylor_correction_carries_linear_fields"]),
    ("taylor_wrong_field", "vol * (p[j] - p[i]) * gw", "vol * (v[j * dim] - v[i * dim]) * gw",
     ["test_shifting_taylor_correction_carries_linear_fields"]),
    # Algorithm 2: predictor, BDF2, pseudo-time update, residuals, r-update
    ("bdf_weight", "double bdf = (3.0 * vk[q] - 4.0 * v[q] + v_prev[q]) / (2.0 * dt);",
     "double bdf = (3.0 * vk[q] - 4.0 * v[q] - v_prev[q]) / (2.0 * dt);", ["test_uniform_flow_is_a_fixed_point"]),
    ("kappa", "double kappa = 2.0 * dt / (2.0 * dt + 3.0 * dtau);", "double kappa = 2.0 * dt / (2.0 * dt + 2.0 * dtau);",
     ["test_pseudo_iteration_contraction_rate"]),
    ("predictor_r", "x0[k] = x[k] + dt * v[k] + dt * dt / 2.0 * F[k];", "x0[k] = x[k] + dt * v[k];",
     ["test_uniform_acceleration_is_exact"]),
    ("predictor_v", "vk[k] = v[k] + dt * F[k];", "vk[k] = v[k] + 0.5 * dt * F[k];", ["test_uniform_acceleration_is_exact"]),
    ("r_update", "if (!P->steady) x[q] = x[q] + dt / 2.0 * (v[q] + vk[q]);",
     "if (!P->steady) x[q] = x[q] + dt * vk[q];", ["test_uniform_acceleration_is_exact"]),
    ("half_step", "phalf[i] = pk[i] + 0.5 * dtau * ap_prev[i];", "phalf[i] = pk[i];", ["test_converged_step_solves_bdf2"]),
    ("rv_scaling", "sum_av = sum_av + dt * sqrt(av2);", "sum_av = sum_av + sqrt(av2);",
     ["test_pseudo_iteration_contraction_rate"]),
    # free-surface runs
    ("free_surface_clamp", "if (P->free_surface && pw[w] < 0.0) pw[w] = 0.0;", ";",
     ["test_free_surface_wall_pressure_is_kept_positive"]),
    ("free_surface_walls_left_out", "if (r > 0.0) divr = divr - vol * dwdr * r;",
     "if (r > 0.0 && j < nf) divr = divr - vol * dwdr * r;", ["test_free_surface_particles_are_not_shifted"]),
]


def _run_pin(fn):
    """Calls a pin over every combination of its parametrize marks."""
    params = {}
    for mark in getattr(fn, "pytestmark", []):
        if mark.name == "parametrize":
            params[mark.args[0]] = list(mark.args[1])
    if not params:
        fn()
        return
    keys = list(params)
    for combo in itertools.product(*(params[k] for k in keys)):
        fn(**dict(zip(keys, combo)))


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return str(tmp_path_factory.mktemp("oracle_mutants"))


@pytest.mark.parametrize("name,original,mistake,targets", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pin(name, original, mistake, targets, mutant_dir):
    src = oracle.source()
    assert src.count(original) == 1, f"{name}: the oracle text this mutant edits has changed"
    path = oracle.compile_source(src.replace(original, mistake), os.path.join(mutant_dir, f"{name}.so"))
    good = oracle.lib()
    oracle._lib = oracle.bind(path)
    try:
        for pin in targets:
            fn = getattr(pins, pin)
            assert inspect.isfunction(fn)
            with pytest.raises(AssertionError):
                _run_pin(fn)
    finally:
        oracle._lib = good
