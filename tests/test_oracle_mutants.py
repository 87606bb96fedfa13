"""Planted mistakes: each test compiles the oracle with one plausible error
(a transposed block, a wrong weight or coefficient, a dropped term, a wrong
sign) and checks that the pins of test_oracle_pins.py catch it.  The
mutations live only in temporary copies of the oracle's C source."""
import pytest

import oracle
import test_oracle_pins as pins

MUTANTS = [
    ("lower_block_not_transposed",
     "colsum[2 * j] += row[j] * xr;", "colsum[2 * j] += Ul[(long)j * n + i] * xr;",
     lambda: pins.test_dmatvec_matches_dense_bruteforce(2, 4)),
    ("rk4_weight",
     "k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]", "k1[q] + 1.0 * k2[q] + 2.0 * k3[q] + k4[q]",
     lambda: pins.test_field_free_rk4_is_stability_polynomial(1)),
    ("taylor_term_factor",
     "T[q] = (dt / m) * Tn[q];", "T[q] = (dt / (m + 1)) * Tn[q];",
     lambda: pins.test_field_free_taylor_is_truncated_exponential(6)),
    ("half_step_field",
     "return 0.5 * (F[k] + F[k + 1]);", "return F[k];",
     lambda: pins.test_step_grid_samples_interpolate_linearly()),
    ("velocity_gauge_sign",
     "const double re = up[2 * a] - dn[2 * a], im = up[2 * a + 1] - dn[2 * a + 1];",
     "const double re = up[2 * a] + dn[2 * a], im = up[2 * a + 1] + dn[2 * a + 1];",
     lambda: pins.test_velocity_gauge_product_matches_dense_bruteforce(2, 3)),
    ("fehlberg_coefficient",
     "-845.0 / 4104.0, 0.0},", "-845.0 / 4105.0, 0.0},",
     lambda: pins.test_rkf45_tableau_satisfies_the_order_conditions()),
    ("gauss_legendre_weight",
     "const double w1 = (322.0 + 13.0 * sqrt(70.0)) / 900.0", "const double w1 = (322.0 + 13.0 * sqrt(70.0)) / 901.0",
     lambda: pins.test_vector_potential_gauss_legendre_matches_the_closed_form()),
    ("adjoint_loss_gradient",
     "G[2 * a] = 2.0 * w[a] * cT[2 * a];", "G[2 * a] = w[a] * cT[2 * a];",
     lambda: pins.test_adjoint_matches_central_differences("rk4", 4, 1, 0)),
    ("lanczos_three_term_recurrence",
     "if (j > 0) w[q] -= be[j] * V[(long)(j - 1) * 2 * N + q];", "(void)0;",
     lambda: pins.test_lanczos_full_krylov_space_is_the_exact_exponential()),
    ("zero_energy_counted_as_bound",
     "if (E[a] < 0.0) b += p; else io += p;", "if (E[a] <= 0.0) b += p; else io += p;",
     lambda: pins.test_populations_partition_the_norm()),
    ("eigenvector_rotation_sign",
     "z[k * m + q] = sn * vp + cs * vq;", "z[k * m + q] = -sn * vp + cs * vq;",
     lambda: pins.test_tridiagonal_eigensolver_matches_numpy(7)),
    ("rk4_last_stage_at_mid_step",
     "orc_field_at(F, samples_per_step, k, 2), dt, work, NULL);",
     "orc_field_at(F, samples_per_step, k, 1), dt, work, NULL);",
     lambda: pins.test_convergence_orders_time_dependent_field()),
    ("adjoint_forward_pass_last_stage_at_mid_step",
     "orc_field_at(F, sps, k, 2), dt, work, NULL);", "orc_field_at(F, sps, k, 1), dt, work, NULL);",
     lambda: pins.test_adjoint_matches_central_differences("rk4", 4, 2, 0)),
    ("taylor_mid_hold_ignored",
     "return orc_field_at(F, sps, k, hold ? 1 : 0);", "return orc_field_at(F, sps, k, 0);",
     lambda: pins.test_convergence_orders_time_dependent_field()),
    ("gauss_legendre_node",
     "const double x1 = sqrt(5.0 - r) / 3.0", "const double x1 = sqrt(5.0 - r) / 3.1",
     lambda: pins.test_vector_potential_gauss_legendre_matches_the_closed_form()),
    ("vector_potential_sign",
     "if (k > 0) A -= gl5(", "if (k > 0) A += gl5(",
     lambda: pins.test_vector_potential_gauss_legendre_matches_the_closed_form()),
    ("lanczos_diagonal_scale",
     "a += vj[q] * w[q];     /* Re<v, w> */", "a += 0.5 * vj[q] * w[q];     /* Re<v, w> */",
     lambda: pins.test_lanczos_full_krylov_space_is_the_exact_exponential()),
    ("fehlberg_embedded_weight",
     "2197.0 / 4104.0, -1.0 / 5.0, 0.0}", "2197.0 / 4104.0, -1.0 / 6.0, 0.0}",
     lambda: pins.test_rkf45_tableau_satisfies_the_order_conditions()),
    ("rkf_safety_factor",
     "0.9 * pow(tol / err, 0.2)", "0.8 * pow(tol / err, 0.2)",
     lambda: pins.test_rkf45_controller_matches_an_independent_simulation()),
]


@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_a_planted_mistake(name, old, new, pin):
    src = oracle.source()
    assert src.count(old) == 1, "mutation site not found: " + name
    with oracle.variant(src.replace(old, new), name):
        with pytest.raises(AssertionError):
            pin()
    pin()                       # the unmutated oracle passes the same pin
