"""Each pin must be able to fail: plant a plausible mistake in a temporary copy
of the oracle (on the CPU), rebuild it, and check that the pin meant to guard
that part rejects it.  The real oracle is untouched."""

import os

import pytest

import oracle as O
from tests import test_oracle_pins as pins

# (name, original text, planted text, pin that must fail, pin arguments)
MUTATIONS = [
    ("rectangle path backtracks",
     "const pstep wbwd[5] = {{mu, -1}, {nu, s}, {mu, +1}, {mu, +1}, {nu, -s}};",
     "const pstep wbwd[5] = {{nu, s}, {mu, -1}, {mu, +1}, {mu, +1}, {nu, -s}};",
     pins.test_generator_is_action_gradient_finite_difference, (-0.25,)),
    ("tall rectangle dropped",
     "const pstep *rp[3] = {tall, wfwd, wbwd};\n                for (int r = 0; r < 3; ++r) {",
     "const pstep *rp[3] = {tall, wfwd, wbwd};\n                for (int r = 1; r < 3; ++r) {",
     pins.test_generator_is_action_gradient_finite_difference, (-0.25,)),
    ("trace term of Q dropped",
     "cplx q = 0.5 * A.m[i][j] - (i == j ? trA / 6.0 : 0.0);",
     "cplx q = 0.5 * A.m[i][j];",
     pins.test_annealed_smoothing_matches_diagonal_restatement, (-0.25, False, (8, 4, 4, 4))),
    ("generator not anti-symmetrised",
     "for (int j = 0; j < 3; ++j) Q.m[i][j] = 0.5 * A.m[i][j] - (i == j ? trA / 6.0 : 0.0);",
     "for (int j = 0; j < 3; ++j) Q.m[i][j] = 0.5 * Om.m[i][j] - (i == j ? trA / 6.0 : 0.0);",
     pins.test_generator_is_action_gradient_finite_difference, (1.0,)),
    ("rectangle coefficient sign",
     "*c1 = (eps - 1.0) / (12.0 * u0 * u0);",
     "*c1 = (1.0 - eps) / (12.0 * u0 * u0);",
     pins.test_overimproved_coefficients_and_alpha_min, ()),
    ("centrifuge rotates both phases the same way",
     "ph[pk[p]] = (1.0 + omega) * lam - omega * sigma;",
     "ph[pk[p]] = (1.0 - omega) * lam + omega * sigma;",
     pins.test_centrifuge_closed_forms, ()),
    ("centrifuge staple phase index",
     "- LAM(nu, xm_nu) + LAM(mu, xm_nu) + LAM(nu, xm_nu_p_mu);",
     "- LAM(nu, xm_nu) + LAM(mu, xp_nu) + LAM(nu, xm_nu_p_mu);",
     pins.test_centrifuge_closed_forms, ()),
    ("sector boundary at pi/2",
     "if (arg > -OR_PI / 3.0 && arg < OR_PI / 3.0) return 0;",
     "if (arg > -OR_PI / 2.0 && arg < OR_PI / 2.0) return 0;",
     pins.test_label_matches_nearest_centre_on_haar_matrices, ()),
    ("exponential truncated",
     "for (int n = 1; n < 40; ++n) {",
     "for (int n = 1; n < 4; ++n) {",
     pins.test_expm_against_eigendecomposition_and_closed_forms, ()),
    ("colour classes without the factor 2",
     "int cc = 2 * x[mu];",
     "int cc = x[mu];",
     pins.test_annealed_smoothing_matches_diagonal_restatement, (-0.25, True, (4, 4, 8, 4))),
    ("action prefactor",
     "Sx /= (2.0 * 3.0 * 4.0 * 3.0);",
     "Sx /= (2.0 * 3.0 * 4.0 * 4.0);",
     pins.test_action_closed_forms, ()),
    ("plaquette orientation",
     "const pstep plaq[4] = {{mu, +1}, {nu, +1}, {mu, -1}, {nu, -1}};",
     "const pstep plaq[4] = {{mu, +1}, {nu, +1}, {nu, -1}, {mu, -1}};",
     pins.test_action_closed_forms, ()),
    ("vortex preservation against the current label",
     "if (vp && label_of_trace(tr) != ref_labels[li]) {",
     "if (vp && label_of_trace(tr) != label_of_trace(m_trace(&Ux))) {",
     pins.test_vortex_preservation_keeps_original_labels, ()),
    ("blocking weight of the staples",
     "m_axpy(&Vb, alpha / 6.0, &S);\n                    mat3 Un = maxretr",
     "m_axpy(&Vb, alpha / 3.0, &S);\n                    mat3 Un = maxretr",
     pins.test_aus_below_alpha_min_leaves_vortex_fields_unchanged, ()),
    ("APE blocking weight before the unit circle projection",
     "m_axpy(&Vb, alpha / 6.0, &S);\n                    mat3 Un;\n",
     "m_axpy(&Vb, alpha / 4.0, &S);\n                    mat3 Un;\n",
     pins.test_ape_ucp_blocking_weights_on_a_constant_field, ("simultaneous",)),
    ("unit circle projection without the determinant phase",
     "cplx f = cexp(-I * phi / 3.0);",
     "cplx f = 1.0;",
     pins.test_ucp_is_the_special_unitary_polar_factor, ()),
    ("unit circle projection with (V^dag V)^-1",
     "E.m[i][k] * (1.0 / sqrt(lam[k])) * conj(E.m[j][k])",
     "E.m[i][k] * (1.0 / lam[k]) * conj(E.m[j][k])",
     pins.test_ucp_is_the_special_unitary_polar_factor, ()),
    ("Runge-Kutta stage coefficient",
     "(8.0 / 9.0) * Z1[i].m[a][b] - (17.0 / 36.0)",
     "(8.0 / 9.0) * Z1[i].m[a][b] - (17.0 / 35.0)",
     pins.test_flow_rk3_is_third_order_and_euler_first_order, ()),
    ("Runge-Kutta first stage weight",
     "X[i].m[a][b] = 0.25 * Z0[i].m[a][b];",
     "X[i].m[a][b] = 0.3 * Z0[i].m[a][b];",
     pins.test_flow_rk3_is_third_order_and_euler_first_order, ()),
    ("vortex preservation ignores the random gauge",
     "    if (!G) return m_trace(Un);",
     "    return m_trace(Un);",
     pins.test_vortex_preservation_in_random_gauge, ()),
    ("clover leaf with the wrong orientation",
     "{{nu, -1}, {mu, +1}, {nu, +1}, {mu, -1}}};",
     "{{mu, +1}, {nu, -1}, {mu, -1}, {nu, +1}}};",
     pins.test_topological_charge_density_on_two_plane_flux, ()),
    ("reconstructed action without the 1/2",
     "sr += 0.5 * creal(m_trace(&FF));",
     "sr += creal(m_trace(&FF));",
     pins.test_reconstructed_action_on_uniform_flux, ()),
    ("re-unitarisation projects with <r1, r0>",
     "for (int k = 0; k < 3; ++k) ip += conj(r0[k]) * r1[k];",
     "for (int k = 0; k < 3; ++k) ip += r0[k] * conj(r1[k]);",
     pins.test_reunit_rows_are_the_qr_factor_and_special_unitary, ()),
    ("re-unitarisation third row not conjugated",
     "r2[k] = conj(r0[a] * r1[b] - r0[b] * r1[a]);",
     "r2[k] = r0[a] * r1[b] - r0[b] * r1[a];",
     pins.test_reunit_rows_are_the_qr_factor_and_special_unitary, ()),
    ("site index with transposed extents",
     "return x[0] + (long)g->L[0] * (x[1] + (long)g->L[1] * (x[2] + (long)g->L[2] * x[3]));",
     "return x[0] + (long)g->L[1] * (x[1] + (long)g->L[0] * (x[2] + (long)g->L[2] * x[3]));",
     pins.test_periodic_extension_repeats_the_result, ()),
    ("cooling subgroup conjugation",
     "Tc.m[p][q] = -be / k;",
     "Tc.m[p][q] = be / k;",
     pins.test_cooling_lowers_action_and_stays_in_su3, ()),
]


@pytest.mark.parametrize("name,old,new,pin,args", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, pin, args):
    src = O.source()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    path = O.compile_variant(src.replace(old, new), str(tmp_path / "liboracle_mut.so"))
    with O.use_library(path):
        with pytest.raises((AssertionError, ValueError)):
            pin(*args)
    # and the unmodified oracle still passes the same pin
    pin(*args)
