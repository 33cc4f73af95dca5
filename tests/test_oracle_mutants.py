"""Planted mistakes in the oracle: each variant changes one expression of
the FP64 oracle the way a plausible slip would (a dropped term, a flipped
sign, a wrong factor, a one-sided average), is compiled into its own
library, and must fail the pin named beside it.  This shows that the pins in
test_oracle_pins.py constrain every part of the step they are meant to:
AB2 and Crank-Nicolson weights (Sec. 2.2), the pressure gradient, the
convective face average, the ellipse of Sec. 2.1, the forcing-node
interpolation, the outflow flux balance, the mass source, the projection,
the pressure update, the added-mass term of the force, the drag's sign and
normalisation and the SOR update.  CPU only.
"""
import pytest

import oracle
import test_oracle_pins as pins

MUTANTS = {
    "ab2_as_euler": (
        [("-1.5 * S->Hu[id] + 0.5 * S->Huo[id]", "-1.0 * S->Hu[id] + 0.0 * S->Huo[id]")],
        pins.test_time_integration_second_order, ()),
    "ab2_as_euler_in_v": (
        [("-1.5 * S->Hv[id] + 0.5 * S->Hvo[id]", "-1.0 * S->Hv[id] + 0.0 * S->Hvo[id]")],
        pins.test_time_integration_second_order, ()),
    "pressure_gradient_sign_in_v": (
        [("+ 0.5 * S->Hvo[id] - gp)", "+ 0.5 * S->Hvo[id] + gp)")],
        pins.test_taylor_green_decay_second_order, ()),
    "explicit_viscous_half_doubled": (
        [("beta * lap_u_at(S, S->u, i, j)", "2.0 * beta * lap_u_at(S, S->u, i, j)")],
        pins.test_taylor_green_decay_second_order, ()),
    "pressure_gradient_sign": (
        [("+ 0.5 * S->Huo[id] - gp)", "+ 0.5 * S->Huo[id] + gp)")],
        pins.test_taylor_green_decay_second_order, ()),
    "one_sided_face_velocity": (
        [("double ue = 0.5 * (u[UI(i, j)] + u[UI(i + 1, j)]);", "double ue = u[UI(i, j)];")],
        pins.test_convection_and_diffusion_operators_second_order, ()),
    "ellipse_minor_axis_doubled": (
        [("bb = 0.5 * S->tc * S->chord", "bb = S->tc * S->chord")],
        pins.test_solid_area_converges_first_order, ()),
    "mass_source_without_body_mean": (
        [("S->cut[id] ? S->D[id] - cbar : 0.0", "S->cut[id] ? S->D[id] : 0.0")],
        pins.test_step_divergence_bound_and_zero_net_mass_source_in_body_cells, ()),
    "added_mass_sign": (
        [("(sy - S->S_prev[1]) * idt", "(S->S_prev[1] - sy) * idt")],
        pins.test_plunging_circle_feels_added_mass_force, ()),
    "interpolation_weight_inverted": (
        [("al[id] = best / (best + D);", "al[id] = D / (best + D);")],
        pins.test_classification_matches_brute_force, (0.37,)),
    "forcing_from_the_wrong_neighbour": (
        [("int oi = i + (d == 0) - (d == 1), oj = j + (d == 2) - (d == 3);",
          "int oi = i - (d == 0) + (d == 1), oj = j - (d == 2) + (d == 3);")],
        pins.test_velocity_sor_matches_dense_solve, (0,)),
    "outflow_flux_correction_dropped": (
        [("for (int j = 0; j < ny; ++j) S->uh[UI(nx, j)] += corr;", "(void)corr;")],
        pins.test_step_divergence_bound_and_zero_net_mass_source_in_body_cells, ()),
    "projection_sign": (
        [("S->u[id] = S->uh[id] - dt * OVER(", "S->u[id] = S->uh[id] + dt * OVER(")],
        pins.test_step_divergence_bound_and_zero_net_mass_source_in_body_cells, ()),
    "pressure_not_accumulated": (
        [("S->p[id] += S->phi[id];", "S->p[id] = S->phi[id];")],
        pins.test_taylor_green_decay_second_order, ()),
    "u_east_diffusion_wrong_cell": (
        [("    S->uE[i] = 1.0 / (S->dx[i] * S->dxc[i]);", "    S->uE[i] = 1.0 / (S->dx[i - 1] * S->dxc[i]);")],
        pins.test_velocity_laplacians_on_a_stretched_grid, ()),
    "u_north_diffusion_wrong_spacing": (
        [("S->uN[j] = j < ny - 1 ? 1.0 / (S->dyc[j + 1] * S->dy[j]) : 0.0;",
          "S->uN[j] = j < ny - 1 ? 1.0 / (S->dyc[j + 1] * S->dy[j + 1]) : 0.0;")],
        pins.test_velocity_laplacians_on_a_stretched_grid, ()),
    "v_south_diffusion_wrong_cell": (
        [("S->vS[j] = 1.0 / (S->dy[j - 1] * S->dyc[j]);", "S->vS[j] = 1.0 / (S->dy[j] * S->dyc[j]);")],
        pins.test_velocity_laplacians_on_a_stretched_grid, ()),
    "u_cross_flux_midpoint_weights": (
        [("  double w = S->wx[i];\n  if (j < ny - 1) {", "  double w = 0.5;\n  if (j < ny - 1) {")],
        pins.test_convection_cross_terms_on_a_stretched_grid, ()),
    "v_cross_flux_midpoint_weights": (
        [("  double w = S->wy[j];\n  double ue", "  double w = 0.5;\n  double ue")],
        pins.test_convection_cross_terms_on_a_stretched_grid, ()),
    "drag_sign": (
        [("st.cd = 2.0 * Fx / S->chord;", "st.cd = -2.0 * Fx / S->chord;")],
        pins.test_steady_cylinder_drag_re40, ()),
    "drag_half": (
        [("st.cd = 2.0 * Fx / S->chord;", "st.cd = Fx / S->chord;")],
        pins.test_steady_cylinder_drag_re40, ()),
    "lift_coefficient_half": (
        [("st.cl = 2.0 * Fy / S->chord;", "st.cl = Fy / S->chord;")],
        pins.test_plunging_circle_feels_added_mass_force, ()),
    "sor_step_reversed": (
        [("fma(omega, gs - phi[id], phi[id])", "fma(omega, phi[id] - gs, phi[id])")],
        pins.test_poisson_sor_matches_dense_solve, (7, 5, False)),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_its_pin(name):
    replacements, pin, args = MUTANTS[name]
    path = oracle.build_variant(name, replacements)
    with oracle.use_library(path):
        with pytest.raises((AssertionError, ValueError, FloatingPointError)):
            pin(*args)


def unique_pins():
    """The distinct (pin, arguments) pairs of the table, in table order."""
    seen = []
    for _, pin, args in MUTANTS.values():
        if (pin, args) not in seen:
            seen.append((pin, args))
    return seen


def test_unchanged_oracle_passes_the_same_pins():
    # the pins used above hold for the oracle as written
    for pin, args in unique_pins():
        pin(*args)


# The U-Net oracle (numpy) is pinned by central finite differences of its
# loss; a slip in any backward rule must break that pin.
import numpy as np  # noqa: E402

from oracle import unet_oracle as U  # noqa: E402
import test_unet  # noqa: E402


def _conv_backward_flipped_taps(x, W, gy):
    gx, gW, gb = _REAL_CONV_BACKWARD(x, W[:, ::-1, :], gy)
    return gx, gW, gb


def _conv_backward_no_bias(x, W, gy):
    gx, gW, gb = _REAL_CONV_BACKWARD(x, W, gy)
    return gx, gW, 0.0 * gb


_REAL_CONV_BACKWARD = U.conv_backward
UNET_MUTANTS = {
    "pool_backward_unscaled": ("pool_backward", lambda g: np.repeat(np.repeat(g, 2, axis=0), 2, axis=1)),
    "up_backward_one_child": ("up_backward", lambda g: g[0::2, 0::2] * 4.0),
    "conv_backward_flipped_taps": ("conv_backward", _conv_backward_flipped_taps),
    "conv_backward_no_bias": ("conv_backward", _conv_backward_no_bias),
}


@pytest.mark.parametrize("name", sorted(UNET_MUTANTS))
def test_planted_unet_backward_mistake_fails_finite_differences(name, monkeypatch):
    attr, fn = UNET_MUTANTS[name]
    monkeypatch.setattr(U, attr, fn)
    with pytest.raises(AssertionError):
        test_unet.test_oracle_gradient_matches_finite_differences()


_REAL_CONV = U.conv
UNET_FORWARD_MUTANTS = {
    "conv_forward_flipped_taps": ("conv", lambda x, W, b: _REAL_CONV(x, W[:, ::-1, :], b)),
    "pool_forward_two_children": ("pool", lambda x: 0.5 * (x[0::2, 0::2] + x[1::2, 1::2])),
}


@pytest.mark.parametrize("name", sorted(UNET_FORWARD_MUTANTS))
def test_planted_unet_forward_mistake_fails_the_torch_reference(name, monkeypatch):
    attr, fn = UNET_FORWARD_MUTANTS[name]
    monkeypatch.setattr(U, attr, fn)
    with pytest.raises(AssertionError):
        test_unet.test_oracle_forward_matches_torch_cpu_reference()
