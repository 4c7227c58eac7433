"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a temporary copy of the oracle's C source (a
wrong sign, a wrong index, a dropped term, a transposed operand, a wrong
factor in an integrator or a diagnostic), compiles it, and runs the pin tests
of test_oracle_pins.py against that copy: at least one pin must fail.
Everything here runs on the CPU.
"""
import os

import pytest

import oracle as _oracle_mod
from oracle import build as _obuild
from tests import test_oracle_pins as pins

MUTANTS = {
    "acc_sign_x": ("nsum_add(&ax, -gm * dx / w);", "nsum_add(&ax, gm * dx / w);"),
    "mass_i_not_j": ("double gm = G * mass[j];", "double gm = G * mass[i];"),
    "eps_not_squared": ("double soft2 = d2 + eps2;", "double soft2 = d2 + eps;"),
    "dropped_dz2": ("double d2 = dx * dx + dy * dy + dz * dz;", "double d2 = dx * dx + dy * dy;"),
    "self_pair_kept": ("if (j == i) continue;", "if (j == i && eps == 0) continue;"),
    "cube_dropped": ("double w = soft2 * soft;", "double w = soft2;"),
    "transposed_dy": ("double dy = yi - pos[3 * j + 1];", "double dy = pos[3 * j + 1] - yi;"),
    "index_z_from_y": ("double dz = zi - pos[3 * j + 2];", "double dz = zi - pos[3 * j + 1];"),
    "pot_sign": ("nsum_add(&p, -gm / soft);", "nsum_add(&p, gm / soft);"),
    "smag_d2_not_distance": ("nsum_add(&s, gm * sqrt(d2) / w);", "nsum_add(&s, gm * d2 / w);"),
    "smag_soft_not_distance": ("nsum_add(&s, gm * sqrt(d2) / w);", "nsum_add(&s, gm * soft / w);"),
    "kdk_drift_first_order": ("pos[k] = pos[k] + (dt / 2) * (vt[k] + vel[k]);", "pos[k] = pos[k] + dt * vel[k];"),
    "kdk_corrector_no_average": ("vel[k] = (vel[k] + vt[k]) / 2 + (dt / 2) * acc[k];", "vel[k] = vt[k] + (dt / 2) * acc[k];"),
    "kdk_predictor_half": ("vt[k] = vel[k] + dt * acc[k];", "vt[k] = vel[k] + (dt / 2) * acc[k];"),
    "rk4_weight": ("pos[k] = pos[k] + (dt / 6) * (vel[k] + 2 * v2[k] + 2 * v3[k] + v4[k]);",
                   "pos[k] = pos[k] + (dt / 6) * (vel[k] + 2 * v2[k] + v3[k] + 2 * v4[k]);"),
    "rk4_stage3_from_stage1": ("rs[k] = pos[k] + dt * v3[k];", "rs[k] = pos[k] + dt * v2[k];"),
    "fr4_asymmetric": ("const double w[3] = {FR4_W1, FR4_W0, FR4_W1};",
                       "const double w[3] = {FR4_W0, FR4_W1, FR4_W1};"),
    "fr4_w0_one_minus_w1": ("#define FR4_W0 -0x1.b3d16dd72c671p+0", "#define FR4_W0 (1 - FR4_W1)"),
    "fr4_weights_dropped": ("oracle_kdk(n, pos, vel, mass, eps, G, w[s] * dt, 1, acc, p, nthreads)",
                            "oracle_kdk(n, pos, vel, mass, eps, G, dt, 1, acc, p, nthreads)"),
    "diag_W_sign": ("nsum_add(&W, m * pot[i] / 2);", "nsum_add(&W, -m * pot[i] / 2);"),
    "diag_W_not_halved": ("nsum_add(&W, m * pot[i] / 2);", "nsum_add(&W, m * pot[i]);"),
    "diag_Lz_transposed": ("nsum_add(&L[2], m * (r[0] * v[1] - r[1] * v[0]));",
                           "nsum_add(&L[2], m * (r[1] * v[0] - r[0] * v[1]));"),
    "diag_K_no_half": ("v[1] * v[1] + v[2] * v[2]) / 2);", "v[1] * v[1] + v[2] * v[2]));"),
}

# (pin function, kwargs); all are run against each mutant
PINS = [
    (pins.test_point_mass_and_test_particles, {"eps": 0.1}),
    (pins.test_point_mass_and_test_particles, {"eps": 0.0}),
    (pins.test_octahedron_closed_form, {"eps": 0.05}),
    (pins.test_tetrahedron_centre_is_force_free, {}),
    (pins.test_brute_force_40_digits, {"n": 7, "eps": 0.01}),
    (pins.test_newtons_third_law, {}),
    (pins.test_kdk_second_order_on_kepler_orbits, {"e": 0.5}),
    (pins.test_kdk_energy_bounded_and_second_order, {}),
    (pins.test_kdk_time_reversible, {}),
    (pins.test_rk4_fourth_order_on_kepler_orbit, {}),
    (pins.test_fr4_fourth_order_on_kepler_orbit, {}),
    (pins.test_fr4_time_reversible, {}),
    (pins.test_diag_two_body_circular, {}),
    (pins.test_diag_three_bodies_by_hand, {}),
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(_obuild.SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    msrc = tmp_path / "mutant.c"
    msrc.write_text(src.replace(old, new))
    lib = _obuild.build(force=True, src=str(msrc), lib=str(tmp_path / "libmutant.so"))
    mut = _oracle_mod.Oracle(lib)
    caught = []
    for fn, kw in PINS:
        try:
            fn(mut, **kw)
        except (AssertionError, ValueError, FloatingPointError):
            caught.append(fn.__name__)
    assert caught, f"no pin caught mutant {name}"


def test_unmutated_copy_passes_every_pin(tmp_path):
    lib = _obuild.build(force=True, src=_obuild.SRC, lib=str(tmp_path / "libcopy.so"))
    ok = _oracle_mod.Oracle(lib)
    for fn, kw in PINS:
        fn(ok, **kw)
    assert os.path.exists(lib)
