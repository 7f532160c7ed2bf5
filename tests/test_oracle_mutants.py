"""Planted mistakes: each test compiles a copy of the oracle with one
plausible error (on the CPU, in a temporary directory) and checks that one of
the pins in test_oracle_pins.py fails for it.  This shows the pins constrain
the part of the method each mistake touches."""
import importlib.util
import os
import subprocess

import pytest

import test_oracle_pins as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dies_oracle.c")

MUTANTS = {
    # Eq. 2: background directions mu = sqrt(u)
    "inject_mu_linear": ("mu = sqrt(u_mu);", "mu = u_mu;", "test_pure_absorber_shells_impact_parameter_quadrature",
                         {"r_in": 0.0}),
    # Eq. 4: tau_S consumed with the absorption coefficient
    "eq4_kappa_typo": ("p.tauS -= ks * l;", "p.tauS -= ka * l;", "test_pure_scatterer_isotropic_field_invariant",
                       {"g": 0.6}),
    # HG inversion with the wrong sign of g
    "hg_sign": ("double mu = (1.0 + g * g - t * t) / (2.0 * g);", "double mu = -(1.0 + g * g - t * t) / (2.0 * g);",
                "test_hg_sampler_moments", {"g": 0.6}),
    # scattering azimuth frozen at 0 (direction pulled toward the radius vector)
    "scatter_no_azimuth": ("dn[i] = mu_s * p->d[i] + st * (cos(phi) * e1[i] + sin(phi) * e2[i]);",
                           "dn[i] = mu_s * p->d[i] + st * e1[i];", "test_pure_scatterer_isotropic_field_invariant",
                           {"g": 0.6}),
    # inward flux of an isotropic field taken as J instead of pi J
    "external_flux_factor": ("L_out[0] = 4.0 * ORC_PI * ORC_PI * R * R * s;", "L_out[0] = 4.0 * ORC_PI * R * R * s;",
                             "test_optically_thin_temperature", {"ffi": 1}),
    # re-emission from the new spectrum instead of the difference spectrum
    "no_difference_spectrum": ("pdiff[k] = bn - Bc[k];", "pdiff[k] = bn;",
                               "test_difference_spectrum_telescopes_to_final_emission", {}),
    # Eq. 5 weight with a wrong exponent
    "kbg_weight_exponent": ("pow(mu, 2.0 - 1.0 / M->k_bg)", "pow(mu, 2.0 - M->k_bg)",
                            "test_weighted_injection_is_unbiased", {"k_bg": 1.0 / 3.0, "ffi": False}),
    # Eq. 12 weight not applied
    "ffi_no_weight": ("    p.w *= q;\n", "\n", "test_weighted_injection_is_unbiased", {"k_bg": 0.5, "ffi": True}),
    # re-emission direction not isotropic
    "reemit_not_isotropic": ("double mu = 2.0 * u_mu - 1.0;",
                             "double mu = u_mu;",
                             "test_absorb_reemit_grey_isotropic_invariant", {}),
    # cell emission normalisation without the 4 pi
    "mass_no_4pi": ("mass[i] = 4.0 * ORC_PI * M->rho[i] * V * Lu2;", "mass[i] = M->rho[i] * V * Lu2;",
                    "test_optically_thin_temperature", {"ffi": 1}),
    # Philox with one Weyl increment wrong
    "philox_key_bump": ("k1 += 0xBB67AE85u;", "k1 += 0xBB67AE84u;", "test_philox_known_answer_vectors", {}),
    # Eq. 7 weight inverted (sampling density over the dust density)
    "scatter_weight_inverted": ("p->w *= orc_hg_pdf2(C->M->g[p->f], mu_s) / orc_hg_pdf2(C->M->g_S, mr);",
                                "p->w *= orc_hg_pdf2(C->M->g_S, mr) / orc_hg_pdf2(C->M->g[p->f], mu_s);",
                                "test_scattering_weighting_conserves_energy_on_average", {"g": 0.6, "g_S": -0.3}),
    # Eq. 6 weight missing
    "reemit_weight_missing": ("    p->w /= orc_hg_pdf2(M->g_E, mr);\n", "\n",
                              "test_reemission_weighting_is_unbiased", {"g_E": 0.5}),
    # Eq. 8 with the exponent's sign flipped
    "path_weight_sign": ("return exp(tau * (k - 1.0)) / k;", "return exp(tau * (1.0 - k)) / k;",
                         "test_weight_functions_have_unit_mean", {}),
    # Eq. 8 weight not applied to the absorption path
    "path_weight_unused": ("  if (kA != 1.0) p->w *= orc_path_weight(kA, p->tauA);\n", "\n",
                           "test_free_path_weighting_is_unbiased", {"kw": {"k_A": 2.5}}),
    # re-emission radius uniform in r instead of in volume
    "remit_radius_linear": ("  return cbrt(a + u * (b - a));", "  return ri + u * (ro - ri);",
                            "test_shell_radius_is_uniform_in_volume", {}),
    # forced interaction of Eqs. 9-12 choosing scattering with probability k_A / k_ext
    "ffi_type_inverted": ("if (u_type * ke < ka) alive = do_absorb(C, &p, &rs, s);",
                          "if (u_type * ke >= ka) alive = do_absorb(C, &p, &rs, s);",
                          "test_forced_interaction_is_unbiased_with_scattering", {"ffi": 1, "albedo": 0.3}),
    # forcing on the absorption depth applied when the ray is scattered
    "ffi_abs_case_flipped": ("if (p.tauS >= tauS0) {", "if (p.tauS < tauS0) {",
                             "test_forced_interaction_is_unbiased_with_scattering", {"ffi": 2, "albedo": 0.5}),
    # forcing on the absorption depth whatever the scattering clock says
    "ffi_abs_scattering_ignored": ("if (p.tauS >= tauS0) {", "if (1) {",
                                   "test_forced_interaction_is_unbiased_with_scattering", {"ffi": 2, "albedo": 0.5}),
    # Eq. 12 weight from the extinction depth while forcing an absorption
    "ffi_abs_weight_extinction": ("double q = -expm1(-tauA0);", "double q = -expm1(-(tauA0 + tauS0));",
                                  "test_forced_interaction_is_unbiased_with_scattering", {"ffi": 2, "albedo": 0.5}),
    # direct-escape part of the absorption forcing not tallied
    "ffi_abs_no_direct_tally": ("      C->sed[p.f] += e_direct;\n      C->st[ST_E_DIRECT] += e_direct;\n"
                                "      C->st[ST_E_ESCAPED] += e_direct;\n", "\n",
                                "test_energy_conservation_ire", {}),
    # reference direction of Eqs. 6-7 with the sign flipped (outwards for the external field)
    "reference_direction_flipped": ("ref[i] = (s == 0) ? -rhat[i] : rhat[i];", "ref[i] = (s == 0) ? rhat[i] : -rhat[i];",
                                    "test_weighting_reference_direction_points_away_from_the_source",
                                    {"external": True}),
    # density-dependent k_A running the wrong way
    "kA_rho_reversed": ("kA[i] = M->kA_hi + (M->kA_lo - M->kA_hi) * (lmax - log(M->rho[i])) / (lmax - lmin);",
                        "kA[i] = M->kA_lo + (M->kA_hi - M->kA_lo) * (lmax - log(M->rho[i])) / (lmax - lmin);",
                        "test_density_dependent_kA_is_log_linear", {}),
}


def _load_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new, 1)
    csrc = tmp_path / f"{name}.c"
    so = tmp_path / f"lib{name}.so"
    csrc.write_text(mutated)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                           str(csrc), "-lm"])
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{name}", os.path.join(ROOT, "oracle", "oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC = str(csrc)
    mod._LIB = str(so)
    mod._lib = None
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pin_catches_planted_mistake(tmp_path, name):
    old, new, pin, kw = MUTANTS[name]
    mod = _load_mutant(tmp_path, name, old, new)
    with pytest.raises(AssertionError):
        getattr(P, pin)(mod, **kw)
