"""The pins catch plausible mistakes: each case plants one mistake in a copy of the C
oracle (compiled here with gcc, CPU only), points the oracle package at the mutant for
the duration of the test, and checks that the pin written for that part of the method
fails on it (and that the same pin passes on the real oracle)."""
import os
import shutil
import subprocess

import pytest

import oracle
import test_oracle_adv as ADV
import test_oracle_conventions as CONV
import test_oracle_eos as EOS
import test_oracle_opacity as OPA

HERE = os.path.dirname(os.path.abspath(oracle.__file__))

MUTANTS = {
    # Eq. adv: upwind cell taken from the wrong side
    "upwind_flipped": ("int in = lower ? f[t] > 0.0 : f[t] < 0.0;",
                       "int in = lower ? f[t] < 0.0 : f[t] > 0.0;",
                       lambda orc: ADV.test_upwind_closed_form_1d(orc, 1.0)),
    # phi_11: S_adv added without its dt in the reduced right-hand side
    "source_without_dt": ("double Eadv = P->E[k] + (P->S_adv ? P->S_adv[k] : 0.0) * P->dt;",
                          "double Eadv = P->E[k] + (P->S_adv ? P->S_adv[k] : 0.0);",
                          ADV.test_source_enters_phi11_times_dt),
    # non-linear C_V: the secant u / T instead of the table's slope du/dT
    "cv_secant": ("W->CV[k] = rho * slope;",
                  "W->CV[k] = rho * u / W->T[k];",
                  EOS.test_tangent_cv_keeps_the_state_on_the_table),
    # opacity power law: exponents of rho and T swapped
    "opacity_exponents_swapped": ("return k[0] + k[1] * pow(rho, k[2]) * pow(T, k[3]);",
                                  "return k[0] + k[1] * pow(rho, k[3]) * pow(T, k[2]);",
                                  OPA.test_rosseland_law_per_cell_states),
    # opacity power law: the constant term dropped
    "opacity_k0_dropped": ("return k[0] + k[1] * pow(rho, k[2]) * pow(T, k[3]);",
                           "return k[1] * pow(rho, k[2]) * pow(T, k[3]);",
                           OPA.test_rosseland_law_in_the_face_coefficient),
    # Rosseland opacity taken at the radiation temperature (E / a)^(1/4) instead of T_g^n
    "opacity_at_radiation_temperature": (
        "double kR = opacity(P->kR, rho, W->T[k]);",
        "double kR = opacity(P->kR, rho, sqrt(sqrt(P->E[k] / orc_const_aR())));",
        OPA.test_rosseland_law_in_the_face_coefficient),
    # Planck opacity taken at the radiation temperature: caught by the exchange closed form
    "planck_at_radiation_temperature": (
        "double kP = opacity(P->kP, rho, W->T[k]);",
        "double kP = opacity(P->kP, rho, sqrt(sqrt(P->E[k] / orc_const_aR())));",
        OPA.test_planck_law_in_the_exchange_closed_form),
    # Rosseland and Planck laws exchanged in the diffusion coefficient
    "sigma_from_planck": ("W->sig[k] = kR * rho;",
                          "W->sig[k] = kP * rho;",
                          OPA.test_rosseland_law_in_the_face_coefficient),
    # Planck law replaced by the Rosseland one in the exchange
    "beta_from_rosseland": ("W->betaP[k] = kP * rho * c * P->dt;",
                            "W->betaP[k] = kR * rho * c * P->dt;",
                            OPA.test_planck_law_in_the_exchange_closed_form),
    # face interpolation weights the wrong way round (sigma, E taken at the mirrored point)
    "face_interpolation_mirrored": ("double th = (P->xf[i] - xk) / d;",
                                    "double th = (xm - P->xf[i]) / d;",
                                    CONV.test_face_values_interpolate_linear_fields_exactly_cartesian),
    # theta distance without the radius (d = dtheta_c instead of r_c dtheta_c)
    "theta_distance_without_r": ("double d = metric * (ym - yk);",
                                 "double d = (ym - yk);",
                                 CONV.test_spherical_face_fluxes_converge_at_second_order),
    # theta distance at the inner face radius instead of the volume centroid's
    "theta_distance_inner_radius": ("double d = metric * (ym - yk);",
                                    "double d = (P->coord == 1 ? P->xf[i] : 1.0) * (ym - yk);",
                                    CONV.test_spherical_face_fluxes_converge_at_second_order),
    # Milne ghost: the full cell width instead of the half-cell distance to the face
    "milne_full_cell": ("double h = fabs(P->xf[i] - W->xc[ic]);",
                        "double h = 2.0 * fabs(P->xf[i] - W->xc[ic]);",
                        CONV.test_milne_eigenmode_decays_as_the_continuum_one),
    # Milne ghost: 1/(3 sigma) in place of the 2/(3 sigma) of Eq. milne (x sides)
    "milne_factor": ("double kk = 2.0 / (3.0 * s * h);\n                double D = c * orc_limiter(P->limiter, 1.5) / s;\n"
                     "                W->Rx[f] = 1.5;",
                     "double kk = 1.0 / (3.0 * s * h);\n                double D = c * orc_limiter(P->limiter, 1.5) / s;\n"
                     "                W->Rx[f] = 1.5;",
                     CONV.test_milne_eigenmode_decays_as_the_continuum_one),
}


def _build_mutant(tmp, find, repl):
    src = open(os.path.join(HERE, "gq_oracle.c")).read()
    assert src.count(find) == 1, find
    shutil.copy(os.path.join(HERE, "gq_oracle.h"), tmp / "gq_oracle.h")
    (tmp / "gq_oracle.c").write_text(src.replace(find, repl))
    lib = tmp / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared", "-o",
                    str(lib), str(tmp / "gq_oracle.c"), "-lm"], check=True, capture_output=True, text=True)
    return str(lib)


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pin_rejects_planted_mistake(name, tmp_path, monkeypatch, orc):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    find, repl, pin = MUTANTS[name]
    pin(orc)                                   # the real oracle passes the pin
    path = _build_mutant(tmp_path, find, repl)
    monkeypatch.setattr(oracle._build, "build", lambda force=False: path)
    monkeypatch.setattr(oracle, "_lib", None)
    with pytest.raises(AssertionError):
        pin(oracle)
