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
import test_oracle_eos as EOS

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
