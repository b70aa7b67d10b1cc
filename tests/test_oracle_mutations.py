"""The pins of the pseudo-time step (Section 4.3, Eq. (29)/(30), Algorithm 3)
catch its plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a plain text
substitution in the pseudo-time smoother), builds that copy on the CPU, binds
it in place of the oracle and runs the pins of tests/test_oracle_smoothers.py:
at least one pin must fail.  The names of the pins that fail are printed, so a
run with -s lists which pin catches which mistake."""
import ctypes
import subprocess

import pytest

from oracle import oracle as O

import test_oracle_smoothers as S

# (name, text in m1_oracle.c, replacement)
MUTATIONS = [
    ("explicit half dropped",
     "o.E = s.E + tau * d.E; o.Fx = s.Fx + tau * d.Fx;\n"
     "                o.Fy = s.Fy + tau * d.Fy; o.T = s.T + tau * d.T;",
     "o = s; (void)d; (void)tau;"),
    ("dtau in place of the limited tau_i",
     "double tau = dmin(dtau, theta * tstar);",
     "double tau = dtau; (void)tstar;"),
    ("weights (w0, w1) swapped",
     "jacobi_sweep(g, dt, sa, ss, ut, w, w2, 1.0, dtau)",
     "jacobi_sweep(g, dt, sa, ss, ut, w, w2, dtau, 1.0)"),
    ("limited along the wrong ray (flux components swapped)",
     "ora_max_admissible_step(s.E, s.Fx, s.Fy, s.T, d.E, d.Fx, d.Fy, d.T, g->c);\n"
     "                double tau",
     "ora_max_admissible_step(s.E, s.Fx, s.Fy, s.T, d.E, d.Fy, d.Fx, d.T, g->c);\n"
     "                double tau"),
    ("theta applied to the unlimited step too",
     "double tau = dmin(dtau, theta * tstar);",
     "double tau = theta * dmin(dtau, tstar);"),
    ("implicit half started from u~ instead of u",
     "memcpy(w, u, 4 * n * sizeof(double));\n        for (int s = 0; s < nu; ++s)",
     "memcpy(w, ut, 4 * n * sizeof(double));\n        for (int s = 0; s < nu; ++s)"),
]


def _build_mutant(tmp_path, old, new):
    src = open(O.SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    path = tmp_path / "m1_oracle_mutant.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-shared", "-fPIC", "-o",
                    str(lib), str(path), "-lm"], check=True)
    return O.bind(ctypes.CDLL(str(lib)))


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pseudo_time_pins_catch_mutation(tmp_path, monkeypatch, name, old, new):
    monkeypatch.setattr(O, "_LIB", _build_mutant(tmp_path, old, new))
    caught = []
    for pin in S.PSEUDO_TIME_PINS:
        try:
            pin()
        except AssertionError:
            caught.append(pin.__name__)
    print(f"\n{name}: caught by {caught}")
    assert caught, f"no pin fails when the oracle has this mistake: {name}"
