"""Plant plausible mistakes in a copy of the oracle and check that the pins catch each.

Each mutant is the oracle source with one textual change (a dropped 1/2, a sign
in Eq. 16, a wrong velocity component in Eq. 17, a wrong bounce-back direction,
a wrong lattice weight, streaming against e_a), compiled to a temporary library
and run against a fast subset of ``test_oracle_pins.py`` in a subprocess. The
subset must FAIL for every mutant. Mistakes are only ever planted on the CPU,
in the oracle.
"""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.c")

FAST_PINS = ("lattice_moments or eq19 or transient_closed_form or mass_conservation or "
             "magic_tau or hydrostatic or uniform_patch or symmetries or (table1 and 10-) or flux_conservation")

MUTANTS = {
    "force_half_dropped": [("0.5 * dt * p->eps * rho * Gx) / denom", "1.0 * dt * p->eps * rho * Gx) / denom"),
                           ("0.5 * dt * p->eps * rho * Gy) / denom", "1.0 * dt * p->eps * rho * Gy) / denom")],
    "eq16_sign": [("(1.0 - 2.0 * tau) * jx / rho", "(1.0 + 2.0 * tau) * jx / rho"),
                  ("(1.0 - 2.0 * tau) * jy / rho", "(1.0 + 2.0 * tau) * jy / rho")],
    "eq17_wrong_component": [("keff[0] = nu / gconst * ubar[0];", "keff[0] = nu / gconst * ubar[1];")],
    "bounce_back_same_direction": [("fnew[c * Q + OPP[a]] = fpost;", "fnew[c * Q + a] = fpost;")],
    "diagonal_weight": [("W[a] = 1.0 / 36.0;", "W[a] = 1.0 / 18.0;")],
    "stream_against_e": [("int xd = x + E[a][0];", "int xd = x - E[a][0];"),
                         ("int yd = y + E[a][1];", "int yd = y - E[a][1];")],
    "drag_factor_two": [("(1.0 + p->eps * dt * p->nu / (2.0 * kap))", "(1.0 + p->eps * dt * p->nu / kap)")],
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    src = open(SRC).read()
    for old, new in MUTANTS[name]:
        assert old in src, f"mutation anchor not found: {old!r}"
        src = src.replace(old, new)
    c = tmp_path / "mutant.c"
    c.write_text(src)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"])
    env = dict(os.environ, LBM_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-k", FAST_PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert "passed" in r.stdout or "failed" in r.stdout, r.stdout + r.stderr
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"


def test_unmutated_copy_passes(tmp_path):
    """The same harness with no mutation passes (so failures above come from the mutations)."""
    so = tmp_path / "libsame.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(so), SRC, "-lm"])
    env = dict(os.environ, LBM_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-k", FAST_PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:]
