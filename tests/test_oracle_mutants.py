"""Plant plausible mistakes in a copy of the oracle and check that the pins catch each.

Each mutant is the oracle source with one textual change (a dropped 1/2, a sign
in Eq. 16, a wrong velocity component in Eq. 17, a wrong bounce-back direction,
a wrong lattice weight, streaming against e_a), compiled to a temporary library
and run against a fast subset of ``test_oracle_pins.py`` in a subprocess (the
D3Q19 mutants against ``test_oracle3d_pins.py``). The
subset must FAIL for every mutant. Mistakes are only ever planted on the CPU,
in the oracle.
"""

import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.c")
SRC3 = os.path.join(ROOT, "oracle", "lbm3d_oracle.c")

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


# mistakes caught by one slower pin, named beside each
TARGETED = {
    # the Darcy-started local problem stopped on the driven mean velocity component alone
    "warm_stop_driven_only": ([("sqrt(dx * dx + dy * dy) <= tol * check_every * sqrt(m[0] * m[0] + m[1] * m[1])",
                                "fabs(m[d] - prev[d]) <= tol * check_every * fabs(m[d])")],
                              "whole_velocity_vector"),
    # the local-global ring emitting the equilibrium at rho u, without the half force of Eq. 6
    "lg_ring_without_half_force": ([("jpx = rb * fx[2] + 0.5 * rb * (p->eps * Gx - drag * fx[2]);", "jpx = rb * fx[2];"),
                                    ("jpy = rb * fx[3] + 0.5 * rb * (p->eps * Gy - drag * fx[3]);", "jpy = rb * fx[3];")],
                                   "local_global"),
    # the pressure term of the mean force with the wrong sign
    "lg_pressure_term_sign": ([("const double f11 = gconst - win[2] / (3.0 * eps), f21 = -win[3] / (3.0 * eps);",
                                "const double f11 = gconst + win[2] / (3.0 * eps), f21 = win[3] / (3.0 * eps);"),
                               ("const double f12 = -win[6] / (3.0 * eps), f22 = gconst - win[7] / (3.0 * eps);",
                                "const double f12 = win[6] / (3.0 * eps), f22 = gconst + win[7] / (3.0 * eps);")],
                              "local_global"),
    # the pressure-only ring refreshed from the ring cell itself instead of its inward neighbour
    "lg_ring_velocity_from_itself": ([("const long ci = (long)yi * se + xi;", "const long ci = c; (void)xi; (void)yi;")],
                                     "local_global"),
    # the pressure-only ring never refreshed
    "lg_ring_never_refreshed": ([("                    apply_at = st + 2;", "                    apply_at = -1;")],
                                "local_global"),
    # the window's density gradient by a one-sided difference
    "lg_gradient_not_halved": ([("sx += 0.5 * (r[0] - r[1]);", "sx += (r[0] - r[1]);"),
                                ("sy += 0.5 * (r[2] - r[3]);", "sy += (r[2] - r[3]);")],
                               "local_global"),
}


# mistakes in the D3Q19 oracle, run against its own pins
MUTANTS3 = {
    "d3q19_edge_weight": [("(shell == 1 ? 1.0 / 18.0 : 1.0 / 36.0)", "(shell == 1 ? 1.0 / 18.0 : 1.0 / 18.0)")],
    "d3q19_stream_against_e": [("const int xd = (x + E3[a][0] + nx) % nx, yd = (y + E3[a][1] + ny) % ny,",
                                "const int xd = (x - E3[a][0] + nx) % nx, yd = (y - E3[a][1] + ny) % ny,")],
    "d3q19_eq16_sign": [("(1.0 - 2.0 * tau) * j[k] / rho", "(1.0 + 2.0 * tau) * j[k] / rho")],
    "d3q19_force_half_dropped": [("j[k] + 0.5 * p->eps * rho * G[k]", "j[k] + 1.0 * p->eps * rho * G[k]")],
    "d3q19_local_drive_axes": [("        p.gy = d == 1 ? gconst : 0.0;\n        p.gz = d == 2 ? gconst : 0.0;",
                                "        p.gy = d == 2 ? gconst : 0.0;\n        p.gz = d == 1 ? gconst : 0.0;")],
    # Eq. 18 applied transposed: rho u = B^-T r instead of B^-1 r
    "d3q19_tensor_transposed": [("u[i] = (Bi[3 * i] * r[0] + Bi[3 * i + 1] * r[1] + Bi[3 * i + 2] * r[2]) / rho;",
                                 "u[i] = (Bi[i] * r[0] + Bi[3 + i] * r[1] + Bi[6 + i] * r[2]) / rho;")],
    # oversampling with the mean over the grown cube's corner instead of the inner leaf
    "d3q19_oversampled_window_origin": [("orc3_mean_velocity_window(&p, f, margin, margin, margin, s, m);\n                if",
                                         "orc3_mean_velocity_window(&p, f, 0, 0, 0, s, m);\n                if"),
                                        ("        orc3_mean_velocity_window(&p, f, margin, margin, margin, s, m);\n        for",
                                         "        orc3_mean_velocity_window(&p, f, 0, 0, 0, s, m);\n        for")],
    # Eq. 18 with the drag term's factor 1/2 dropped: (I + eps nu K*^-1) rho u = r
    "d3q19_tensor_drag_half": [("const double h = 0.5 * p->eps * p->nu;\n        for (int i = 0; i < 3; ++i)",
                                "const double h = 1.0 * p->eps * p->nu;\n        for (int i = 0; i < 3; ++i)")],
}


def _build(tmp_path, src2, src3, name):
    c2, c3 = tmp_path / f"{name}.c", tmp_path / f"{name}3d.c"
    c2.write_text(src2)
    c3.write_text(src3)
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(c2), str(c3), "-lm"])
    return so


def _pins(so, pins_file, expr, stop_first=True):
    env = dict(os.environ, LBM_ORACLE_LIB=str(so))
    args = [sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", os.path.join(ROOT, "tests", pins_file)]
    if stop_first:
        args.insert(4, "-x")
    if expr:
        args += ["-k", expr]
    return subprocess.run(args, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def _mutate(src, changes):
    for old, new in changes:
        assert old in src, f"mutation anchor not found: {old!r}"
        src = src.replace(old, new)
    return src


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    so = _build(tmp_path, _mutate(open(SRC).read(), MUTANTS[name]), open(SRC3).read(), "mutant")
    r = _pins(so, "test_oracle_pins.py", FAST_PINS)
    assert "passed" in r.stdout or "failed" in r.stdout, r.stdout + r.stderr
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name", sorted(TARGETED))
def test_targeted_pin_catches_mutant(name, tmp_path):
    changes, expr = TARGETED[name]
    so = _build(tmp_path, _mutate(open(SRC).read(), changes), open(SRC3).read(), "mutant")
    r = _pins(so, "test_oracle_pins.py", expr)
    assert "passed" in r.stdout or "failed" in r.stdout, r.stdout + r.stderr
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name", sorted(MUTANTS3))
def test_3d_pins_catch_mutant(name, tmp_path):
    so = _build(tmp_path, open(SRC).read(), _mutate(open(SRC3).read(), MUTANTS3[name]), "mutant")
    r = _pins(so, "test_oracle3d_pins.py", None)
    assert "passed" in r.stdout or "failed" in r.stdout, r.stdout + r.stderr
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"


def test_unmutated_copy_passes(tmp_path):
    """The same harness with no mutation passes (so failures above come from the mutations)."""
    so = _build(tmp_path, open(SRC).read(), open(SRC3).read(), "same")
    r = _pins(so, "test_oracle_pins.py", FAST_PINS, stop_first=False)
    assert r.returncode == 0, r.stdout[-3000:]
    r = _pins(so, "test_oracle3d_pins.py", None, stop_first=False)
    assert r.returncode == 0, r.stdout[-3000:]


# ---------------------------------------------------- the surrogate oracle's base and gate
SUR_SRC = os.path.join(ROOT, "oracle", "surrogate.py")
SUR_MUTANTS = {
    "bounds_axis_of_y_tubes": [("h_cols = 1.0 / np.mean(1.0 / k, axis=0)", "h_cols = 1.0 / np.mean(1.0 / k, axis=1)")],
    "upper_bound_arithmetic": [("return (np.mean(h_rows), 1.0 / np.mean(1.0 / a_cols),",
                                "return (np.mean(h_rows), np.mean(a_cols),")],
    "width_not_halved": [("wx = 1.0 if mode == 1 else max(0.5 * (hix - lox), 0.05)",
                          "wx = 1.0 if mode == 1 else max(1.0 * (hix - lox), 0.05)")],
    "phase_order_transposed": [("for a in (0, 1) for b in (0, 1)])", "for b in (0, 1) for a in (0, 1)])")],
    "gate_population_std": [("/ (m_members - 1)) if m_members > 1", "/ m_members) if m_members > 1")],
    "gate_bounds_exclusive": [("if not (stat_lo[k] <= stats[i, k] <= stat_hi[k]):",
                               "if not (stat_lo[k] < stats[i, k] < stat_hi[k]):")],
    "darcy_arithmetic_faces": [("faces.append((np.roll(idx, -1, axis=axis).ravel(), (2.0 * k * kn / (k + kn)).ravel(), axis))",
                                "faces.append((np.roll(idx, -1, axis=axis).ravel(), (0.5 * (k + kn)).ravel(), axis))")],
    "darcy_drive_reversed": [("q.append((kf * (p[i] - p[j] + (1.0 if axis == axis_d else 0.0))).reshape(n_y, n_x))",
                              "q.append((kf * (p[j] - p[i] + (1.0 if axis == axis_d else 0.0))).reshape(n_y, n_x))")],
    "gate_mean_of_k_not_log": [("keff[i] = (np.exp(mean[0]), 0.0, 0.0, np.exp(mean[1]))",
                                "keff[i] = (np.exp(y[:, i, 0]).mean(), 0.0, 0.0, np.exp(y[:, i, 1]).mean())")],
}


@pytest.mark.parametrize("name", sorted(SUR_MUTANTS))
def test_surrogate_oracle_pins_catch_planted_mistake(name, monkeypatch):
    import importlib.util
    import test_surrogate_oracle as pins
    src = open(SUR_SRC).read()
    for old, new in SUR_MUTANTS[name]:
        assert old in src, f"mutation anchor not found: {old!r}"
        src = src.replace(old, new)
    spec = importlib.util.spec_from_loader(f"sur_mutant_{name}", loader=None)
    mod = importlib.util.module_from_spec(spec)
    exec(compile(src, f"sur_mutant_{name}", "exec"), mod.__dict__)
    monkeypatch.setattr(pins, "S", mod)
    tests = [getattr(pins, t) for t in dir(pins) if t.startswith("test_")
             and ("phase" in t or "bounds" in t or "base" in t or "gate" in t or "checkerboard" in t
                  or "darcy" in t)]
    failed = 0
    for t in tests:
        try:
            t()
        except (AssertionError, ValueError, IndexError):
            failed += 1
    assert failed > 0, f"no pin caught the planted mistake {name}"


# ---------------------------------------------------- the Python oracle's start states and rules
# Each mutant rewrites one function of oracle/__init__.py (its source, one textual change),
# compiled in the module's own namespace and swapped in for the duration of the pins named
# beside it; at least one of those pins must fail.
PY_MUTANTS = {
    "lg_darcy_drive_sign": ("lg_darcy_state", [("b[pos[a]] -= kf * drive * sgn", "b[pos[a]] += kf * drive * sgn")],
                            "local_global_darcy_start"),
    "lg_darcy_ring_pressure_dropped": ("lg_darcy_state", [("b[pos[a]] += kf * pb[c]", "b[pos[a]] += 0.0 * pb[c]")],
                                       "local_global_darcy_start"),
    "lg_darcy_velocity_one_face": ("lg_darcy_state", [("ux = g_const / nu * 0.5 * (qx[y, x - 1] + qx[y, x])",
                                                       "ux = g_const / nu * qx[y, x]")],
                                   "mirror_symmetry"),
    "coarse_to_fine_weights_swapped": ("coarse_to_fine", [("fx = (X - i0)[None, None, :]", "fx = (Y - j0)[None, None, :]"),
                                                          ("fy = (Y - j0)[None, :, None]", "fy = (X - i0)[None, :, None]")],
                                       "coarse_to_fine"),
    "lg_select_condition_inverted": ("lg_select", [("sv[0] / sv[1] <= cond_max", "sv[0] / sv[1] >= cond_max")],
                                     "selection_rule"),
    "lg_select_unsymmetrised": ("lg_select", [("out[i] = [ks[0, 0], sym, sym, ks[1, 1]] if good else ref[i]",
                                               "out[i] = k[i] if good else ref[i]")],
                                "selection_rule"),
    "darcy_start_velocity_one_face": ("darcy_start", [("ux = 0.5 * (qx + np.roll(qx, 1, axis=1)) * g_const / nu",
                                                       "ux = qx * g_const / nu")],
                                      "mirror_symmetry"),
}


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_python_oracle_pins_catch_planted_mistake(name, monkeypatch):
    import inspect
    import textwrap
    import oracle
    import test_oracle_pins as pins
    fname, changes, expr = PY_MUTANTS[name]
    src = textwrap.dedent(inspect.getsource(getattr(oracle, fname)))
    for old, new in changes:
        assert old in src, f"mutation anchor not found: {old!r}"
        src = src.replace(old, new)
    ns = dict(vars(oracle))
    exec(compile(src, f"mutant_{name}", "exec"), ns)
    monkeypatch.setattr(oracle, fname, ns[fname])
    tests = [getattr(pins, t) for t in dir(pins) if t.startswith("test_") and expr in t]
    assert tests, f"no pin matches {expr!r}"
    failed = 0
    for t in tests:
        try:
            if "ring" in inspect.signature(t).parameters:
                for ring in (1, 2):
                    t(ring)
            else:
                t()
        except (AssertionError, ValueError, IndexError, np.linalg.LinAlgError):
            failed += 1
    assert failed > 0, f"no pin caught the planted mistake {name}"
