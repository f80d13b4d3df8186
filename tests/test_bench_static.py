"""bench.py on the CPU: every global name a function uses is defined, and the argument parser loads."""
import builtins
import os
import subprocess
import symtable
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BENCH = os.path.join(ROOT, "bench.py")


def _undefined_globals(src: str, filename: str):
    top = symtable.symtable(src, filename, "exec")
    module_names = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
    missing = set()

    def walk(t):
        for s in t.get_symbols():
            if s.is_referenced() and s.is_global() and not s.is_assigned():
                n = s.get_name()
                if n not in module_names and n not in ("__file__", "__name__") and not hasattr(builtins, n):
                    missing.add((t.get_name(), n))
        for c in t.get_children():
            walk(c)

    walk(top)
    return sorted(missing)


def test_bench_functions_use_only_defined_globals():
    src = open(BENCH).read()
    assert _undefined_globals(src, BENCH) == []


def test_bench_help_runs():
    r = subprocess.run([sys.executable, BENCH, "--help"], capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert "--pipeline" in r.stdout and "--impl" in r.stdout
