"""Host sanitizers on the FP64 oracle: it is built with AddressSanitizer and
UndefinedBehaviorSanitizer and run in a subprocess on a small problem that
takes every path (UPML on all faces, a PEC box, current and resistive
voltage sources, probes, the running DFT, energy, div B and field output).
Any sanitizer report fails the test.  Skipped where gcc's sanitizer runtimes
are not installed."""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _runtime(name):
    try:
        path = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True,
                              check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_oracle_under_asan_and_ubsan(tmp_path):
    asan = _runtime("libasan.so")
    if asan is None or _runtime("libubsan.so") is None:
        pytest.skip("gcc sanitizer runtimes not installed")
    lib = tmp_path / "liboracle_san.so"
    subprocess.run(["gcc", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                    "-fno-sanitize-recover=undefined", "-fopenmp", "-shared", "-fPIC", "-o", str(lib),
                    os.path.join(ROOT, "oracle", "fdtd_oracle.c"), "-lm"], check=True)
    script = textwrap.dedent(f"""
        import sys
        sys.path.insert(0, {ROOT!r})
        import numpy as np
        import oracle
        from paper_1008_2602_gb300 import workloads as W
        oracle.build = lambda force=False: {str(lib)!r}
        p = W.random_problem(3, 17, 13, 11, upml=3, n_steps=40)
        p = W.add_voltage_sources(p, [(7, 6, 5, 2)], V0=5.0, Rs=10.0)
        r = oracle.run(p, energy=True, divb=True, fields=True, vsrc_current=True, n_threads=2)
        assert np.isfinite(r["trace"]).all() and np.isfinite(r["fields"]).all()
        q = W.random_problem(4, 9, 8, 7, upml=0, n_steps=20).replace(upml_depth=(0,) * 6,
                                                                     walls=(W.WALL_PMC,) * 6)
        oracle.run(q, fields=True, n_threads=1)
        print("sanitized oracle ok")
    """)
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, env=env, timeout=600)
    report = r.stdout + r.stderr
    assert r.returncode == 0, report[-3000:]
    assert "sanitized oracle ok" in r.stdout
    assert "AddressSanitizer" not in report and "runtime error" not in report, report[-3000:]
