"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer: the C
oracle's time step and the library's DVM utilities (error paths included),
each built into its own small test binary."""
import os
import shutil
import subprocess

import pytest

from lbm_inputs import DVM_TABLES
from oracle import dvm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-fsanitize=address,undefined", "-fno-omit-frame-pointer", "-fno-sanitize-recover=all",
       "-g", "-O1"]


def _build(tmp_path, compiler, sources, includes, out):
    exe = str(tmp_path / out)
    cmd = [compiler] + SAN + [f"-I{i}" for i in includes] + sources + ["-o", exe, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        if "sanitize" in r.stderr or "asan" in r.stderr.lower():
            pytest.skip("sanitizer runtime not available: " + r.stderr[-200:])
        raise AssertionError(r.stderr)
    return exe


def _run(exe, stdin):
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe], input=stdin, capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr
    return r.stdout.split()


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no gcc")
@pytest.mark.parametrize("name,N,Nx,Ny", [("D2V16", 3, 3, 8), ("D2V33", 4, 5, 4), ("D2V32", 3, 2, 12),
                                         ("D3V107xz", 3, 7, 6)])
@pytest.mark.parametrize("wall_mode,force_a3", [(0, 0), (1, 1)])
def test_oracle_step_under_sanitizers(tmp_path, name, N, Nx, Ny, wall_mode, force_a3):
    """Both readings of the wall and of the N = 4 force term; the transformed
    wall does not conserve mass exactly (a drift of order dt/tau Ma^2)."""
    exe = _build(tmp_path, "gcc", [os.path.join(ROOT, "tests", "sanitize", "oracle_driver.c"),
                                   os.path.join(ROOT, "oracle", "lbm_oracle.c")],
                 [os.path.join(ROOT, "oracle")], "oracle_san")
    e, w, c = dvm.dvm2d(name, DVM_TABLES)
    lines = [f"{len(w)} {c!r} {N} {Nx} {Ny} 0.3 0.002 40 {wall_mode} {force_a3}"]
    lines += [f"{int(a)} {int(b)} {x!r}" for (a, b), x in zip(e.tolist(), w.tolist())]
    dmass, uc = _run(exe, "\n".join(lines) + "\n")
    assert float(dmass) < (1e-13 if wall_mode == 0 else 1e-5) and float(uc) > 0


@pytest.mark.skipif(shutil.which("g++") is None, reason="no g++")
@pytest.mark.parametrize("name", ["D2V16", "D2V33", "D3V107", "D3V96"])
def test_dvm_utilities_under_sanitizers(tmp_path, name):
    exe = _build(tmp_path, "g++", [os.path.join(ROOT, "tests", "sanitize", "dvm_driver.cpp"),
                                   os.path.join(ROOT, "paper_1510_08886_gb300", "csrc", "dvm.cpp")],
                 [os.path.join(ROOT, "include")], "dvm_san")
    t = DVM_TABLES[name]
    lines = [f"{t['D']} {len(t['groups'])} {t['c']!r}"]
    lines += [" ".join(str(v) for v in rep) + f" {vg} {wg!r}" for rep, vg, wg in t["groups"]]
    V, Vq, Q, rc_cap, rc_null = (int(x) for x in _run(exe, "\n".join(lines) + "\n"))
    assert V == t["V"]
    assert Q == t["Q"]
    assert rc_cap == -1 and rc_null == -1
    if t["D"] == 3:
        assert Vq == len(dvm.dvm2d(name + "xz", DVM_TABLES)[1])
