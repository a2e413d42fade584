"""The oracle and the host-side arithmetic checks under AddressSanitizer and
UndefinedBehaviorSanitizer (on the CPU): out-of-bounds reads or writes, use
of freed memory, signed overflow, shifts out of range or misaligned accesses
abort the run.  The oracle walks small random substrates with every option
(the three interactions, absorbing membranes, spin concentrations, Baxter's
rule, dead labels, walls, several shapes, relaxation modes) and its results
equal those of the regular build bit for bit."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import os, sys
import numpy as np
sys.path.insert(0, os.environ["ROOT"])
sys.path.insert(0, os.path.join(os.environ["ROOT"], "tests"))
from conftest import make_workload
import oracle
out = []
for seed in range(9):
    rng = np.random.default_rng(100 + seed)
    lab = rng.integers(0, 4, size=(5, 6, 7))
    n = 60
    G = rng.normal(size=(1 + seed % 3, n)) * (rng.uniform(size=(1 + seed % 3, n)) < 0.4)
    mode = rng.integers(0, 3, size=n).astype(np.uint8) if seed % 2 else None
    wl = make_workload(lab, voxel_um=0.2, D=rng.uniform(0.8, 2.5, 4), kappa=rng.uniform(0.0, 0.6, (4, 4)),
                       T2=rng.uniform(30, 90, 4), T1=rng.uniform(300, 900, 4), dt=1e-3, n_steps=n, G=G,
                       mode=mode, dirs=rng.normal(size=(3, 3)), b=np.array([0.0, 0.7]),
                       rec_steps=np.array([20, n]), n_walkers=300, seed=seed + 1,
                       periodic=(1, seed % 2, 1), dead=[0, 0, 0, 1] if seed % 3 == 0 else None,
                       interaction=seed % 3, rho=0.3 if seed % 4 == 1 else None,
                       conc=rng.uniform(0.5, 1.5, 4) if seed % 4 == 2 else None,
                       perm_model=1 if seed % 4 == 3 else 0)
    r = oracle.run(wl, 0, wl.n_walkers, n_threads=2)
    S, asum = oracle.readout(r, wl)
    out.append(np.concatenate([r["o"].ravel(), r["A"].ravel(), np.asarray(S).view(np.float64).ravel(), [asum]]))
np.save(os.environ["OUT"], np.concatenate(out))
print("ok")
"""


def _run(tmp_path, sanitize):
    env = dict(os.environ, ROOT=ROOT, OUT=str(tmp_path / ("san.npy" if sanitize else "ref.npy")))
    if sanitize:
        asan = subprocess.check_output(["gcc", "-print-file-name=libasan.so"], text=True).strip()
        if not os.path.isabs(asan):
            pytest.skip("no AddressSanitizer runtime")
        env.update(RMS_ORACLE_SANITIZE="1", LD_PRELOAD=asan,
                   ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
                   UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-3000:]


def test_oracle_under_sanitizers(tmp_path):
    import numpy as np
    _run(tmp_path, sanitize=False)
    _run(tmp_path, sanitize=True)
    np.testing.assert_array_equal(np.load(tmp_path / "san.npy"), np.load(tmp_path / "ref.npy"))


def test_soft_fp64_check_under_ubsan(tmp_path):
    exe = tmp_path / "soft_fp64_check_ubsan"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                           "-fsanitize=undefined", "-fno-sanitize-recover=all",
                           os.path.join(ROOT, "tests", "soft_fp64_check.cpp"), "-o", str(exe)])
    out = subprocess.run([str(exe), "100000", "3"], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
