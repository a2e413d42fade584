"""The plain FP64 form's products, divisions and square root run on the
integer ALU (paper_2012_06478_gb300/csrc/soft_fp64.cuh); they must give the
IEEE round-to-nearest-even result bit for bit.  The same source, compiled for
the host, is compared with the host's IEEE operations over every normal
exponent, the walker step's operand ranges, values within one unit of a
rounding midpoint (products with exact ties), powers of two and extreme
mantissas, and perfect squares; the operands it hands back to the hardware
are checked to be exactly the ones outside its range."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_soft_division_and_sqrt_are_ieee(tmp_path):
    exe = tmp_path / "soft_fp64_check"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                           os.path.join(ROOT, "tests", "soft_fp64_check.cpp"), "-o", str(exe)])
    for seed in (1, 2):
        out = subprocess.run([str(exe), "400000", str(seed)], capture_output=True, text=True)
        assert out.returncode == 0, out.stdout
        f = out.stdout.split()
        assert f[0] == "tested" and int(f[1]) > 5_000_000 and int(f[3]) == 0 and f[-1] == "1", out.stdout
