"""The double-float Matern evaluation of the mixed precisions
(csrc/matern_df.cuh) on the CPU: the header's device functions are compiled
for the host with stand-ins for the CUDA intrinsics (tests/df_host) and
checked against long double on split coordinates.  TwoSum and the fused
product are exact; the closed forms nu = 1/2, 3/2, 5/2 stay within 1e-13 of
theta1 (the same bar as the generator's elementwise GPU tests), and within
3e-14 relative for x < 1.  Needs a host C++ compiler with an 80-bit or wider
long double (x86-64, aarch64)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.join(ROOT, "tests", "df_host")
CSRC = os.path.join(ROOT, "paper_1708_02835_gb300", "csrc")


def _run():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        # matern_df.cuh includes <cuda_runtime.h> and "matern.cuh" (from its own
        # directory): compile a copy next to the host stand-ins instead
        os.makedirs(os.path.join(d, "inc"))
        with open(os.path.join(d, "inc", "cuda_runtime.h"), "w") as f:
            f.write('#include "cuda_shim.h"\n')
        shutil.copy(os.path.join(CSRC, "matern_df.cuh"), os.path.join(d, "inc", "matern_df.cuh"))
        shutil.copy(os.path.join(HERE, "matern.cuh"), os.path.join(d, "inc", "matern.cuh"))
        exe = os.path.join(d, "check_df")
        cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(d, "inc"), "-I", HERE, "-I", CSRC,
               os.path.join(HERE, "check_df.cpp"), "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-3000:]
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120).stdout.strip()
    return dict(kv.split("=") for kv in out.split())


def test_double_float_matern_on_the_host():
    import numpy as np
    if np.finfo(np.longdouble).eps >= 2.0 ** -60:
        pytest.skip("long double is not wider than 60 bits here")
    v = _run()
    assert int(v["bad_sum"]) == 0 and int(v["bad_prod"]) == 0
    for k in ("abs1", "abs2", "abs3"):
        assert float(v[k]) <= 1e-13, v
    for k in ("rel1", "rel2", "rel3"):
        assert float(v[k]) <= 3e-14, v
