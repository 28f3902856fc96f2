"""A plain C99 program compiles against include/mlmc.h, links the library and
runs its host-only entry points (no GPU): the boundary is usable from C."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "mlmc.h"

int main(void) {
  mlmc_params p;
  mlmc_format f;
  memset(&p, 0, sizeof p);
  p.S0 = 100.0; p.K = 100.0; p.r = 0.05; p.sigma = 0.2; p.T = 1.0;
  p.payoff = MLMC_EURO; p.scheme = MLMC_EULER; p.icdf_method = 1; p.icdf_bits = 10;
  if (mlmc_default_format(&p, 3, &f) != MLMC_OK) return 1;
  if (mlmc_default_format(NULL, 3, &f) != MLMC_EINVAL) return 2;
  p.icdf_fields = 3;                       /* only Method 2 takes fields */
  if (mlmc_default_format(&p, 3, &f) != MLMC_EINVAL) return 3;
  printf("%s|%s|%d %d\n", mlmc_version(), mlmc_strerror(MLMC_EINVAL), f.f[6], f.e[6]);
  return 0;
}
"""


@pytest.fixture(scope="module")
def libdir():
    if shutil.which("nvcc") is None or shutil.which("gcc") is None:
        pytest.skip("nvcc or gcc not available")
    from paper_2502_07123_gb300 import build
    return os.path.dirname(build.build())


def test_c_program_uses_the_boundary(libdir, tmp_path):
    src = tmp_path / "caller.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "caller"
    cuda_lib = "/usr/local/cuda/lib64"
    cmd = ["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           "-L", libdir, "-lmlmc_gb300", "-Wl,-rpath," + libdir]
    if os.path.isdir(cuda_lib):
        cmd += ["-L", cuda_lib, "-Wl,-rpath," + cuda_lib]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    version, err, fmt = r.stdout.strip().split("|")
    assert "sm_103a" in version and err
    f_s, e_s = (int(x) for x in fmt.split())
    assert 10 <= f_s <= 21 and e_s >= 1
