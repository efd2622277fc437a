"""The coordinate arithmetic of the kernels divides by the lattice radices Lx/2, Ly, Lz with
multiplier constants (division by invariant integers, Granlund and Montgomery 1994), set on
the host by geom_set_divisor and applied by geom_div, the same __host__ __device__ code the
kernels run. This CPU test compiles a host program against that header and checks
geom_div(n) == n / d for every n below 2^22 and the top of the 32-bit range, for every
radix d from 1 to 128 (even lattice extents up to 256 in x and 128 in y, z)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1112_5280_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "dslash.cuh"
int main() {
  long long bad = 0, checked = 0;
  for (unsigned d = 1; d <= 128; ++d) {
    lqcd::Geom g{};
    lqcd::geom_set_divisor(g, 0, d);
    for (unsigned n = 0; n < (1u << 22); ++n, ++checked)
      if (lqcd::geom_div(g, 0, n) != n / d) ++bad;
    for (unsigned n = 0xffffffffu - (1u << 16); n != 0; ++n, ++checked)
      if (lqcd::geom_div(g, 0, n) != n / d) ++bad;
  }
  std::printf("%lld %lld\n", checked, bad);
  return bad != 0;
}
"""


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_division_by_invariant_integers_is_exact(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not available")
    src = tmp_path / "geom_div.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "geom_div"
    subprocess.run([nvcc, "-std=c++17", "-O2", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}",
                    "-o", str(exe), str(src)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    checked, bad = map(int, out.stdout.split())
    assert out.returncode == 0 and bad == 0 and checked == 128 * ((1 << 22) + (1 << 16) + 1)
