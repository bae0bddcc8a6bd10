"""The division constants the kernels decode sites with (geom_set_divisors in csrc/geometry.cuh,
host code): for every lattice extent d, the multiply-high q = (t + ((n - t) >> 1)) >> (l - 1),
t = floor(n * m / 2^32), with the constants (m, l) the host computes, must equal floor(n / d) for
every 32-bit n.  The constants are printed by a small host program built from the header; the
division is checked here on random and edge-case n against Python's integer division."""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EXTENTS = [2, 4, 6, 8, 10, 12, 14, 16, 18, 20, 24, 28, 32, 40, 48, 64, 96, 128, 192, 256, 510, 512]

HARNESS = r"""
#include <cstdio>
#include "geometry.cuh"
int main() {
  const int ext[] = {%s};
  for (int d : ext) {
    nd::Geom g{};
    g.L[0] = 2; g.L[1] = d; g.L[2] = d; g.L[3] = d;
    nd::geom_set_divisors(g);
    std::printf("%%d %%u %%d\n", d, g.div_m[3], g.div_l[3]);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def constants(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and not shutil.which("nvcc"):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("divisors")
    src = d / "harness.cu"
    src.write_text(HARNESS % ", ".join(str(e) for e in EXTENTS))
    exe = d / "harness"
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "paper_1010_5636_gb300", "csrc"), str(src),
                    "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    rows = [tuple(int(x) for x in ln.split()) for ln in out.strip().splitlines()]
    return {dd: (m, l) for dd, m, l in rows}


@pytest.mark.parametrize("d", EXTENTS)
def test_multiply_high_division_is_exact(constants, d):
    m, l = constants[d]
    assert 0 <= m < 2 ** 32 and l >= 1
    rng = random.Random(d)
    ns = [0, 1, d - 1, d, d + 1, 2 * d - 1, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 1]
    ns += [rng.getrandbits(32) for _ in range(20000)] + [rng.getrandbits(26) for _ in range(20000)]
    ns += [k * d + r for k in (1, 1000, 123457) for r in (-1, 0, 1) if 0 <= k * d + r < 2 ** 32]
    for n in ns:
        t = (n * m) >> 32
        q = (t + ((n - t) >> 1)) >> (l - 1)
        assert q == n // d, (d, n, q)
