"""The double-float split that stores the OK_W_DF64 copy of W (csrc/ok_split.cuh), compiled for the
host: for every finite input it must give bit for bit the pair the definition gives,
hi = RN_float(d) and lo = RN_float(d - hi), also where it takes its integer path."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1311_5029_gb300", "csrc")

HARNESS = r"""
#include "ok_split.cuh"
#include <cmath>
#include <cstdio>
#include <random>
using namespace okgb;
static dd definition(double d) {
  const float hi = (float)d;
  return dd(hi, (float)(d - (double)hi));
}
int main() {
  std::mt19937_64 rng(20131120);
  long long n = 0, fast = 0, bad = 0;
  auto check = [&](double d) {
    const dd a = split_df(d), b = definition(d);
    long long D;
    memcpy(&D, &d, 8);
    const int ed = (int)((D >> 52) & 0x7ff);
    ++n;
    if (ed >= 1023 - 74 && ed <= 1023 + 126) ++fast;
    if (memcmp(&a, &b, sizeof a) != 0) {
      if (bad < 5) printf("mismatch %a: (%a, %a) vs (%a, %a)\n", d, a.hi, a.lo, b.hi, b.lo);
      ++bad;
    }
  };
  for (int k = 0; k < 2000000; ++k) {  // arbitrary bit patterns
    const unsigned long long u = rng();
    double d;
    memcpy(&d, &u, 8);
    if (std::isfinite(d)) check(d);
  }
  std::uniform_real_distribution<double> un(-4.0, 4.0);
  for (int k = 0; k < 2000000; ++k) check(un(rng));  // the magnitudes of W entries
  for (int e = -160; e <= 140; e += 3)                 // around powers of two, both signs
    for (int t = -600; t <= 600; ++t) {
      const double p = std::ldexp(1.0, e);
      check(p + t * std::ldexp(1.0, e - 53));
      check(-(p + t * std::ldexp(1.0, e - 53)));
      check(p * (1.0 + t * 0x1p-25));
    }
  const double edge[] = {0.0, -0.0, 0x1.fffffep127, 0x1.fffffefffffffp127, 0x1p-126, 0x1p-74, 0x1.fffffffffffffp-75,
                         4.9406564584124654e-324, 1.0, -1.0, 0x1.000001p0, 0x1.0000008p0, 0x1.fffffffp0};
  for (double d : edge) check(d);
  printf("checked %lld fast %lld bad %lld\n", n, fast, bad);
  return bad != 0 || fast < n / 3;
}
"""


def test_split_matches_definition(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "split_check.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "split_check"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-o", str(exe), str(src)], check=True,
                   capture_output=True, timeout=300)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
