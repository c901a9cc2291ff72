"""The integer-pipe float <-> double conversions of the FP64 refinement kernels
(csrc/oci_cvt.cuh) return bit for bit what a C cast returns (IEEE 754:
binary32 -> binary64 exact, binary64 -> binary32 round to nearest, ties to
even).  The header is compiled for the host with g++; every binary32 bit
pattern is converted, and binary64 inputs cover every exponent around the
binary32 range with random fractions, the exact halfway cases of both parities,
fractions of all ones (the carry into the exponent), and random bit patterns."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_00264_gb300", "csrc")

SRC = r"""
#include <math.h>
#include <stdio.h>
#include "oci_cvt.cuh"
using namespace oci;

static uint64_t sm = 0x9E3779B97F4A7C15ull;
static uint64_t next64() {  // splitmix64
  uint64_t z = (sm += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double dfrom(uint64_t u) { double d; memcpy(&d, &u, 8); return d; }
static long bad = 0, checked = 0;
static void check_d(uint64_t u) {
  const double x = dfrom(u);
  const float a = d2f_rn(x), b = (float)x;
  checked++;
  if (isnan(b) ? !isnan(a) : cvt_fbits(a) != cvt_fbits(b)) {
    if (bad++ < 5) printf("d2f %016llx: %08x vs %08x\n", (unsigned long long)u, cvt_fbits(a), cvt_fbits(b));
  }
}
int main() {
  long fbad = 0;
  for (uint64_t i = 0; i <= 0xffffffffull; i++) {
    const float f = cvt_bitsf((uint32_t)i);
    const double a = f2d_exact(f), b = (double)f;
    uint64_t ua, ub;
    memcpy(&ua, &a, 8);
    memcpy(&ub, &b, 8);
    if (isnan(b) ? !isnan(a) : ua != ub) {
      if (fbad++ < 5) printf("f2d %08x\n", (unsigned)i);
    }
  }
  for (uint64_t sgn = 0; sgn < 2; sgn++)
    for (uint64_t e = 860; e <= 1190; e++) {
      const uint64_t top = (sgn << 63) | (e << 52);
      check_d(top);
      check_d(top | 0xfffffffffffffull);           // all-ones fraction: carry into the exponent
      for (uint64_t k = 0; k < 64; k++) {
        const uint64_t f23 = next64() & 0x7fffffull;
        check_d(top | (f23 << 29) | (1ull << 28));  // exact halfway, both parities of f23
        check_d(top | ((f23 | 1) << 29) | (1ull << 28));
        check_d(top | ((f23 & ~1ull) << 29) | (1ull << 28));
        check_d(top | (f23 << 29) | (1ull << 28) | 1);  // just above halfway
        check_d(top | (f23 << 29) | ((1ull << 28) - 1));  // just below halfway
      }
      for (int k = 0; k < 20000; k++) check_d(top | (next64() & 0xfffffffffffffull));
    }
  check_d(0x7ff0000000000000ull); check_d(0xfff0000000000000ull);  // infinities
  check_d(0x7ff8000000000001ull); check_d(0x0000000000000001ull);  // NaN, smallest subnormal
  check_d(0x8000000000000000ull); check_d(0);                      // signed zeros
  for (long k = 0; k < 20000000; k++) check_d(next64());
  printf("f2d_bad %ld d2f_bad %ld d2f_checked %ld\n", fbad, bad, checked);
  return (fbad || bad) ? 1 : 0;
}
"""


def test_integer_conversions_equal_c_casts(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "cvt.cpp"
    src.write_text(SRC)
    exe = tmp_path / "cvt"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "f2d_bad 0 d2f_bad 0" in r.stdout
    assert int(r.stdout.split()[-1]) > 20_000_000
