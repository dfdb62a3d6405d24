"""The FP32 form's FP64 <-> FP32 conversions (integer bit manipulation in
csrc/dmn_device.cuh) against the host's IEEE 754 conversions.

The helpers are compiled for the host with nvcc and run on the CPU: narrow_rn
must equal the C cast (round to nearest, ties to even) everywhere in FP32's
normal range, including exact ties, rounding carries into the exponent and
overflow; below 2^-126 it returns a signed zero (documented), and NaN stays
NaN.  widen must equal the exact C cast for every normal, zero, infinite and
NaN FP32 number.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r'''
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstdint>
#include <cstring>
#include "dmn_device.cuh"
using namespace dmn;

static unsigned long long rng = 0x9e3779b97f4a7c15ull;
static unsigned long long next() {   // splitmix64
  unsigned long long z = (rng += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
static int bad = 0;
static long checked = 0;
static void check_narrow(double x) {
  const float got = narrow_rn(x);
  ++checked;
  if (std::isnan(x)) { if (!std::isnan(got)) { ++bad; printf("nan %a\n", x); } return; }
  const double ax = std::fabs(x);
  if (ax < 0x1p-126 && !(ax == 0x1p-126)) {
    // below the normal range: a signed zero, unless the value rounds up to 2^-126 itself
    const float want = (float)x;
    const bool ok = (bits_of(got) == (bits_of(x) >> 32 & 0x80000000u)) ||
                    (std::fabs((double)want) == 0x1p-126 && bits_of(got) == bits_of(want));
    if (!ok) { ++bad; if (bad < 10) printf("small %a -> %a\n", x, (double)got); }
    return;
  }
  const float want = (float)x;
  if (bits_of(got) != bits_of(want)) { ++bad; if (bad < 10) printf("narrow %a -> %a, want %a\n", x, (double)got, (double)want); }
}
static void check_widen(float x) {
  const double got = widen(x);
  ++checked;
  if (std::isnan(x)) { if (!std::isnan(got)) { ++bad; printf("nan widen\n"); } return; }
  if (x != 0.0f && std::fabs(x) < 0x1p-126f) {
    if (bits_of(got) != ((unsigned long long)(bits_of(x) & 0x80000000u) << 32)) { ++bad; printf("sub widen\n"); }
    return;
  }
  const double want = (double)x;
  if (bits_of(got) != bits_of(want)) { ++bad; if (bad < 10) printf("widen %a -> %a\n", (double)x, got); }
}
int main() {
  // random bit patterns over the whole binary64 range, and concentrated on FP32's range
  for (int i = 0; i < 2000000; ++i) {
    unsigned long long u = next();
    double x;
    memcpy(&x, &u, 8);
    check_narrow(x);
    const unsigned long long e = 860 + next() % 330;   // exponents 2^-163 .. 2^166
    u = (u & 0x800fffffffffffffull) | (e << 52);
    memcpy(&x, &u, 8);
    check_narrow(x);
  }
  // exact ties and their neighbours, carries into the exponent, the ends of the range
  for (int i = 0; i < 200000; ++i) {
    const unsigned f = (unsigned)next();
    const unsigned e = 1 + (unsigned)(next() % 254);
    const unsigned fb = (f & 0x807fffffu) | (e << 23);
    const double base = (double)float_of(fb);
    const unsigned long long b = bits_of(base);
    for (long long d = -2; d <= 2; ++d) {
      check_narrow(double_of(b + (1ull << 28) + d));   // half an FP32 ulp above base, +-2 FP64 ulps
      check_narrow(double_of(b + d));
    }
  }
  const double special[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, -NAN, 0x1p-126, -0x1p-126, 0x1.fffffep127,
                            0x1.fffffefffffffp127, 0x1.ffffffp127, 0x1p128, 1e300, -1e300, 0x1p-127, 0x1.ffffffp-127,
                            0x1.fffffe8p-127, 5e-324, 1.0, -1.0, 0.1, 3.0, 1.0 + 0x1p-24, 1.0 + 0x1.8p-23};
  for (double x : special) check_narrow(x);
  // every FP32 number with a stride, plus all exponents with random fractions
  for (unsigned long long u = 0; u < (1ull << 32); u += 4099) check_widen(float_of((unsigned)u));
  for (unsigned e = 0; e < 256; ++e)
    for (int i = 0; i < 2000; ++i) check_widen(float_of(((unsigned)next() & 0x807fffffu) | (e << 23)));
  printf("checked %ld bad %d\n", checked, bad);
  return bad != 0;
}
'''


def test_conversions_match_ieee_casts(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "conv.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "conv"
    inc = os.path.join(ROOT, "paper_2103_08253_gb300", "csrc")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-I", inc, "-o", str(exe), str(src)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout
    assert "bad 0" in r.stdout
