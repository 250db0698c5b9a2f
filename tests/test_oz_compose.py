"""Host check of the integer rounding used by the tensor-core product epilogues.

oz_compose (paper_1504_05090_gb300/csrc/oz_compose.cuh) rounds
2^E (hi + 2^-28 lo) to FP64 with integer instructions.  The header also
compiles as plain C++; this test builds a small program with the host compiler
and compares it bit for bit with the FP64 definition (two exact conversions and
one fused multiply-add, which round the exact value once), on random digit
sums, on exact ties and carries, and across the exponent range.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_1504_05090_gb300", "csrc", "oz_compose.cuh")

PROGRAM = r"""
#include "oz_compose.cuh"
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
static double ref(long long hi, long long lo, int E, bool neg, bool& ok) {
  double sum = std::fma(static_cast<double>(lo), 0x1p-28, static_cast<double>(hi));
  if (neg) sum = -sum;
  long long bits;
  std::memcpy(&bits, &sum, 8);
  const int Ex = static_cast<int>((bits >> 52) & 0x7FF), E2 = Ex + E;
  ok = Ex != 0 && Ex != 0x7FF && E2 > 0 && E2 < 2047;
  bits = (bits & ~(0x7FFLL << 52)) | (static_cast<long long>(E2 & 0x7FF) << 52);
  double d;
  std::memcpy(&d, &bits, 8);
  return d;
}
int main() {
  std::mt19937_64 rng(7);
  long long bad = 0, n = 0;
  auto check = [&](long long hi, long long lo, int E, bool neg) {
    bool o1, o2;
    const double a = dqmc::oz_compose(hi, lo, E, neg, o1), b = ref(hi, lo, E, neg, o2);
    ++n;
    if (o2 && (!o1 || std::memcmp(&a, &b, 8) != 0)) ++bad;
    if (o1 && !o2 && !(hi == 0 && lo == 0)) {
      double s = std::fma(static_cast<double>(lo), 0x1p-28, static_cast<double>(hi));
      if (s != 0.0) ++bad;  // only an exact zero may be usable here and not there
    }
  };
  // digit sums P_d of up to 2^25, combined as the epilogues combine them
  for (int it = 0; it < 400000; ++it) {
    long long p[8];
    const int mag = static_cast<int>(rng() % 26);
    for (int d = 0; d < 8; ++d) {
      const long long lim = 1LL << (rng() % (mag + 1));
      p[d] = static_cast<long long>(rng() % (2 * lim + 1)) - lim;
      if (rng() % 8 == 0) p[d] = 0;
    }
    long long hi = 0, lo = 0;
    for (int d = 0; d < 4; ++d) hi += p[d] << (7 * (3 - d));
    for (int d = 4; d < 8; ++d) lo += p[d] << (7 * (7 - d));
    if (rng() % 16 == 0) hi = 0;
    if (rng() % 64 == 0) {  // cancellation between hi and lo
      hi = static_cast<long long>(rng() % (1 << 18)) - (1 << 17);
      lo = -(hi << 28) + (static_cast<long long>(rng() % 9) - 4);
    }
    check(hi, lo, static_cast<int>(rng() % 200) - 100, (rng() & 1) != 0);
  }
  // ties and carries at every bit position of lo
  for (long long hi : {1LL, 3LL, (1LL << 44) + 1, (1LL << 45) - 1, -(1LL << 45) + 1, -7LL, 0LL})
    for (int s = 0; s < 30; ++s)
      for (long long delta : {-1LL, 0LL, 1LL}) {
        const long long lo = (1LL << s) + delta;
        check(hi, lo, 0, false);
        check(hi, -lo, 3, true);
        check(hi, lo + (1LL << 40), -5, false);
      }
  // exponent range, including results that leave the normal range (ok = false)
  for (int E = -1100; E <= 1100; E += 7) check(12345678901LL, 987654321LL, E, (E & 1) != 0);
  std::printf("%lld %lld\n", n, bad);
  return 0;
}
"""


def test_integer_rounding_equals_fp64_rounding(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "compose.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "compose"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    n, bad = int(out[0]), int(out[1])
    assert n > 400000
    assert bad == 0
