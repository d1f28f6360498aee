"""The integer-pipe conversions of csrc/alb_cvt.cuh against IEEE 754.

The header compiles as plain host C++; a small driver built here with g++
converts random and boundary bit patterns both ways and compares each result
with the host's own conversion (a C cast, IEEE round-to-nearest-even), which
is what CUDA's cvt.rn instructions compute. Every case must agree bit for bit
except those the header states: inputs below FP32's normal range give a
signed zero. Runs on the CPU only.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "paper_2009_13426_gb300", "csrc")

DRIVER = r"""
#include <math.h>
#include <stdio.h>
#include <stdint.h>
#include <string.h>
#include <limits.h>
#include "alb_cvt.cuh"

static uint64_t st = 0x9e3779b97f4a7c15ull;
static uint64_t next() {  /* splitmix64 */
  uint64_t z = (st += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
static double d_of(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
static uint64_t b_of(double d) { uint64_t b; memcpy(&b, &d, 8); return b; }
static float f_of(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t fb_of(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

static long bad = 0, n_d2f = 0, n_f2d = 0, n_i2d = 0, n_flush = 0;

static void check_d2f(double d) {
  const float got = alb::cvt_f32_rn(d);
  float want = (float)d;
  ++n_d2f;
  if (isnan(d)) { if (!isnan(got)) { if (bad++ < 10) printf("d2f NaN %a\n", d); } return; }
  if (fabs(d) < 0x1p-126) {  /* stated: a zero of the input's sign */
    ++n_flush;
    want = signbit(d) ? -0.0f : 0.0f;
  }
  if (fb_of(got) != fb_of(want)) {
    if (bad++ < 10) printf("d2f %a: got %a want %a\n", d, (double)got, (double)want);
  }
}
static void check_f2d(float f) {
  const double got = alb::cvt_f64(f);
  double want = (double)f;
  ++n_f2d;
  if (isnan(f)) { if (!isnan(got)) { if (bad++ < 10) printf("f2d NaN\n"); } return; }
  if (f != 0.0f && fabsf(f) < 0x1p-126f) { ++n_flush; want = signbit(f) ? -0.0 : 0.0; }
  if (b_of(got) != b_of(want)) {
    if (bad++ < 10) printf("f2d %a: got %a want %a\n", (double)f, got, want);
  }
}
static void check_i2d(int n) {
  const double got = alb::cvt_f64(n);
  const double want = (double)n;
  ++n_i2d;
  if (b_of(got) != b_of(want)) {
    if (bad++ < 10) printf("i2d %d: got %a want %a\n", n, got, want);
  }
}

int main() {
  /* FP64 -> FP32: random patterns over all exponents, then exponents near
     FP32's range with random fractions, then the rounding boundaries */
  for (int k = 0; k < 2000000; ++k) check_d2f(d_of(next()));
  for (int k = 0; k < 2000000; ++k) {
    const uint64_t r = next();
    const uint64_t ex = 896 - 30 + (r % 320);  /* FP32 exponents -30 .. 289 */
    check_d2f(d_of((r & 0x800fffffffffffffull) | (ex << 52)));
  }
  for (uint64_t ex = 860; ex <= 1160; ++ex) {
    for (int s = 0; s < 2; ++s) {
      const uint64_t base = ((uint64_t)s << 63) | (ex << 52);
      for (uint64_t m23 = 0; m23 < 4; ++m23) {
        const uint64_t tops[4] = {0, 1, 0x7ffffe, 0x7fffff};
        const uint64_t kept = tops[m23] << 29;
        const uint64_t drops[6] = {0, 1, 0x0fffffff, 0x10000000, 0x10000001, 0x1fffffff};
        for (int j = 0; j < 6; ++j) check_d2f(d_of(base | kept | drops[j]));
      }
    }
  }
  const double specials[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, -NAN, 1.0, -1.0,
                             3.4028234663852886e38, 3.4028235677973366e38, 3.402823567797337e38,
                             0x1p-126, -0x1p-126, 0x1.fffffep-127, 0x1p-149, 4.9e-324,
                             1e-300, 1e300, 0.1, 1.0 / 3.0};
  for (double d : specials) check_d2f(d);

  /* FP32 -> FP64: every exponent with random fractions, and the specials */
  for (int k = 0; k < 2000000; ++k) check_f2d(f_of((uint32_t)next()));
  for (uint32_t e = 0; e < 256; ++e)
    for (int k = 0; k < 64; ++k)
      check_f2d(f_of((uint32_t)(next() & 0x807fffffu) | (e << 23)));
  const float fspecials[] = {0.0f, -0.0f, INFINITY, -INFINITY, NAN, 1.0f, -1.0f, 3.4028235e38f,
                             0x1p-126f, 0x1p-149f, -0x1p-149f, 1e-3f, -1e-3f};
  for (float f : fspecials) check_f2d(f);

  /* int32 -> FP64: random, powers of two and their neighbours, the ends */
  for (int k = 0; k < 2000000; ++k) check_i2d((int)(uint32_t)next());
  for (int p = 0; p < 31; ++p) {
    const int v = 1 << p;
    check_i2d(v); check_i2d(v - 1); check_i2d(v + 1);
    check_i2d(-v); check_i2d(-v + 1); check_i2d(-v - 1);
  }
  check_i2d(0); check_i2d(INT_MAX); check_i2d(INT_MIN); check_i2d(INT_MIN + 1);
  for (int v = -70000; v <= 70000; ++v) check_i2d(v);

  printf("cases d2f %ld f2d %ld i2d %ld flushed %ld bad %ld\n", n_d2f, n_f2d, n_i2d, n_flush, bad);
  return bad != 0;
}
"""


def test_integer_conversions_match_ieee(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "cvt_check.cpp"
    exe = tmp_path / "cvt_check"
    src.write_text(DRIVER)
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", HEADER_DIR,
                    str(src), "-o", str(exe)], check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    counts = dict(zip(r.stdout.split()[1::2], r.stdout.split()[2::2]))
    assert int(counts["d2f"]) > 4_000_000 and int(counts["f2d"]) > 2_000_000
    assert int(counts["i2d"]) > 2_000_000 and int(counts["bad"]) == 0
    # the flushed range was reached (both directions have inputs there)
    assert int(counts["flushed"]) > 1000


# Mistakes planted in copies of the header: ties rounded away from zero, the
# exponent threshold of the flushed range off by one, the int32 exponent bias
# off by one, the FP32 -> FP64 bias off by one, the fraction shifted by one
# bit. Each must make the comparison fail.
PLANTED = [
    ("((r == 0x10000000u) & (m & 1u))", "(r == 0x10000000u)"),
    ("b = e <= 0 ? 0u : b;", "b = e < 0 ? 0u : b;"),
    ("(1054 - lz)", "(1053 - lz)"),
    ("e + 896u", "e + 895u"),
    ("(x >> 12)", "(x >> 11)"),
]


def test_planted_mistakes_fail(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    header = open(os.path.join(HEADER_DIR, "alb_cvt.cuh")).read()
    (tmp_path / "cvt_check.cpp").write_text(DRIVER)
    for k, (good, bad) in enumerate(PLANTED):
        assert header.count(good) == 1, good
        d = tmp_path / ("m%d" % k)
        d.mkdir()
        (d / "alb_cvt.cuh").write_text(header.replace(good, bad))
        exe = d / "cvt_check"
        subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", str(d),
                        str(tmp_path / "cvt_check.cpp"), "-o", str(exe)],
                       check=True, capture_output=True, text=True)
        r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
        assert r.returncode != 0, ("planted mistake not caught", bad)
