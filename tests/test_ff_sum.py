"""The float-float sums of the rank-16 column solves (Knuth's two-sum and the
(s, c) accumulation in `csrc/nmf_tc16s.cuh`), compiled for the host with
nvcc and checked in exact rational arithmetic on the CPU (no GPU):

* two_sum(a, b) = (s, e) with s = fl(a + b) and s + e == a + b exactly, for
  random FP32 pairs across 2^-60 .. 2^60 of both signs, cancellations and
  ties included;
* ff_add over 256 terms (the lanes and groups of a block) leaves
  |(s + c) - sum| below 2^-40 of the sum of magnitudes, where a plain FP32
  sum of the same terms is off by up to ~2^-24 per term.
"""
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2101_08431_gb300", "csrc")

HARNESS = r'''
#include "nmf_tc16.cu"
#include <cstdio>
#include <cstdint>
#include <cstring>
using namespace nmfgb::tc16s;
static uint32_t bits(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }
static float flt(uint32_t u) { float f; std::memcpy(&f, &u, 4); return f; }
int main() {
  uint32_t a, b;
  char mode[8];
  // "P a b": one two_sum; "S n x1 .. xn": ff_add over the terms
  while (std::scanf("%7s", mode) == 1) {
    if (mode[0] == 'P') {
      std::scanf("%x %x", &a, &b);
      float s, e;
      two_sum(flt(a), flt(b), s, e);
      std::printf("%08x %08x\n", bits(s), bits(e));
    } else {
      int n;
      std::scanf("%d", &n);
      float s = 0.f, c = 0.f;
      for (int i = 0; i < n; ++i) {
        std::scanf("%x", &a);
        ff_add(s, c, flt(a), 0.f);
      }
      std::printf("%08x %08x\n", bits(s), bits(c));
    }
  }
  return 0;
}
'''


def _f(u):
    return struct.unpack("<f", struct.pack("<I", u))[0]


def _u(f):
    return struct.unpack("<I", struct.pack("<f", np.float32(f)))[0]


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("ff")
    src = d / "ff.cu"
    src.write_text(HARNESS)
    exe = d / "ff"
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        "--expt-relaxed-constexpr", "-diag-suppress", "177", "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return str(exe)


def _run(exe, lines):
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    return [tuple(int(w, 16) for w in ln.split()) for ln in out.stdout.strip().splitlines()]


def test_two_sum_is_exact(harness):
    rng = np.random.default_rng(7)
    n = 4000
    ea, eb = rng.integers(-60, 61, n), rng.integers(-60, 61, n)
    a = (rng.uniform(1, 2, n) * 2.0 ** ea * rng.choice([-1, 1], n)).astype(np.float32)
    b = (rng.uniform(1, 2, n) * 2.0 ** eb * rng.choice([-1, 1], n)).astype(np.float32)
    b[:500] = -a[:500] * np.float32(1 + 2 ** -20)                     # cancellations
    b[500:1000] = (a[500:1000] * np.float32(2 ** -24)).astype(np.float32)   # half-ulp ties
    pairs = [(_u(x), _u(y)) for x, y in zip(a, b)]
    res = _run(harness, ["P %08x %08x" % p for p in pairs])
    assert len(res) == n
    for (ua, ub), (us, ue) in zip(pairs, res):
        fa, fb, fs, fe = _f(ua), _f(ub), _f(us), _f(ue)
        assert fs == float(np.float32(fa) + np.float32(fb))
        assert Fraction(fs) + Fraction(fe) == Fraction(fa) + Fraction(fb), (fa, fb, fs, fe)


def test_ff_accumulation_error(harness):
    rng = np.random.default_rng(11)
    lines, terms = [], []
    for t in range(40):
        x = (rng.standard_normal(256) * 2.0 ** rng.integers(-8, 9, 256)).astype(np.float32)
        if t % 4 == 0:
            x = np.abs(x)                        # sums of squares and norms: all terms positive
        terms.append(x)
        lines.append("S 256 " + " ".join("%08x" % _u(v) for v in x))
    res = _run(harness, lines)
    for x, (us, uc) in zip(terms, res):
        exact = sum(Fraction(float(v)) for v in x)
        mag = sum(abs(Fraction(float(v))) for v in x)
        got = Fraction(_f(us)) + Fraction(_f(uc))
        assert abs(got - exact) <= mag * Fraction(1, 2 ** 40), float(abs(got - exact) / mag)
        plain = np.float32(0)
        for v in x:
            plain = np.float32(plain + v)
        # the carried error is what a plain FP32 sum loses (a check that the pin can fail)
        assert abs(got - exact) <= abs(Fraction(float(plain)) - exact)
