"""Bounds of the rank-16 tensor-core M pass's launch shapes, checked on the
CPU for every row count up to 2^20 and every cluster size (no GPU: the shape
arithmetic is host code).  A host harness compiled with nvcc calls the
library's own `tc16_shape` with the kernel's constants and checks that every
shape it accepts keeps the kernel's accesses in bounds:

* shared memory within the per-CTA limit, and below the 256 KB that the
  14-bit start-address field of a tcgen05 shared-memory descriptor reaches;
* rows per CTA a multiple of 128 (the P-MMA's 128-row chunks) covering ld;
* tensor memory a power of two <= 512 columns holding the NS B accumulators
  (32 columns each) and the P chunks (16 columns each);
* the B-MMA's reads (rows 32-63 of its M = 64 A operand run 512 bytes past
  each K-step) inside the X slab and its zero padding, and the P-MMA's reads
  inside a slot;
* the received-partials ring of each solve group within its arrays.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2101_08431_gb300", "csrc")

HARNESS = r'''
#include "nmf_tc16.cu"
#include <cstdio>
using namespace nmfgb;
using namespace nmfgb::tc16;
static int bad = 0;
#define CHECK(c, ...) do { if (!(c)) { if (bad++ < 10) { std::printf("FAIL %s: ", #c); std::printf(__VA_ARGS__); std::printf("\n"); } } } while (0)
int main() {
  const int optin = 232448;
  long long shapes = 0;
  for (int ld = 32; ld <= (1 << 20); ld += (ld < 65536 ? 32 : 4096)) {
    bool any = false;
    for (int C = 1; C <= 16; C <<= 1) {
      Tc16Plan L;
      if (!tc16_shape(ld, C, optin, &L)) continue;
      any = true;
      ++shapes;
      const int R = L.R, NS = L.NS, nown = TJ / C;
      CHECK(L.smem <= (size_t)optin, "ld %d C %d smem %zu", ld, C, L.smem);
      CHECK(L.smem < 256 * 1024, "ld %d C %d smem %zu", ld, C, L.smem);
      CHECK(R % 128 == 0 && (long long)R * C >= ld, "ld %d C %d R %d", ld, C, R);
      CHECK(NS >= 2 && NS <= NSMAX, "ld %d C %d NS %d", ld, C, NS);
      CHECK((L.tmem_cols & (L.tmem_cols - 1)) == 0 && L.tmem_cols >= 32 && L.tmem_cols <= 512, "tmem %d", L.tmem_cols);
      CHECK(L.tmem_cols >= NS * 32 + (R / 128) * 16, "ld %d C %d tmem %d", ld, C, L.tmem_cols);
      CHECK(slot_bytes(R) == (size_t)R * ROW_BYTES, "slot");
      CHECK(L.smem == small_bytes() + ax_bytes(R) + (size_t)NS * slot_bytes(R), "smem sum");
      // B-MMA: last K-step over a full CTA slab, K-group 1, M-group 7, end of a core matrix
      const size_t bmax = (size_t)(R / 16 - 1) * 1024 + 512 + 7 * 128 + 127;
      CHECK(bmax < ax_bytes(R), "ld %d C %d B-MMA read %zu of %zu", ld, C, bmax, ax_bytes(R));
      const size_t bslot = (size_t)(R / 16 - 1) * 1024 + 512 + 3 * 128 + 127;
      CHECK(bslot < slot_bytes(R), "B operand read %zu", bslot);
      // P-MMA: last chunk, lo half, MN-group 15, K-group 1
      const size_t pmax = (size_t)(R / 128 - 1) * 16 * 512 + 256 + 15 * 512 + 128 + 127;
      CHECK(pmax < slot_bytes(R), "ld %d C %d P-MMA read %zu", ld, C, pmax);
      const int NSG = (NS * nown + NG - 1) / NG > 2 ? (NS * nown + NG - 1) / NG : 2;
      CHECK(NSG <= NSG_MAX && NSG * C <= XROWS, "ld %d C %d NSG %d", ld, C, NSG);
      CHECK(nown * C == TJ, "ownership");
    }
    // every ld up to 16 x the largest slab that fits has at least one shape
    if (ld <= 8192) CHECK(any, "no shape for ld %d", ld);
  }
  std::printf("%lld shapes checked, %d failures\n", shapes, bad);
  return bad ? 1 : 0;
}
'''


def test_tc16_shapes_stay_in_bounds(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "harness.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "harness"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                        "--expt-relaxed-constexpr", "-diag-suppress", "177", "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "0 failures" in out.stdout
