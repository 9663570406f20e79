"""Bounds of the rank-16 tensor-core pass's launch plans, checked on the CPU
(no GPU: the plan and the unit decomposition are host arithmetic).  A host
harness compiled with nvcc calls the library's own `tc16s::plan` and the
kernels' own unit maps (`bg_unit`, `pg_unit`, `wrap_col`, `xs_off`, `swz`)
for row counts up to 2^17, window sizes from 1 to 10^5 columns and several
ring positions, and walks every work unit of every CTA the way the B-GEMM
and P-GEMM kernels do, checking:

* shared memory within the per-CTA limit and below the 256 KB that the
  14-bit start-address field of a tcgen05 shared-memory descriptor reaches;
  2 <= stages <= NSMAX;
* every tensor copy: its box inside the mirrored M (rows inside ld, columns
  p0 .. p0 + box - 1 inside mcap + MIRROR, and each window column of the box
  either the physical column itself or its mirror), the innermost coordinate
  a multiple of 16 bytes, its destination a 1024-byte aligned slab of its
  stage; the split X / Y operands inside their buffers;
* chunk rows a multiple of 16 (whole MMA K-steps); every row of a tile
  covered by exactly one row split, every 64-column granule by exactly one
  column split;
* the MMA operand reads (last K-step, last core matrix) inside the converted
  area and the operand area of a stage, the converters' swizzled reads
  inside their slab;
* the epilogues' writes inside the B and P partial buffers, the solve
  kernel's writes inside the split Y and its block partials inside their
  buffer.
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
#include <vector>
using namespace nmfgb;
using namespace nmfgb::tc16s;
static int bad = 0;
#define CHECK(c, ...) do { if (!(c)) { if (bad++ < 10) { std::printf("FAIL %s: ", #c); std::printf(__VA_ARGS__); std::printf("\n"); } } } while (0)

int main() {
  const int optin = 232448, nsm = 152;
  long long plans = 0, cols = 0;
  const int ms[] = {1, 2, 15, 63, 64, 65, 127, 128, 129, 300, 1000, 2047, 6144, 16384, 100000};
  for (int ld = 32; ld <= (1 << 17); ld += (ld < 4096 ? 32 : (ld < 16384 ? 1024 : 8192))) {
    for (int m : ms) {
      if ((long long)m * ld > (1ll << 30)) continue;   // the largest windows on smaller ld
      for (int cap_extra : {0, 37}) {
        const int mcap = m + cap_extra;
        for (int head : {0, mcap / 2, mcap - 1}) {
          Plan L;
          if (!plan(ld, m, nsm, optin, &L)) { CHECK(false, "no plan ld %d m %d", ld, m); continue; }
          ++plans;
          Problem p{};
          p.n = ld; p.ld = ld; p.m = m; p.mcap = mcap; p.head = head; p.k = 16;
          CHECK(L.smemB <= (size_t)optin && L.smemP <= (size_t)optin, "smem");
          CHECK(L.smemB < 256 * 1024 && L.smemP < 256 * 1024, "descriptor reach");
          CHECK(L.NSB >= 2 && L.NSB <= NSMAX && L.NSP >= 2 && L.NSP <= NSMAX, "stages");
          CHECK(L.smemB == (size_t)CTL_BYTES + (size_t)L.NSB * BG_STAGE, "smemB");
          CHECK(L.smemP == (size_t)CTL_BYTES + (size_t)L.NSP * PG_STAGE, "smemP");
          CHECK(CTL_BYTES % 1024 == 0 && BG_STAGE % 1024 == 0 && PG_STAGE % 1024 == 0, "slab alignment");
          CHECK(L.SB >= 1 && (size_t)L.SB * mcap * 16 * 4 <= bpart_bytes(mcap), "Bpart ld %d m %d SB %d", ld, m, L.SB);
          CHECK(L.SP >= 1 && L.SP <= nsm, "SP %d", L.SP);   // P, H, terms partials: nsm slabs allocated
          CHECK(L.gridB >= 1 && L.gridB <= 2 * nsm && L.gridP >= 1 && L.gridP <= 2 * nsm, "grids");
          CHECK(2 * (L.smemB + 1024) <= (size_t)optin + 1024 && 2 * (L.smemP + 1024) <= (size_t)optin + 1024,
                "two CTAs per SM");
          {   // block partials, group partials and totals of reduce_blocks; its tickets
            for (int grid : {L.gridS, L.gridF}) {
              const size_t ngr = (grid + RGROUP - 1) / RGROUP;
              CHECK(((size_t)grid + ngr + 1) * RED * 8 <= red_bytes(nsm), "red");
              CHECK(1 + ngr <= ticket_count(nsm), "tickets");
            }
          }
          CHECK(L.cpg >= 1 && (long long)L.gridS * (SOLVE_T / 16) * L.cpg >= (long long)((m + PG_COLS - 1) / PG_COLS) * PG_COLS,
                "solve groups cover the padded window");
          CHECK(L.cpgF >= 1 && (long long)L.gridF * (SOLVE_T / 16) * L.cpgF >= (long long)((m + PG_COLS - 1) / PG_COLS) * PG_COLS,
                "solve groups cover the padded window");
          // ---- B-GEMM
          const int ntile = (m + BG_COLS - 1) / BG_COLS;
          const int nunits = ntile * L.SB;
          std::vector<int> rowcov((size_t)ntile * ld, 0);
          for (int b = 0; b < L.gridB; ++b)
            for (int u = b; u < nunits; u += L.gridB) {
              int tile, split, r0, r1;
              bg_unit(p, L.SB, u, tile, split, r0, r1);
              CHECK(split < L.SB && tile < ntile && r0 <= r1 && r1 <= ld && r0 % 32 == 0 && r1 % 32 == 0, "unit");
              CHECK(r1 - r0 >= 64 || ld < 64, "split rows ld %d SB %d: %d", ld, L.SB, r1 - r0);
              const int nv = std::min(BG_COLS, m - tile * BG_COLS);
              CHECK(nv >= 1, "nv");
              // the tile's window columns are consecutive columns of the mirrored
              // ring: box columns p0 .. p0 + 127 inside mcap + MIRROR
              const int p0 = wrap_col(head, tile * BG_COLS, mcap);
              CHECK(p0 >= 0 && p0 < mcap && p0 + BG_COLS <= mcap + MIRROR, "box columns");
              for (int j = 0; j < nv; ++j) {
                const int phys = wrap_col(head, tile * BG_COLS + j, mcap);
                const int ext = p0 + j;   // column of the mirrored buffer the box reads
                CHECK(ext == phys || (ext >= mcap && ext - mcap == phys && phys < MIRROR), "mirror col %d %d", ext, phys);
                ++cols;
              }
              for (int rc = r0; rc < r1; rc += BG_ROWS) {
                const int rows = std::min(BG_ROWS, r1 - rc);
                CHECK(rows % SLAB_ROWS == 0 && rows >= 16, "rows %d", rows);
                const int nslab = rows / SLAB_ROWS;
                for (int h = 0; h < nslab; ++h) {
                  const int x = rc + h * SLAB_ROWS;
                  CHECK((x * 4) % 16 == 0 && x + SLAB_ROWS <= ld, "box rows");
                  CHECK((h * BG_SLAB) % 1024 == 0 && h * BG_SLAB + BG_SLAB <= BG_XOFF, "slab dst");
                }
                CHECK((long long)(rc + rows) * 64 <= (long long)xs_bytes(ld), "X src");
                CHECK((long long)nslab * BG_SLAB + rows * 64 < (1 << 20), "tx");
                for (int r = rc; r < rc + rows; ++r) rowcov[(size_t)tile * ld + r]++;
                // MMA reads of the last K-step: A hi/lo, B
                const int ks = rows / 16 - 1;
                CHECK(BG_ALO + ks * 4096 + 2048 + 15 * 128 + 128 <= BG_XOFF, "A read");
                CHECK(BG_XOFF + ks * 1024 + 512 + 3 * 128 + 128 <= BG_STAGE, "B read");
                // converter reads (swizzled chunks) and writes
                const int g = rows / 8 - 1, j = 127;
                CHECK(swz(j, 2 * (g & 3) + 1) + 16 <= BG_SLAB && (g >> 2) < nslab, "cv read");
                CHECK(BG_ALO + g * 2048 + (j >> 3) * 128 + (j & 7) * 16 + 16 <= BG_XOFF, "cv write");
              }
            }
          for (size_t i = 0; i < rowcov.size(); ++i)
            if (rowcov[i] != 1) { CHECK(false, "row cover ld %d m %d: %d", ld, m, rowcov[i]); break; }
          // ---- P-GEMM
          const int nrb = (ld + PG_ROWS - 1) / PG_ROWS, ncg = (m + PG_COLS - 1) / PG_COLS;
          std::vector<int> gcov((size_t)nrb * ncg, 0);
          for (int b = 0; b < L.gridP; ++b)
            for (int u = b; u < nrb * L.SP; u += L.gridP) {
              int rb, split, g0, g1;
              pg_unit(p, L.SP, u, rb, split, g0, g1);
              CHECK(rb < nrb && split < L.SP && g0 <= g1 && g1 <= ncg, "punit");
              const int r0 = rb * PG_ROWS, rows = std::min(PG_ROWS, ld - r0);
              CHECK(rows >= 32 && rows % SLAB_ROWS == 0, "prows");
              for (int h = 0; h < rows / SLAB_ROWS; ++h)
                CHECK(r0 + h * SLAB_ROWS + SLAB_ROWS <= ld && h < 4 && (h * PG_SLAB) % 1024 == 0, "pbox rows");
              for (int g = g0; g < g1; ++g) {
                gcov[(size_t)rb * ncg + g]++;
                const int nv = std::min(PG_COLS, m - g * PG_COLS);
                CHECK(nv >= 1, "pnv");
                const int p0 = wrap_col(head, g * PG_COLS, mcap);
                CHECK(p0 >= 0 && p0 < mcap && p0 + PG_COLS <= mcap + MIRROR, "pbox columns");
                for (int j = 0; j < nv; ++j) {
                  const int phys = wrap_col(head, g * PG_COLS + j, mcap);
                  const int ext = p0 + j;
                  CHECK(ext == phys || (ext >= mcap && ext - mcap == phys && phys < MIRROR), "pmirror");
                  ++cols;
                }
                CHECK((size_t)(g + 1) * PG_COLS * 64 <= ys_bytes(mcap), "Y src");
                CHECK(PG_ALO + 3 * 4096 + 15 * 256 + 128 + 128 <= PG_YOFF, "PA read");
                CHECK(PG_YOFF + 3 * 1024 + 512 + 3 * 128 + 128 <= PG_STAGE, "PB read");
                CHECK(3 * PG_SLAB + swz(63, 7) + 16 <= PG_YOFF, "pcv read");
              }
              // epilogue rows stay inside ld
              CHECK(r0 + rows <= ld, "prow");
            }
          for (size_t i = 0; i < gcov.size(); ++i)
            if (gcov[i] != 1) { CHECK(false, "granule cover ld %d m %d", ld, m); break; }
          // ---- solve: split Y writes up to the padded window
          const int ncolp = ncg * PG_COLS;
          CHECK(xs_off(ncolp - 1, 31) + 2 <= (int)ys_bytes(mcap), "Ys write");
        }
      }
    }
  }
  std::printf("%lld plans, %lld tile columns checked, %d failures\n", plans, cols, bad);
  return bad ? 1 : 0;
}
'''


def test_tc16_plans_stay_in_bounds(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "harness.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "harness"
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        "--expt-relaxed-constexpr", "-diag-suppress", "177", "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "0 failures" in out.stdout
