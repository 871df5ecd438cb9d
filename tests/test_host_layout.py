"""Host-side layout and dispatch rules of the slice GEMM, checked on the CPU
by compiling the library's internal header with the host compiler (no GPU):

* the pre-swizzled digit tile layouts: the single-CTA layout and the halves
  layout of B tiles for CTA pairs are both bijections of (row, 16-byte chunk)
  onto the 32 KiB tile; in the halves layout each 64-row half is one
  contiguous 16 KiB block made of two 8 KiB atoms along k, rows 128 bytes
  apart, and both layouts put chunk c of row r at chunk position c ^ (r % 8)
  of its 128-byte row (the swizzle the MMA descriptors name);
* which products run on CTA pairs: bf16 digits, two or more tile-rows of A,
  no split-k; never the FP8 digits; dims made for B alone (m = 0) do not
  choose pairs by themselves, which is why the host-buffer pipeline copies the
  choice of its largest block to every split and product sharing B's planes;
* the workspace does not depend on the choice (the halves layout fills the
  same bytes);
* the plan of the no-allocation call: the split-k plan of the grown-workspace
  call when it fits the fixed scratch, else the unsplit product."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1211_1581_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROGRAM = r"""
#include "mxm_internal.h"
#include <cstdio>
#include <vector>
using namespace mxm;
static int fails = 0;
#define CHECK(c) do { if (!(c)) { std::printf("FAIL %s line %d\n", #c, __LINE__); ++fails; } } while (0)
int main() {
  // layouts: bijections onto the 2048 16-byte chunks of a 32 KiB tile
  for (int layout = 0; layout < 2; ++layout) {
    std::vector<int> seen(kOzTileBytes / 16, 0);
    for (int r = 0; r < kOzTileRows; ++r)
      for (int c = 0; c < kOzChunksPerRow; ++c) {
        const int off = layout ? oz_chunk_offset_halves(r, c) : oz_chunk_offset(r, c);
        CHECK(off % 16 == 0 && off >= 0 && off < kOzTileBytes);
        if (off % 16 == 0 && off >= 0 && off < kOzTileBytes) seen[off / 16] += 1;
        // chunk position inside the 128-byte row: the 128-byte swizzle
        CHECK(((off % 128) / 16) == ((c & 7) ^ (r & 7)));
      }
    int once = 0;
    for (int v : seen) once += (v == 1);
    CHECK(once == kOzTileBytes / 16);
  }
  // halves: rows 64h .. 64h + 63 fill bytes [16 KiB h, 16 KiB (h + 1)); inside a
  // half, atom a (k 64a .. 64a + 63) at 8 KiB a, row r % 64 at 128 (r % 64)
  for (int r = 0; r < kOzTileRows; ++r)
    for (int c = 0; c < kOzChunksPerRow; ++c) {
      const int off = oz_chunk_offset_halves(r, c);
      const int h = r / 64, a = c / 8;
      CHECK(off / (kOzTileBytes / 2) == h);
      CHECK((off % (kOzTileBytes / 2)) / (kOzAtomBytes / 2) == a);
      CHECK((off % (kOzAtomBytes / 2)) / 128 == r % 64);
    }
  // dispatch
  {
    OzakiDims d = ozaki_dims(300, 200, 257, 7, 7);  // Mt = 3
    CHECK(d.Mt == 3 && d.pair == 1 && ozaki_cta2(d) && ozaki_b_halves(d));
    d = ozaki_dims(128, 200, 257, 7, 7);            // one tile-row: single CTAs
    CHECK(d.pair == 0 && !ozaki_cta2(d) && !ozaki_b_halves(d));
    d = ozaki_dims(8192, 8192, 8192, 7, 7, true);  // balanced digits ride in bf16 too
    CHECK(d.pair == 1 && ozaki_cta2(d));
    d = ozaki_dims_fp8(8192, 8192, 8192, 12);       // E4M3 digits: single CTAs
    CHECK(d.pair == 0 && !ozaki_cta2(d) && !ozaki_b_halves(d));
    d = ozaki_dims_splitk(256, 65536, 128, 7, 7);   // few C tiles, long k: split-k
    CHECK(d.splits > 1 && d.pair == 0 && !ozaki_cta2(d));
    d = ozaki_dims_splitk(8192, 8192, 8192, 7, 7);  // enough tiles: no split-k, pairs
    CHECK(d.splits == 1 && d.pair == 1 && ozaki_cta2(d));
    OzakiDims db = ozaki_dims(0, 8192, 4096, 7, 7); // B alone: no choice of its own
    CHECK(db.pair == 0);
    OzakiDims dg = ozaki_dims(100, 8192, 4096, 7, 7);  // a short last panel of A ...
    dg.pair = 1;                                       // ... given the shared choice
    CHECK(ozaki_cta2(dg) && dg.Mt == 1);               // runs on pairs, rank 1 idle
  }
  // the no-allocation plan: mxm_f64_emul's split-k plan when it fits the
  // cap, else the unsplit product; either way within the cap or refused
  {
    const size_t cap = size_t(64) << 20;
    OzakiDims d = ozaki_dims_capped(256, 2048, 256, 7, 7, cap);    // 4 tiles x 4 ranges
    CHECK(d.splits == 4 && ozaki_layout(d).total <= cap);
    CHECK(d.splits == ozaki_dims_splitk(256, 2048, 256, 7, 7).splits);
    d = ozaki_dims_capped(1024, 1024, 1024, 7, 7, cap);           // split plan too big
    CHECK(ozaki_dims_splitk(1024, 1024, 1024, 7, 7).splits == 2);
    CHECK(ozaki_layout(ozaki_dims_splitk(1024, 1024, 1024, 7, 7)).total > cap);
    CHECK(d.splits == 1 && ozaki_layout(d).total <= cap);
    d = ozaki_dims_capped(2048, 2048, 2048, 7, 7, cap);           // refused by the caller
    CHECK(ozaki_layout(d).total > cap);
  }
  // the workspace does not depend on the choice
  {
    OzakiDims a = ozaki_dims(1000, 3000, 700, 7, 7), b = a;
    b.pair = 0;
    const OzakiLayout La = ozaki_layout(a), Lb = ozaki_layout(b);
    CHECK(La.total == Lb.total && La.bslices == Lb.bslices && La.sums == Lb.sums);
  }
  std::printf("%s %d\n", fails ? "FAILED" : "ok", fails);
  return fails ? 1 : 0;
}
"""


def test_tile_layouts_and_pair_dispatch(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("host compiler or CUDA headers missing")
    src = tmp_path / "layout_check.cpp"
    exe = tmp_path / "layout_check"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-std=c++17", "-O1", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}",
                    f"-I{CUDA_INC}", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip().endswith("ok 0")
