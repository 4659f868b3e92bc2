"""Host logic of the binning plan (ddgs::plan_binning, a host function of the
library's internal header), compiled into a small host program with nvcc and
run on the CPU (no GPU needed): for many layouts, the binning blocks cover
every view's tiles in bands of at most BIN_HIST_MAX tiles, an empty request
gets no block, and the tile counters stay below hist_slot_bound, the size the
workspace and the static scratch reserve for them."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "ddgs_internal.cuh"

static uint64_t state = 12345;
static int64_t rnd(int64_t lo, int64_t hi) {  // inclusive, xorshift64
  state ^= state << 13; state ^= state >> 7; state ^= state << 17;
  return lo + (int64_t)(state % (uint64_t)(hi - lo + 1));
}

int main() {
  int layouts = 0;
  for (int it = 0; it < 4000; ++it) {
    const int tile = 8 << rnd(0, 2);
    const int R = (int)rnd(1, 6);
    std::vector<ddgs::ReqTab> req(R + 1);
    std::vector<ddgs::ViewTab> view;
    int64_t tiles = 0;
    for (int r = 0; r < R; ++r) {
      req[r].n = rnd(0, 3) == 0 ? 0 : rnd(1, it % 7 == 0 ? 3000000 : 20000);
      const int nv = (int)rnd(0, it % 11 == 0 ? 300 : 8);
      for (int k = 0; k < nv; ++k) {
        ddgs::ViewTab t{};
        t.req = r;
        const int shape = (int)rnd(0, 3);
        t.H = shape == 0 ? (int)rnd(1, 64) : shape == 1 ? (int)rnd(1, 2048) : shape == 2 ? 8 : (int)rnd(1, 4096);
        t.W = shape == 2 ? (int)rnd(1, 300000) : (int)rnd(1, 4096);
        t.tiles_x = (t.W + tile - 1) / tile;
        t.tile_base = tiles;
        tiles += (int64_t)t.tiles_x * ((t.H + tile - 1) / tile);
        view.push_back(t);
      }
    }
    const int V = (int)view.size();
    view.push_back(ddgs::ViewTab{});
    view[V].tile_base = tiles;
    const int64_t budget = rnd(0, 1) ? ddgs::BIN_SLOT_BUDGET : (int64_t(1) << 18);
    ddgs::RenderShape s{};
    ddgs::plan_binning(view.data(), V, req.data(), tiles, tile, s, budget);
    int64_t items = 0, slots = 0;
    for (int v = 0; v < V; ++v) {
      const ddgs::ViewTab &t = view[v];
      const int64_t tx = t.tiles_x, ty = (t.H + tile - 1) / tile, n = req[t.req].n;
      const int64_t bx = t.bands_x, by = (ty + t.band_h - 1) / t.band_h;
      if ((n == 0) != (t.chunks == 0)) { printf("FAIL chunks %d for n %lld\n", t.chunks, (long long)n); return 1; }
      if ((int64_t)t.band_w * t.band_h > ddgs::BIN_HIST_MAX) { printf("FAIL band too large\n"); return 1; }
      if ((int64_t)t.band_w * bx < tx || (int64_t)t.band_h * by < ty) { printf("FAIL bands do not cover the view\n"); return 1; }
      if (bx != (tx + t.band_w - 1) / t.band_w) { printf("FAIL bands_x\n"); return 1; }
      if (t.item_base != items || t.hist_base != slots) { printf("FAIL bases\n"); return 1; }
      items += (int64_t)t.chunks * bx * by;
      slots += (int64_t)t.chunks * bx * by * t.band_w * t.band_h;
      if (t.chunks > 0 && (int64_t)t.band_w * t.band_h > s.hist_area) { printf("FAIL hist_area\n"); return 1; }
    }
    if (items != s.n_items || slots != s.hist_slots || view[V].item_base != items) { printf("FAIL totals\n"); return 1; }
    if (s.hist_slots >= ddgs::hist_slot_bound(tiles, budget)) {
      printf("FAIL slots %lld >= bound %lld (tiles %lld)\n", (long long)s.hist_slots,
             (long long)ddgs::hist_slot_bound(tiles, budget), (long long)tiles);
      return 1;
    }
    ++layouts;
  }
  printf("ok %d\n", layouts);
  return 0;
}
"""


def test_binning_plan_covers_views_and_stays_within_the_counter_bound(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "plan.cu"
    src.write_text(_PROGRAM)
    exe = tmp_path / "plan"
    inc = os.path.join(ROOT, "paper_2406_02518_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", inc, "-I",
                    os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True, timeout=300)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok 4000")
