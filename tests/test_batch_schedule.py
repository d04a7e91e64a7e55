"""The batched step's host schedule (csrc/batch_schedule.h), compiled here
as plain C++: for random mixes of instance sizes and resident-CTA counts,
both tile orders cover every tile of every instance exactly once, each CTA
gets at least one run and its runs stay inside their instances, no more CTAs
than resident ones are used, and (with no more instances than CTAs) no CTA
carries more than an eighth above an even split plus two chunks (K <= 8)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2206_02145_gb300", "csrc")

PROG = r'''
#include <cstdio>
#include <random>
#include "batch_schedule.h"
int main() {
  std::mt19937 rng(7);
  int bad = 0;
  for (int trial = 0; trial < 3000 && bad < 5; ++trial) {
    const int n = 1 + rng() % (trial % 5 == 0 ? 1500 : 90);
    const int G = 1 + rng() % 900;
    std::vector<int> tiles(n);
    for (int& t : tiles) t = 1 + rng() % (trial % 3 == 0 ? 5000 : 200);
    for (int order = 0; order < 2; ++order) {
      std::vector<lbk::BatchSeg> segs;
      std::vector<int> cs;
      lbk::batch_schedule(tiles, G, order, &segs, &cs);
      const int grid = int(cs.size()) - 1;
      if (grid < 1 || grid > G || cs[0] != 0 || cs[grid] != int(segs.size())) {
        printf("trial %d order %d: grid %d of %d\n", trial, order, grid, G); ++bad; continue;
      }
      std::vector<std::vector<int>> hit(n);
      long long total = 0, maxload = 0;
      for (int i = 0; i < n; ++i) { hit[i].assign(tiles[i], 0); total += tiles[i]; }
      for (int b = 0; b < grid; ++b) {
        if (cs[b + 1] <= cs[b]) { printf("trial %d: CTA %d has no run\n", trial, b); ++bad; }
        long long load = 0;
        for (int r = cs[b]; r < cs[b + 1]; ++r) {
          const lbk::BatchSeg& g = segs[r];
          if (g.inst < 0 || g.inst >= n || g.count < 1 || g.stride < 1) { ++bad; continue; }
          for (int k = 0; k < g.count; ++k) {
            const long long t = g.first + (long long)k * g.stride;
            if (t < 0 || t >= tiles[g.inst]) { printf("trial %d: tile outside\n", trial); ++bad; break; }
            ++hit[g.inst][t];
          }
          load += g.count;
        }
        if (load > maxload) maxload = load;
      }
      for (int i = 0; i < n; ++i)
        for (int t = 0; t < tiles[i]; ++t)
          if (hit[i][t] != 1) { printf("trial %d: tile %d of %d seen %d times\n", trial, t, i, hit[i][t]); ++bad; i = n; break; }
      const long long even = (total + grid - 1) / grid;
      if (maxload > even + even / 8 + 16 && n <= G) { printf("trial %d: load %lld against %lld\n", trial, maxload, even); ++bad; }
    }
  }
  printf(bad ? "FAIL\n" : "ok\n");
  return bad != 0;
}
'''


def test_schedule_covers_every_tile_once_and_balances(tmp_path):
    src = tmp_path / "sched.cc"
    src.write_text(PROG)
    exe = tmp_path / "sched"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", HDR, "-o", str(exe), str(src)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout[-2000:]
