// Host-side schedule of the batched 2D step: the order of the batch's tiles
// and their split over the resident CTAs (plain C++, no CUDA: the library's
// plan builder and the host tests compile it).
#pragma once

#include <algorithm>
#include <vector>

namespace lbk {

// One run of a batched CTA's work: the tiles first, first + stride, ...
// (count of them) of instance inst, numbered row-major within the instance.
struct BatchSeg {
  int inst, first, stride, count;
};

// The order of the batch's tiles and their split over the G resident CTAs.
// The instances' tiles (tiles[i] of instance i, row-major) are cut into
// chunks of K consecutive tiles, so that a CTA steps K neighbours in a row one
// after another (the pushes across their common edges meet in L2 while the
// sectors are still there).  order 1: the instances one after another.
// order 0: instances of at most a quarter of a wave (G K / 4 tiles) one after
// another, then the chunks of the larger ones round after round over those
// instances (chunk q of every instance that has one, then chunk q + 1, ...),
// so that every large instance is stepped as a band of rows that moves
// through it while all of them advance together.  Which order is faster
// depends on the mix (measured on 16 equal 512^2 FP16 instances: order 0;
// on 64 uneven 256^2..768^2 ones: order 1); the tuner times both.  CTA b
// takes chunks b, b + G, b + 2G, ... of the list, as the single-instance
// step's CTAs take tiles, so every CTA gets a mix of instances and of edge
// and interior tiles.  K is the largest of 8, 4, 2, 1 that still gives every
// CTA at least 16 chunks (balance within one chunk in sixteen); one instance
// takes K = 1, which is the single-instance step's walk.  A CTA's consecutive
// tiles of one instance at a constant stride form one run.  Out: the runs CTA
// after CTA, and per CTA the index of its first run (cta_seg[b] ..
// cta_seg[b + 1]).
inline void batch_schedule(const std::vector<int>& tiles, int G, int order, std::vector<BatchSeg>* segs,
                    std::vector<int>* cta_seg) {
  const int n = int(tiles.size());
  long long total = 0;
  int maxt = 0;
  for (int t : tiles) {
    total += t;
    maxt = std::max(maxt, t);
  }
  int K = 1;
  if (n > 1)
    for (int k : {8, 4, 2})
      if (total >= 16LL * k * G) {
        K = k;
        break;
      }
  struct Chunk {
    int inst, first, count;
  };
  std::vector<Chunk> chunks;
  auto small = [&](int i) { return order == 1 || 4LL * tiles[i] <= (long long)G * K; };
  for (int i = 0; i < n; ++i)  // instances within a quarter of a wave: one after another
    if (small(i))
      for (int q = 0; q * K < tiles[i]; ++q)
        chunks.push_back({i, q * K, std::min(K, tiles[i] - q * K)});
  for (int q = 0; q * K < maxt; ++q)  // the others: round after round
    for (int i = 0; i < n; ++i)
      if (!small(i) && q * K < tiles[i]) chunks.push_back({i, q * K, std::min(K, tiles[i] - q * K)});
  const int nc = int(chunks.size());
  const int grid = std::min(G, nc);
  segs->clear();
  cta_seg->assign(1, 0);
  for (int b = 0; b < grid; ++b) {
    BatchSeg run{-1, 0, 1, 0};
    auto add = [&](int inst, int t) {
      if (run.count > 0 && run.inst == inst) {
        const int last = run.first + (run.count - 1) * run.stride;
        if (run.count == 1 && t > last) {
          run.stride = t - last;
          ++run.count;
          return;
        }
        if (t - last == run.stride) {
          ++run.count;
          return;
        }
      }
      if (run.count > 0) segs->push_back(run);
      run = BatchSeg{inst, t, 1, 1};
    };
    for (int q = b; q < nc; q += grid)
      for (int r = 0; r < chunks[q].count; ++r) add(chunks[q].inst, chunks[q].first + r);
    if (run.count > 0) segs->push_back(run);
    cta_seg->push_back(int(segs->size()));
  }
}

}  // namespace lbk
