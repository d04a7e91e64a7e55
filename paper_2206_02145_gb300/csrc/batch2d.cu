// Batched 2D step: many independent instances (different grids, parameters
// and seeds) advanced by ONE persistent launch per time step.  The host orders
// the instances' tiles and splits them over the resident CTAs once per plan
// (batch_schedule): every CTA gets runs of tiles, each of one instance, and
// feeds its pipeline with that instance's TMA descriptors (kept in global
// memory).  The per-tile work is exactly the
// single-grid kernel's (step2d_tile.cuh), so a batched instance evolves bit
// for bit like the same instance stepped alone.
//
// Several tile shapes / pipeline depths are compiled; the host times them on
// the live batch (all produce the same bits) and keeps the fastest.
#include <algorithm>
#include <vector>

#include "batch2d_kernels.cuh"
#include "tma_host.h"

namespace lbk {
namespace {

cudaError_t dispatch_any(int storage, int flow, int v, bool mask, bool chm, bool setup, int* ctas,
                         int* smem, const BatchDesc* d, const BatchSeg* sg, const int* cs,
                         int grid, cudaStream_t s) {
  switch (storage) {
    case ST_FP16:
      return batch_dispatch_fp16(flow, v, mask, chm, setup, ctas, smem, d, sg, cs, grid, s);
    case ST_BF16:
      return batch_dispatch_bf16(flow, v, mask, chm, setup, ctas, smem, d, sg, cs, grid, s);
    default:
      return batch_dispatch_fp32(flow, v, mask, chm, setup, ctas, smem, d, sg, cs, grid, s);
  }
}


// the solid flags of one instance's TX x TY tiles (tile or one-node halo holds
// a solid node), into flags[0 .. ntx * nty)
__global__ void batch_solid_tiles_kernel(const Model m, unsigned char* flags, int ntx, int nty,
                                         int tx, int ty) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntx * nty) return;
  const int x0 = (t % ntx) * tx, y0 = (t / ntx) * ty;
  bool any = false;
  for (int ly = -1; ly <= ty; ++ly)
    for (int lx = -1; lx <= tx; ++lx) any |= solid_mapped(m, x0 + lx, y0 + ly);
  flags[t] = any ? 1 : 0;
}

}  // namespace

int batch_variant_count() { return batch::kNumVariants; }
int batch_variant_rows(int v) { return batch::kVariants[v].ty; }
int batch_variant_stages(int v) { return batch::kVariants[v].stages; }

cudaError_t batch_plan_build(const BatchMember* members, int count, int storage, int flow, int v,
                             int order, BatchPlan* plan) {
  const int ty = batch::kVariants[v].ty, tx = 32;
  const size_t es = storage == ST_FP32 ? 4 : 2;
  const int qfg = (flow ? 9 : 0) + 9;
  const int hx = int(16 / es);
  std::vector<BatchDesc> host[2];
  std::vector<int> tiles;
  int tile0 = 0;
  bool mask = false;
  for (int i = 0; i < count; ++i) mask = mask || members[i].m.solid != nullptr;
  int all_tiles = 0;
  for (int i = 0; i < count; ++i)
    all_tiles += ((members[i].m.nx + tx - 1) / tx) * ((members[i].m.ny + ty - 1) / ty);
  cudaError_t e;
  if (mask) {  // (the masks were written on the instances' streams)
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    if ((e = cudaMalloc(&plan->solid_tiles, size_t(all_tiles))) != cudaSuccess) return e;
    if ((e = cudaMemset(plan->solid_tiles, 0, size_t(all_tiles))) != cudaSuccess) return e;
  }
  for (int i = 0; i < count; ++i) {
    const Model& m = members[i].m;
    const int ntx = (m.nx + tx - 1) / tx, nty = (m.ny + ty - 1) / ty;
    for (int c = 0; c < 2; ++c) {
      BatchDesc d{};
      const uint64_t dims3[3] = {uint64_t(m.nx), uint64_t(m.ny), uint64_t(qfg + 9)};
      const uint64_t str3[2] = {uint64_t(m.px) * es, uint64_t(m.plane) * es};
      const uint32_t box_fg[3] = {uint32_t(tx), uint32_t(ty), uint32_t(qfg)};
      const uint32_t box_h[3] = {uint32_t(tx + 2 * hx), uint32_t(ty + 2), 9};
      const uint64_t dims2[2] = {uint64_t(m.nx), uint64_t(m.ny)};
      const uint64_t str2[1] = {uint64_t(m.px) * 4};
      const uint32_t box_r[2] = {uint32_t(tx), uint32_t(ty)};
      if (!encode_tiled(&d.fg, pop_tensor_type(storage), 3, members[i].pops[c], dims3, str3,
                        box_fg) ||
          !encode_tiled(&d.h, pop_tensor_type(storage), 3, members[i].pops[c], dims3, str3,
                        box_h) ||
          !encode_tiled(&d.ring, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, members[i].rings[c], dims2,
                        str2, box_r))
        return cudaErrorInvalidValue;
      if (es == 2) {  // the two per-node U planes of 16-bit storage (g reference)
        const uint64_t dimsu[3] = {uint64_t(m.nx), uint64_t(m.ny), 2};
        const uint64_t stru[2] = {uint64_t(m.px) * 2, uint64_t(m.plane) * 2};
        const uint32_t box_uo[3] = {uint32_t(tx), uint32_t(ty), 1};
        const uint32_t box_uh[3] = {uint32_t(tx + 16), uint32_t(ty + 2), 1};
        if (!m.rel_g || !m.uring ||
            !encode_tiled(&d.uown, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, m.uring, dimsu, stru,
                          box_uo) ||
            !encode_tiled(&d.uhal, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, m.uring, dimsu, stru,
                          box_uh))
          return cudaErrorInvalidValue;
      }
      d.m = m;
      if (m.solid) d.m.solid_tiles = plan->solid_tiles + tile0;
      d.c = c;
      d.src = members[i].pops[c];
      d.dst = members[i].pops[c ^ 1];
      d.ring_cur = static_cast<float*>(members[i].rings[c ^ 1]);
      d.err = members[i].err;
      d.ntx = ntx;
      host[c].push_back(d);
    }
    tiles.push_back(ntx * nty);
    if (m.solid) {
      batch_solid_tiles_kernel<<<(ntx * nty + 127) / 128, 128>>>(m, plan->solid_tiles + tile0, ntx,
                                                                  nty, tx, ty);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    tile0 += ntx * nty;
  }
  plan->total_tiles = tile0;
  plan->variant = v;
  plan->storage = storage;
  plan->flow = flow;
  plan->mask = mask;
  plan->chm = members[0].m.chm;
  for (int c = 0; c < 2; ++c) {
    if ((e = cudaMalloc(&plan->desc[c], sizeof(BatchDesc) * count)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(plan->desc[c], host[c].data(), sizeof(BatchDesc) * count,
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return e;
  }
  // the resident CTAs of this variant, then the split of the tiles over them
  if ((e = dispatch_any(storage, flow, v, plan->mask, plan->chm, true, &plan->ctas, &plan->smem,
                        nullptr, nullptr, nullptr, 0, nullptr)) != cudaSuccess)
    return e;
  std::vector<BatchSeg> segs;
  std::vector<int> cta_seg;
  batch_schedule(tiles, plan->ctas, order, &segs, &cta_seg);
  plan->order = order;
  plan->grid = int(cta_seg.size()) - 1;
  if ((e = cudaMalloc(&plan->segs, sizeof(BatchSeg) * segs.size())) != cudaSuccess) return e;
  if ((e = cudaMemcpy(plan->segs, segs.data(), sizeof(BatchSeg) * segs.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  if ((e = cudaMalloc(&plan->cta_seg, sizeof(int) * cta_seg.size())) != cudaSuccess) return e;
  if ((e = cudaMemcpy(plan->cta_seg, cta_seg.data(), sizeof(int) * cta_seg.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  if (mask && (e = cudaDeviceSynchronize()) != cudaSuccess) return e;
  plan->bytes = 2 * sizeof(BatchDesc) * count + sizeof(BatchSeg) * segs.size() +
                sizeof(int) * cta_seg.size() + (mask ? size_t(all_tiles) : 0);
  return cudaSuccess;
}

cudaError_t batch_plan_launch(const BatchPlan& plan, int c, cudaStream_t s) {
  int ctas = plan.ctas, smem = plan.smem;
  return dispatch_any(plan.storage, plan.flow, plan.variant, plan.mask, plan.chm, false, &ctas,
                      &smem, plan.desc[c], plan.segs, plan.cta_seg, plan.grid, s);
}

void batch_plan_free(BatchPlan* plan) {
  for (int c = 0; c < 2; ++c)
    if (plan->desc[c]) cudaFree(plan->desc[c]);
  if (plan->segs) cudaFree(plan->segs);
  if (plan->cta_seg) cudaFree(plan->cta_seg);
  if (plan->solid_tiles) cudaFree(plan->solid_tiles);
  *plan = BatchPlan{};
}

}  // namespace lbk
