// Batched 2D step: many independent instances (different grids, parameters
// and seeds) advanced by ONE persistent launch per time step.  The tiles of
// all instances form one work list; a CTA walks it round-robin, looks up the
// instance of each tile in a tile -> instance table, and feeds its pipeline
// with that instance's TMA descriptors (kept in global memory).  The per-tile
// work is exactly the single-grid kernel's (step2d_tile.cuh), so a batched
// instance evolves bit for bit like the same instance stepped alone.
//
// Several tile shapes / pipeline depths are compiled; the host times them on
// the live batch (all produce the same bits) and keeps the fastest.
#include <vector>

#include "step2d_tile.cuh"
#include "tma_host.h"

namespace lbk {
namespace {

constexpr int kBatchSpin = 1 << 22;

// registers held to 20 resident warps per SM (five CTAs of 32 x 4), the
// occupancy of the single-instance step
template <typename T, bool FLOW, int TX, int TY, int S>
__global__ void __launch_bounds__(TX* TY, (640 / (TX * TY)) > 2 ? 640 / (TX * TY) : 2)
    step2d_batch_kernel(const BatchDesc* __restrict__ descs,
                        const unsigned short* __restrict__ tile_inst, int total_tiles) {
  using L = Tiles2D<T, FLOW, TX, TY>;
  constexpr int NT = TX * TY, SX = TX + 2, SY = TY + 2;
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[S];
  __shared__ float sh_phi[SY][SX];
  __shared__ __align__(16) Model sm;  // model of the instance being computed
  __shared__ int cur_inst;
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int tid = threadIdx.x;
  const int first = blockIdx.x, G = gridDim.x;

  auto issue = [&](int tile, int s) {
    const BatchDesc& d = descs[tile_inst[tile]];
    const int lt = tile - d.tile0;
    issue_tile_2d<T, FLOW, TX, TY>(&d.fg, &d.h, &d.ring, &d.uown, &d.uhal, d.c, &full[s],
                                   smem + s * L::STAGE, (lt % d.ntx) * TX, (lt / d.ntx) * TY);
  };

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
    fence_barrier_init();
    cur_inst = -1;
  }
  __syncthreads();
  if (tid == 0)
    for (int k = 0; k < S; ++k)
      if (first + k * G < total_tiles) issue(first + k * G, k);

  for (int k = 0;; ++k) {
    const int tile = first + k * G;
    if (tile >= total_tiles) break;
    const int s = k % S;
    const bool ok = mbar_wait_bounded(&full[s], uint32_t((k / S) & 1), kBatchSpin);
    if (__syncthreads_or(!ok)) {
      // a tile never arrived: report on its instance, let copies land, stop
      if (tid == 0) {
        atomicOr(descs[tile_inst[tile]].err, 2u);
        for (int j = 1; j < S; ++j) {
          const int kk = k + j;
          if (first + kk * G < total_tiles)
            mbar_wait_bounded(&full[kk % S], uint32_t((kk / S) & 1), kBatchSpin);
        }
      }
      __syncthreads();
      return;
    }
    const int inst = tile_inst[tile];
    const BatchDesc& d = descs[inst];
    if (inst != cur_inst) {  // uniform: every thread read cur_inst after the last barrier
      const uint32_t* from = reinterpret_cast<const uint32_t*>(&d.m);
      uint32_t* to = reinterpret_cast<uint32_t*>(&sm);
      for (int w = tid; w < int(sizeof(Model) / 4); w += NT) to[w] = from[w];
      __syncthreads();
      if (tid == 0) cur_inst = inst;
    }
    const int lt = tile - d.tile0;
    tile_2d<T, FLOW, TX, TY, false, false>(sm, static_cast<const T*>(d.src), static_cast<T*>(d.dst),
                             d.ring_cur, d.err, (lt % d.ntx) * TX, (lt / d.ntx) * TY, d.c,
                             smem + s * L::STAGE, &sh_phi[0][0]);
    __syncthreads();  // stage s, sh_phi and sm are free again
    if (tid == 0 && tile + S * G < total_tiles) {
      fence_proxy_async_smem();
      issue(tile + S * G, s);
    }
  }
}

// Compiled variants: (tile rows, pipeline stages).
struct Variant {
  int ty, stages;
};
constexpr Variant kVariants[] = {{4, 2}, {8, 2}, {2, 3}, {4, 3}};
constexpr int kNumVariants = int(sizeof(kVariants) / sizeof(kVariants[0]));

template <typename T, bool FLOW, int TY, int S>
struct VariantImpl {
  static constexpr int TX = 32;
  using L = Tiles2D<T, FLOW, TX, TY>;
  static cudaError_t setup(int* ctas, int* smem) {
    auto kern = step2d_batch_kernel<T, FLOW, TX, TY, S>;
    *smem = S * L::STAGE + 128;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, *smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * TY, *smem)) !=
        cudaSuccess)
      return e;
    *ctas = sms * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
  }
  static cudaError_t launch(const BatchDesc* d, const unsigned short* ti, int total, int ctas,
                            int smem, cudaStream_t s) {
    const int grid = total < ctas ? total : ctas;
    step2d_batch_kernel<T, FLOW, TX, TY, S><<<grid, TX * TY, smem, s>>>(d, ti, total);
    return cudaGetLastError();
  }
};

template <typename T, bool FLOW>
cudaError_t dispatch(int v, bool setup, int* ctas, int* smem, const BatchDesc* d,
                     const unsigned short* ti, int total, cudaStream_t s) {
#define LBPF_VARIANT(I, TY, S)                                               \
  case I:                                                                    \
    return setup ? VariantImpl<T, FLOW, TY, S>::setup(ctas, smem)            \
                 : VariantImpl<T, FLOW, TY, S>::launch(d, ti, total, *ctas, *smem, s);
  switch (v) {
    LBPF_VARIANT(0, 4, 2)
    LBPF_VARIANT(1, 8, 2)
    LBPF_VARIANT(2, 2, 3)
    LBPF_VARIANT(3, 4, 3)
    default: return cudaErrorInvalidValue;
  }
#undef LBPF_VARIANT
}

cudaError_t dispatch_any(int storage, int flow, int v, bool setup, int* ctas, int* smem,
                         const BatchDesc* d, const unsigned short* ti, int total, cudaStream_t s) {
  switch (storage) {
    case ST_FP16:
      return flow ? dispatch<__half, true>(v, setup, ctas, smem, d, ti, total, s)
                  : dispatch<__half, false>(v, setup, ctas, smem, d, ti, total, s);
    case ST_BF16:
      return flow ? dispatch<__nv_bfloat16, true>(v, setup, ctas, smem, d, ti, total, s)
                  : dispatch<__nv_bfloat16, false>(v, setup, ctas, smem, d, ti, total, s);
    default:
      return flow ? dispatch<float, true>(v, setup, ctas, smem, d, ti, total, s)
                  : dispatch<float, false>(v, setup, ctas, smem, d, ti, total, s);
  }
}

}  // namespace

int batch_variant_count() { return kNumVariants; }
int batch_variant_rows(int v) { return kVariants[v].ty; }
int batch_variant_stages(int v) { return kVariants[v].stages; }

cudaError_t batch_plan_build(const BatchMember* members, int count, int storage, int flow, int v,
                             BatchPlan* plan) {
  const int ty = kVariants[v].ty, tx = 32;
  const size_t es = storage == ST_FP32 ? 4 : 2;
  const int qfg = (flow ? 9 : 0) + 9;
  const int hx = int(16 / es);
  std::vector<BatchDesc> host[2];
  std::vector<unsigned short> inst;
  int tile0 = 0;
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
      d.c = c;
      d.src = members[i].pops[c];
      d.dst = members[i].pops[c ^ 1];
      d.ring_cur = static_cast<float*>(members[i].rings[c ^ 1]);
      d.err = members[i].err;
      d.ntx = ntx;
      d.tile0 = tile0;
      d.ntiles = ntx * nty;
      host[c].push_back(d);
    }
    for (int t = 0; t < ntx * nty; ++t) inst.push_back((unsigned short)i);
    tile0 += ntx * nty;
  }
  plan->total_tiles = tile0;
  plan->variant = v;
  plan->storage = storage;
  plan->flow = flow;
  cudaError_t e;
  for (int c = 0; c < 2; ++c) {
    if ((e = cudaMalloc(&plan->desc[c], sizeof(BatchDesc) * count)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(plan->desc[c], host[c].data(), sizeof(BatchDesc) * count,
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return e;
  }
  if ((e = cudaMalloc(&plan->tile_inst, sizeof(unsigned short) * inst.size())) != cudaSuccess)
    return e;
  if ((e = cudaMemcpy(plan->tile_inst, inst.data(), sizeof(unsigned short) * inst.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  plan->bytes = 2 * sizeof(BatchDesc) * count + sizeof(unsigned short) * inst.size();
  return dispatch_any(storage, flow, v, true, &plan->ctas, &plan->smem, nullptr, nullptr, 0,
                      nullptr);
}

cudaError_t batch_plan_launch(const BatchPlan& plan, int c, cudaStream_t s) {
  int ctas = plan.ctas, smem = plan.smem;
  return dispatch_any(plan.storage, plan.flow, plan.variant, false, &ctas, &smem, plan.desc[c],
                      plan.tile_inst, plan.total_tiles, s);
}

void batch_plan_free(BatchPlan* plan) {
  for (int c = 0; c < 2; ++c)
    if (plan->desc[c]) cudaFree(plan->desc[c]);
  if (plan->tile_inst) cudaFree(plan->tile_inst);
  *plan = BatchPlan{};
}

}  // namespace lbk
