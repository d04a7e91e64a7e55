// The batched 2D step kernel and its compiled variants (tile rows, pipeline
// stages, solid-node path, flow collision).  Each storage type's variants are
// instantiated in a translation unit of their own (batch2d_fp32.cu,
// batch2d_fp16.cu, batch2d_bf16.cu) so that they compile in parallel; the host
// side (batch2d.cu) reaches them through batch_dispatch_<storage>.
#pragma once

#include <cstddef>

#include "step2d_tile.cuh"

namespace lbk {
namespace batch {

// announce `bytes` more incoming transactions on the current phase without
// arriving (the phase still waits for its arrival count)
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// untiled bulk copy global -> shared of `bytes` (both addresses 16-byte
// aligned, bytes a multiple of 16), completing on `bar`
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

constexpr int kBatchSpin = 1 << 22;

// What the computation of a stage needs besides its tile data, written by
// the thread that issues the stage's loads.
struct StageMeta {
  const void* src;
  void* dst;
  float* ring_cur;
  unsigned* err;
  int x0, y0, c, inst;
};
// bytes of an instance's model copied into a stage (16-byte multiple) and the
// stage's slot for it after the tile data
constexpr int kModelCopy = (int(sizeof(Model)) + 15) / 16 * 16;
constexpr int kModelSlot = (kModelCopy + 127) / 128 * 128;
static_assert(offsetof(BatchDesc, m) % 16 == 0 &&
                  offsetof(BatchDesc, m) + kModelCopy <= sizeof(BatchDesc),
              "the model copy must be an aligned span of the descriptor");

// Registers held to 20 resident warps per SM (five CTAs of 32 x 4), the
// occupancy of the single-instance step.  MASK: solid nodes (each instance's
// model points at the per-tile flags of this variant's tiles); CHM: the
// central Hermite MRT flow collision.
//
// CTA b works through its runs segs[cta_seg[b] .. cta_seg[b + 1]) tile by
// tile.  Thread 0 walks the runs S tiles ahead of the computation: per run it
// reads the run and its instance's buffers once, per tile it issues the
// tile's loads into a stage and writes the stage's StageMeta; when the
// stage's model slot holds another instance's model, the model is copied into
// it by the TMA with the tile data (same barrier).  The computation then reads
// everything from shared memory: no global lookups on a tile's critical path.
template <typename T, bool FLOW, int TX, int TY, int S, bool MASK, bool CHM>
__global__ void __launch_bounds__(TX* TY, (640 / (TX * TY)) > 2 ? 640 / (TX * TY) : 2)
    step2d_batch_kernel(const BatchDesc* __restrict__ descs, const BatchSeg* __restrict__ segs,
                        const int* __restrict__ cta_seg) {
  using L = Tiles2D<T, FLOW, TX, TY>;
  constexpr int SX = TX + 2, SY = TY + 2;
  constexpr int STAGE = L::STAGE + kModelSlot;
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[S];
  __shared__ float sh_phi[SY][SX];
  __shared__ StageMeta meta[S];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int tid = threadIdx.x;
  const int sb = cta_seg[blockIdx.x], se = cta_seg[blockIdx.x + 1];
  int ntiles = 0;  // this CTA's tiles (every thread)
  for (int r = sb; r < se; ++r) ntiles += segs[r].count;

  // thread 0: the next tile to load and the run it belongs to
  int is = sb, ik = 0, issued = 0, intx = 1, ic = 0;
  int slot_inst[S];
#pragma unroll
  for (int k = 0; k < S; ++k) slot_inst[k] = -1;
  BatchSeg ig{0, 0, 1, 0};
  const BatchDesc* id = descs;
  StageMeta im{};
  auto issue_next = [&](int s) {
    if (is >= se) return;
    if (ik == 0) {
      ig = segs[is];
      id = descs + ig.inst;
      intx = id->ntx;
      ic = id->c;
      im.src = id->src;
      im.dst = id->dst;
      im.ring_cur = id->ring_cur;
      im.err = id->err;
      im.c = ic;
      im.inst = ig.inst;
    }
    const int lt = ig.first + ik * ig.stride;
    im.x0 = (lt % intx) * TX;
    im.y0 = (lt / intx) * TY;
    meta[s] = im;
    unsigned char* st = smem + s * STAGE;
#pragma unroll
    for (int k = 0; k < S; ++k)
      if (k == s && slot_inst[k] != ig.inst) {
        mbar_expect_tx(&full[s], kModelCopy);
        bulk_load(st + L::STAGE, &id->m, kModelCopy, &full[s]);
        slot_inst[k] = ig.inst;
      }
    issue_tile_2d<T, FLOW, TX, TY>(&id->fg, &id->h, &id->ring, &id->uown, &id->uhal, ic,
                                   &full[s], st, im.x0, im.y0);
    ++issued;
    if (++ik == ig.count) {
      ++is;
      ik = 0;
    }
  };

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int k = 0; k < S; ++k) issue_next(k);

  for (int k = 0; k < ntiles; ++k) {
    const int s = k % S;
    const bool ok = mbar_wait_bounded(&full[s], uint32_t((k / S) & 1), kBatchSpin);
    // (a barrier: the issuing thread's StageMeta of stage s is visible after it)
    if (__syncthreads_or(!ok)) {
      // a tile never arrived: report on its instance, let copies land, stop
      if (tid == 0) {
        atomicOr(meta[s].err, 2u);
        for (int j = k + 1; j < issued; ++j)
          mbar_wait_bounded(&full[j % S], uint32_t((j / S) & 1), kBatchSpin);
      }
      __syncthreads();
      return;
    }
    const StageMeta mt = meta[s];
    unsigned char* st = smem + s * STAGE;
    tile_2d<T, FLOW, TX, TY, MASK, CHM>(*reinterpret_cast<const Model*>(st + L::STAGE),
                                        static_cast<const T*>(mt.src), static_cast<T*>(mt.dst),
                                        mt.ring_cur, mt.err, mt.x0, mt.y0, mt.c, st,
                                        &sh_phi[0][0]);
    __syncthreads();  // stage s (tile data, model slot, meta) and sh_phi are free again
    if (tid == 0) {
      fence_proxy_async_smem();
      issue_next(s);
    }
  }
}

// Compiled variants: (tile rows, pipeline stages).
struct Variant {
  int ty, stages;
};
constexpr Variant kVariants[] = {{4, 2}, {8, 2}, {2, 3}, {4, 3}};
constexpr int kNumVariants = int(sizeof(kVariants) / sizeof(kVariants[0]));

template <typename T, bool FLOW, int TY, int S, bool MASK, bool CHM>
struct VariantImpl {
  static constexpr int TX = 32;
  using L = Tiles2D<T, FLOW, TX, TY>;
  static cudaError_t setup(int* ctas, int* smem) {
    auto kern = step2d_batch_kernel<T, FLOW, TX, TY, S, MASK, CHM>;
    *smem = S * (L::STAGE + kModelSlot) + 128;
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
  static cudaError_t launch(const BatchDesc* d, const BatchSeg* segs, const int* cta_seg,
                            int grid, int smem, cudaStream_t s) {
    step2d_batch_kernel<T, FLOW, TX, TY, S, MASK, CHM>
        <<<grid, TX * TY, smem, s>>>(d, segs, cta_seg);
    return cudaGetLastError();
  }
};

template <typename T, bool FLOW, bool MASK, bool CHM>
cudaError_t dispatch_v(int v, bool setup, int* ctas, int* smem, const BatchDesc* d,
                       const BatchSeg* segs, const int* cta_seg, int grid, cudaStream_t s) {
#define LBPF_VARIANT(I, TY, S)                                                          \
  case I:                                                                               \
    return setup ? VariantImpl<T, FLOW, TY, S, MASK, CHM>::setup(ctas, smem)            \
                 : VariantImpl<T, FLOW, TY, S, MASK, CHM>::launch(d, segs, cta_seg, grid, \
                                                                  *smem, s);
  switch (v) {
    LBPF_VARIANT(0, 4, 2)
    LBPF_VARIANT(1, 8, 2)
    LBPF_VARIANT(2, 2, 3)
    LBPF_VARIANT(3, 4, 3)
    default: return cudaErrorInvalidValue;
  }
#undef LBPF_VARIANT
}

template <typename T, bool FLOW>
inline cudaError_t dispatch(int v, bool mask, bool chm, bool setup, int* ctas, int* smem,
                            const BatchDesc* d, const BatchSeg* sg, const int* cs, int grid,
                            cudaStream_t s) {
  if constexpr (FLOW) {
    if (chm)
      return mask ? dispatch_v<T, FLOW, true, true>(v, setup, ctas, smem, d, sg, cs, grid, s)
                  : dispatch_v<T, FLOW, false, true>(v, setup, ctas, smem, d, sg, cs, grid, s);
  }
  if (chm) return cudaErrorInvalidValue;  // the central Hermite MRT needs the flow lattice
  return mask ? dispatch_v<T, FLOW, true, false>(v, setup, ctas, smem, d, sg, cs, grid, s)
              : dispatch_v<T, FLOW, false, false>(v, setup, ctas, smem, d, sg, cs, grid, s);
}

// every variant of one storage type T
template <typename T>
cudaError_t dispatch_storage(int flow, int v, bool mask, bool chm, bool setup, int* ctas,
                             int* smem, const BatchDesc* d, const BatchSeg* sg, const int* cs,
                             int grid, cudaStream_t s) {
  return flow ? dispatch<T, true>(v, mask, chm, setup, ctas, smem, d, sg, cs, grid, s)
              : dispatch<T, false>(v, mask, chm, setup, ctas, smem, d, sg, cs, grid, s);
}

}  // namespace batch
}  // namespace lbk
