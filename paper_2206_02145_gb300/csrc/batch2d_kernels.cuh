// The batched 2D step kernel and its compiled variants (tile rows, pipeline
// stages, solid-node path, flow collision).  Each storage type's variants are
// instantiated in a translation unit of their own (batch2d_fp32.cu,
// batch2d_fp16.cu, batch2d_bf16.cu) so that they compile in parallel; the host
// side (batch2d.cu) reaches them through batch_dispatch_<storage>.
#pragma once

#include "step2d_tile.cuh"

namespace lbk {
namespace batch {

constexpr int kBatchSpin = 1 << 22;

// Registers held to 20 resident warps per SM (five CTAs of 32 x 4), the
// occupancy of the single-instance step.  MASK: solid nodes (each instance's
// model points at the per-tile flags of this variant's tiles); CHM: the
// central Hermite MRT flow collision.
template <typename T, bool FLOW, int TX, int TY, int S, bool MASK, bool CHM>
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
    tile_2d<T, FLOW, TX, TY, MASK, CHM>(sm, static_cast<const T*>(d.src), static_cast<T*>(d.dst),
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

template <typename T, bool FLOW, int TY, int S, bool MASK, bool CHM>
struct VariantImpl {
  static constexpr int TX = 32;
  using L = Tiles2D<T, FLOW, TX, TY>;
  static cudaError_t setup(int* ctas, int* smem) {
    auto kern = step2d_batch_kernel<T, FLOW, TX, TY, S, MASK, CHM>;
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
    step2d_batch_kernel<T, FLOW, TX, TY, S, MASK, CHM><<<grid, TX * TY, smem, s>>>(d, ti, total);
    return cudaGetLastError();
  }
};

template <typename T, bool FLOW, bool MASK, bool CHM>
cudaError_t dispatch_v(int v, bool setup, int* ctas, int* smem, const BatchDesc* d,
                       const unsigned short* ti, int total, cudaStream_t s) {
#define LBPF_VARIANT(I, TY, S)                                                         \
  case I:                                                                              \
    return setup ? VariantImpl<T, FLOW, TY, S, MASK, CHM>::setup(ctas, smem)           \
                 : VariantImpl<T, FLOW, TY, S, MASK, CHM>::launch(d, ti, total, *ctas, *smem, s);
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
                     const BatchDesc* d, const unsigned short* ti, int total, cudaStream_t s) {
  if constexpr (FLOW) {
    if (chm)
      return mask ? dispatch_v<T, FLOW, true, true>(v, setup, ctas, smem, d, ti, total, s)
                  : dispatch_v<T, FLOW, false, true>(v, setup, ctas, smem, d, ti, total, s);
  }
  if (chm) return cudaErrorInvalidValue;  // the central Hermite MRT needs the flow lattice
  return mask ? dispatch_v<T, FLOW, true, false>(v, setup, ctas, smem, d, ti, total, s)
              : dispatch_v<T, FLOW, false, false>(v, setup, ctas, smem, d, ti, total, s);
}

// every variant of one storage type T
template <typename T>
cudaError_t dispatch_storage(int flow, int v, bool mask, bool chm, bool setup, int* ctas,
                             int* smem, const BatchDesc* d, const unsigned short* ti, int total,
                             cudaStream_t s) {
  return flow ? dispatch<T, true>(v, mask, chm, setup, ctas, smem, d, ti, total, s)
              : dispatch<T, false>(v, mask, chm, setup, ctas, smem, d, ti, total, s);
}

}  // namespace batch
}  // namespace lbk
