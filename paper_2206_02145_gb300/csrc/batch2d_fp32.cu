// Batched 2D step: the kernel variants of FP32 population storage.
#include "batch2d_kernels.cuh"

namespace lbk {

cudaError_t batch_dispatch_fp32(int flow, int v, bool mask, bool chm, bool setup, int* ctas,
                              int* smem, const BatchDesc* d, const BatchSeg* segs,
                              const int* cta_seg, int grid, cudaStream_t s) {
  return batch::dispatch_storage<float>(flow, v, mask, chm, setup, ctas, smem, d, segs, cta_seg,
                                       grid, s);
}

}  // namespace lbk
