// Launchers of the U-Net surrogate kernels (unet.cu).  NHWC bf16 tensors;
// `C*` is the channel stride of a buffer and `*off` the first channel used,
// so that concatenated buffers need no copies.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pdl.cuh"

namespace lbk {
namespace nn {

using bf16 = __nv_bfloat16;

// the network's kernels follow one another with programmatic dependent
// launch (pdl.cuh)
using lbk::launch_pdl;
using lbk::pdl_trigger;
using lbk::pdl_wait;

struct ConvArgs {
  const bf16* x;   // [N][H][W][Cx], channels ci_off .. ci_off + Cin
  int Cx, ci_off, Cin;
  const bf16* w;   // [9][Cout][Cin] (tap-major, input channels innermost)
  const float* bias;  // [Cout] or null
  bf16* y;         // [N][H][W][Cy], channels co_off .. co_off + Cout
  int Cy, co_off, Cout;
  int N, H, W;
  int relu;            // apply max(0, .) to the output
  const bf16* mask;    // zero the output where mask <= 0 (same layout as y), or null
  int tensor_path;     // 1: tcgen05 kernel (conv_tc.cu) where the shape allows; 0: mma.sync
  unsigned* err;       // device word: bit 2 set if a tcgen05 kernel timed out waiting
  // optional 1x1 head on the output (head_y null: none), computed in the
  // convolution's epilogue where its tiling allows (*head_done = 1), else
  // left to the caller (*head_done = 0): head_y [N][H][W][head_out] FP32,
  // head_w [head_out][Cout], head_b [head_out]
  const float* head_w;
  const float* head_b;
  float* head_y;
  int head_out;
  int* head_done;
  // optional 2 x 2 average pooling of the output (pool_y null: none), in the
  // epilogue where the tiling allows (*pool_done = 1): pool_y
  // [N][H/2][W/2][pool_Cy], channels pool_off .. pool_off + Cout
  bf16* pool_y;
  int pool_Cy, pool_off;
  int* pool_done;
};
// requirements: W % 64 == 0, Cin % 16 == 0, Cout % 32 == 0, strides/offsets % 8 == 0
cudaError_t conv3x3(const ConvArgs& a, cudaStream_t s);
// the tcgen05 / TMEM / TMA kernel: W % 128 == 0 (or W == 64 with H even),
// N H W % 128 == 0, Cin % 16 == 0, Cout % 32 == 0 and <= 256, strides / offsets % 8 == 0
bool conv3x3_tc_supported(const ConvArgs& a);
cudaError_t conv3x3_tc(const ConvArgs& a, unsigned* err, cudaStream_t s);

struct WgradArgs {
  const bf16* x;   // layer input, as in ConvArgs
  int Cx, ci_off, Cin;
  const bf16* dy;  // gradient of the layer's pre-activation [N][H][W][Cdy], channels co_off..
  int Cdy, co_off, Cout;
  float* dw;       // [9][Cout][Cin] FP32, accumulated (+=)
  float* db;       // [Cout] FP32 bias gradient sum of dy, accumulated (+=); null: not formed
  long long npix;  // N * H * W
  int H, W;
  int chunk;       // pixels per CTA (multiple of 16) of the per-tap kernel
  // scratch for the partial sums (floats, wgrad_scratch of the layer), owned
  // by the caller, so that dw and db are summed in a fixed order; too small
  // or null: the per-tap kernel with atomics, and no bias gradient (error)
  float* part;
  size_t part_cap;
};
cudaError_t wgrad3x3(const WgradArgs& a, cudaStream_t s);
// floats of scratch wgrad3x3 needs for a layer (the nine-tap kernel's
// partials where its shape allows it, else the per-tap kernel's partials at
// `chunk` pixels per chunk and the bias partials) for sums in a fixed order
size_t wgrad_scratch(int Cout, int Cin, int N, int H, int W, int chunk);

// db[c] += sum over the pixels of g[p][off + c], in a fixed order through
// part (at least bias_grad_scratch(C, npix) floats)
size_t bias_grad_scratch(int C, long long npix);
cudaError_t bias_grad(const bf16* g, int Cg, int off, int C, long long npix, float* db,
                      float* part, size_t part_cap, cudaStream_t s);
cudaError_t relu_mask(bf16* g, int Cg, int goff, const bf16* act, int Ca, int aoff, int C,
                      long long npix, cudaStream_t s);
cudaError_t avgpool2(const bf16* x, int Cx, int xoff, bf16* y, int Cy, int yoff, int C, int B,
                     int H, int W, cudaStream_t s);
cudaError_t avgpool2_bwd_add_mask(bf16* gs, const bf16* gp, const bf16* act, int Cs, int soff,
                                  int C, int B, int H, int W, cudaStream_t s);
cudaError_t upsample2(const bf16* x, bf16* y, int C, int B, int H, int W, cudaStream_t s);
cudaError_t upsample2_bwd_mask(const bf16* g, bf16* gx, const bf16* act, int C, int B, int H,
                               int W, cudaStream_t s);
cudaError_t head_fwd(const bf16* x, int C, const float* w, const float* b, float* y, int O,
                     long long npix, cudaStream_t s);
// scratch of head_bwd (floats): per block its dw and db sums
size_t head_bwd_scratch(int C, int O, long long npix);
cudaError_t head_bwd(const bf16* x, int C, const float* w, const float* gy, int O, long long npix,
                     bf16* gx, float* dw, float* db, float* part, size_t part_cap,
                     cudaStream_t s);
cudaError_t mse(const float* y, const float* t, long long n, float* gy, float* loss,
                cudaStream_t s);
// Multi-tensor launches: a table in device memory lists the tensors, each
// covering ceil(n / kSegBlock) consecutive blocks starting at block blk0
// (blk0 ascending from 0); `blocks` is the sum over the table.
constexpr int kSegBlock = 1024;  // values per block
struct AdamSeg {  // one parameter tensor: FP32 value, gradient, moments, bf16 copy (or null)
  float *w, *g, *m, *v;
  bf16* wb;
  long long n, blk0;
};
struct FlipSeg {  // one convolution's weights [9][cout][cin] and their flip-transpose
  const bf16* w;
  bf16* wt;
  int cout, cin;
  long long blk0;
};
// Adam step t (bias-corrected) over every tensor of the table; clears the gradients
cudaError_t adam_multi(const AdamSeg* segs, int nseg, long long blocks, float lr, float b1,
                       float b2, float eps, int t, cudaStream_t s);
// wt[8 - tap][ci][co] = w[tap][co][ci] for every convolution of the table
cudaError_t flip_multi(const FlipSeg* segs, int nseg, long long blocks, cudaStream_t s);

}  // namespace nn
}  // namespace lbk
