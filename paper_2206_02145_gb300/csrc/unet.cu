// Kernels of the BF16 U-Net surrogate (NHWC bf16 activations, FP32
// accumulation and master weights):
//   conv3x3_kernel   implicit-GEMM 3x3 convolution on the warp-level mma.sync
//                    path (M = pixels, N = output channels, K = 9 x input
//                    channels); also the data gradient, run on flipped /
//                    transposed weights.  Shapes the tcgen05 kernel of
//                    conv_tc.cu takes go there instead.
//   wgrad3x3_kernel  weight gradient, K = pixels, split over CTAs, FP32 atomics
//   element-wise     bias gradient, ReLU masks, 2x2 average pooling and its
//                    gradient, nearest 2x upsampling and its gradient, the 1x1
//                    head, MSE loss, Adam, weight transposition, input packing
#include "lbpf_internal.cuh"
#include "unet.cuh"
#include "unet_ops.cuh"

namespace lbk {
namespace nn {
namespace {

constexpr int kThreads = 128;

// ---- 3x3 convolution, implicit GEMM ------------------------------------------------
// Tile: 64 pixels of one image row x BN output channels; 4 warps as 2 x 2,
// each 32 pixels x BN/2 channels (2 x BN/16 mma tiles).  K steps of 16 input
// channels of one tap, double-buffered through cp.async.
template <int BN>
__global__ void __launch_bounds__(kThreads) conv3x3_kernel(const ConvArgs a) {
  constexpr int BM = 64, LD = 24;  // 48-byte padded rows: conflict-free ldmatrix
  __shared__ __align__(16) bf16 sA[2][BM][LD];
  __shared__ __align__(16) bf16 sB[2][BN][LD];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp & 1, wn = warp >> 1;
  const int pix0 = blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int wcol = pix0 % a.W, hrow = (pix0 / a.W) % a.H, img = pix0 / (a.W * a.H);
  const int cchunks = a.Cin / 16, ksteps = 9 * cchunks;

  float acc[2][BN / 16][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < BN / 16; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

  auto load = [&](int ks, int buf) {
    const int tap = ks / cchunks, c0 = (ks % cchunks) * 16;
    const int ky = tap / 3, kx = tap % 3;
    {
      const int r = tid >> 1, half = tid & 1;
      const int hh = hrow + ky - 1, ww = wcol + r + kx - 1;
      const bool ok = hh >= 0 && hh < a.H && ww >= 0 && ww < a.W;
      const size_t pix = (size_t(img) * a.H + (ok ? hh : 0)) * a.W + (ok ? ww : 0);
      cp_async16(&sA[buf][r][half * 8], a.x + pix * a.Cx + a.ci_off + c0 + half * 8, ok ? 16 : 0);
    }
    for (int i = tid; i < BN * 2; i += kThreads) {
      const int r = i >> 1, half = i & 1;
      cp_async16(&sB[buf][r][half * 8],
                 a.w + (size_t(tap) * a.Cout + n0 + r) * a.Cin + c0 + half * 8, 16);
    }
    cp_async_commit();
  };

  load(0, 0);
  for (int ks = 0; ks < ksteps; ++ks) {
    const int buf = ks & 1;
    if (ks + 1 < ksteps) {
      load(ks + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    uint32_t af[2][4], bfr[BN / 16][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
      ldmatrix_x4(af[mt], &sA[buf][wm * 32 + mt * 16 + (lane & 15)][(lane >> 4) * 8]);
#pragma unroll
    for (int nt = 0; nt < BN / 16; ++nt)
      ldmatrix_x2(bfr[nt], &sB[buf][wn * (BN / 2) + nt * 8 + (lane & 7)][((lane >> 3) & 1) * 8]);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < BN / 16; ++nt) mma_bf16(acc[mt][nt], af[mt], bfr[nt]);
    __syncthreads();
  }
  // epilogue: bias, optional ReLU, optional mask (zero where mask <= 0), bf16 out
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < BN / 16; ++nt)
#pragma unroll
      for (int hlf = 0; hlf < 2; ++hlf) {
        const size_t p = size_t(pix0) + wm * 32 + mt * 16 + (lane >> 2) + hlf * 8;
        const int co = n0 + wn * (BN / 2) + nt * 8 + (lane & 3) * 2;
        float v0 = acc[mt][nt][hlf * 2 + 0], v1 = acc[mt][nt][hlf * 2 + 1];
        if (a.bias) {
          v0 += a.bias[co];
          v1 += a.bias[co + 1];
        }
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (a.mask) {
          const bf16* mk = a.mask + p * a.Cy + a.co_off + co;
          if (!(__bfloat162float(mk[0]) > 0.f)) v0 = 0.f;
          if (!(__bfloat162float(mk[1]) > 0.f)) v1 = 0.f;
        }
        *reinterpret_cast<__nv_bfloat162*>(a.y + p * a.Cy + a.co_off + co) =
            __floats2bfloat162_rn(v0, v1);
      }
}

// ---- weight gradient ---------------------------------------------------------------
// dW[tap][co][ci] += sum_p dy[p][co] x[p + shift(tap)][ci] over a chunk of
// pixels.  M = BM output channels, N = BN input channels; each pipeline stage
// holds KP pixels of dy and of the tap-shifted x ([pixel][channel] tiles,
// 16-byte cp.async, zero fill outside the image and past the chunk), S stages
// deep so that S - 1 stages are in flight while one is multiplied; the MMA
// steps K = 16 pixels through a stage with ldmatrix.trans.  4 warps as 2 x 2.
template <int BM, int BN, int KP, int S>
__global__ void __launch_bounds__(kThreads) wgrad3x3_kernel(const WgradArgs a) {
  constexpr int LDA = BM + 8, LDB = BN + 8;
  extern __shared__ __align__(16) unsigned char wg_smem[];
  bf16(*sA)[KP][LDA] = reinterpret_cast<bf16(*)[KP][LDA]>(wg_smem);
  bf16(*sB)[KP][LDB] = reinterpret_cast<bf16(*)[KP][LDB]>(wg_smem + S * KP * LDA * 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp & 1, wn = warp >> 1;
  constexpr int WM = BM / 2, WN = BN / 2;  // warp tile
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int tap = blockIdx.z % 9, chunk = blockIdx.z / 9;
  const int ky = tap / 3, kx = tap % 3;
  const long long p_begin = (long long)chunk * a.chunk;
  long long p_end = p_begin + a.chunk;
  if (p_end > a.npix) p_end = a.npix;
  const int ksteps = int((p_end - p_begin + KP - 1) / KP);

  float acc[WM / 16][WN / 8][4];
#pragma unroll
  for (int i = 0; i < WM / 16; ++i)
#pragma unroll
    for (int j = 0; j < WN / 8; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

  auto load = [&](int ks, int buf) {
    const long long pb = p_begin + (long long)ks * KP;
    for (int i = tid; i < KP * (BM / 8); i += kThreads) {
      const int r = i / (BM / 8), c = (i % (BM / 8)) * 8;
      const bool in = pb + r < p_end;
      cp_async16(&sA[buf][r][c], a.dy + (in ? pb + r : p_begin) * a.Cdy + a.co_off + m0 + c,
                 in ? 16 : 0);
    }
    for (int i = tid; i < KP * (BN / 8); i += kThreads) {
      const int r = i / (BN / 8), c = (i % (BN / 8)) * 8;
      const long long p = pb + r;
      const int w = int(p % a.W), h = int((p / a.W) % a.H);
      const long long img = p / ((long long)a.W * a.H);
      const int hh = h + ky - 1, ww = w + kx - 1;
      const bool ok = p < p_end && hh >= 0 && hh < a.H && ww >= 0 && ww < a.W;
      const long long q = ok ? (img * a.H + hh) * a.W + ww : 0;
      cp_async16(&sB[buf][r][c], a.x + q * a.Cx + a.ci_off + n0 + c, ok ? 16 : 0);
    }
  };
  // prologue: stages 0 .. S - 2 in flight (one commit group per stage, empty
  // groups past the end keep the counting uniform)
#pragma unroll
  for (int st = 0; st < S - 1; ++st) {
    if (st < ksteps) load(st, st);
    cp_async_commit();
  }
  for (int ks = 0; ks < ksteps; ++ks) {
    cp_async_wait<S - 2>();  // stage ks has landed
    __syncthreads();         // ... for every thread, and stage ks - 1 is free
    const int nxt = ks + S - 1;
    if (nxt < ksteps) load(nxt, nxt % S);
    cp_async_commit();
    const int buf = ks % S;
#pragma unroll
    for (int kk = 0; kk < KP; kk += 16) {
      uint32_t af[WM / 16][4], bfr[WN / 8][2];
#pragma unroll
      for (int mt = 0; mt < WM / 16; ++mt)
        ldmatrix_x4_t(af[mt], &sA[buf][kk + (lane & 7) + ((lane >> 4) << 3)]
                                  [wm * WM + mt * 16 + ((lane >> 3) & 1) * 8]);
#pragma unroll
      for (int nt = 0; nt < WN / 8; ++nt)
        ldmatrix_x2_t(bfr[nt], &sB[buf][kk + (lane & 15)][wn * WN + nt * 8]);
#pragma unroll
      for (int mt = 0; mt < WM / 16; ++mt)
#pragma unroll
        for (int nt = 0; nt < WN / 8; ++nt) mma_bf16(acc[mt][nt], af[mt], bfr[nt]);
    }
  }
  cp_async_wait<0>();
#pragma unroll
  for (int mt = 0; mt < WM / 16; ++mt)
#pragma unroll
    for (int nt = 0; nt < WN / 8; ++nt)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int co = m0 + wm * WM + mt * 16 + (lane >> 2) + (k >> 1) * 8;
        const int ci = n0 + wn * WN + nt * 8 + (lane & 3) * 2 + (k & 1);
        const size_t e = (size_t(tap) * a.Cout + co) * a.Cin + ci;
        if (a.part)  // this chunk's partial; summed over the chunks in a fixed order
          a.part[size_t(chunk) * 9 * a.Cout * a.Cin + e] = acc[mt][nt][k];
        else
          atomicAdd(a.dw + e, acc[mt][nt][k]);
      }
}

// out[i] += sum over p < nparts of part[p * stride + i], i < n, in a fixed
// order: a block takes 32 consecutive outputs, its 8 warps sum every 8th
// partial each, then warp 0 adds the 8 warp sums
__global__ void __launch_bounds__(256) sum_partials_kernel(const float* part, long long stride,
                                                           int nparts, int n, float* out) {
  __shared__ float red[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 32 + lane;
  float t = 0.f;
  if (i < n)
    for (int p = warp; p < nparts; p += 8) t += part[p * stride + i];
  red[warp][lane] = t;
  __syncthreads();
  if (warp == 0 && i < n) {
    float u = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) u += red[w][lane];
    out[i] += u;
  }
}
cudaError_t sum_partials(const float* part, long long stride, int nparts, int n, float* out,
                         cudaStream_t s) {
  if (n < 1 || nparts < 1) return cudaSuccess;
  sum_partials_kernel<<<(n + 31) / 32, 256, 0, s>>>(part, stride, nparts, n, out);
  return cudaGetLastError();
}

// Nine taps at once: a CTA owns a 32 x 32 (co, ci) tile of every tap and a
// run of `chunk` pixel patches of 2 image rows x 64 pixels.  Per patch it
// loads dy once ([128 px][32 co]) and x once as the patch with a one-pixel
// halo ([4 rows][66 px][32 ci], zero fill outside the image), both by
// cp.async into a double buffer; each K step of 16 pixels loads the dy
// fragment once and multiplies it by the nine tap-shifted x fragments (the
// shift is a row offset into the halo tile).  The nine 32 x 32 partial sums
// go to part[(tile * nchunks + chunk) * 9 * 1024 + ...].  The CTAs of the
// first input-channel tile (n0 = 0) also sum dy over their pixels, the bias
// gradient's partial, into part[bias_off + (co_tile * nchunks + chunk) * 32
// + co].  wgrad_reduce_kernel adds both over the chunks into dw and db in a
// fixed order (no atomics, so the result does not depend on the schedule).
constexpr int kWP = 128;                  // pixels per patch (2 rows x 64)
constexpr int kWHalo = 4 * 66;            // halo pixels per patch
constexpr int kWLD = 40;                  // smem row pitch (32 channels + 8)

__global__ void __launch_bounds__(kThreads) wgrad_taps_kernel(const WgradArgs a, int chunk,
                                                              int nchunks, int patches,
                                                              size_t bias_off) {
  extern __shared__ __align__(16) unsigned char wt_smem[];
  bf16(*sA)[kWP][kWLD] = reinterpret_cast<bf16(*)[kWP][kWLD]>(wt_smem);
  bf16(*sB)[kWHalo][kWLD] = reinterpret_cast<bf16(*)[kWHalo][kWLD]>(wt_smem + 2 * kWP * kWLD * 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp & 1, wn = warp >> 1;  // warp tile: 16 co x 16 ci
  const int ntn = a.Cin / 32;
  const int tile = blockIdx.x / nchunks, ck = blockIdx.x % nchunks;
  const int m0 = (tile / ntn) * 32, n0 = (tile % ntn) * 32;
  const int pbeg = ck * chunk;
  const int pend = min(pbeg + chunk, patches);
  const int pw = a.W / 64, ph = a.H / 2;  // patches per image row pair, per image column

  float acc[9][2][4];
#pragma unroll
  for (int t = 0; t < 9; ++t)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[t][j][k] = 0.f;

  // bias partial: thread (co pair tid & 15, pixel group tid >> 4 of 16 pixels)
  const bool with_bias = a.db != nullptr && n0 == 0;
  float bsum0 = 0.f, bsum1 = 0.f;
  auto load = [&](int pt, int buf) {
    const int img = pt / (pw * ph), r = pt % (pw * ph);
    const int h0 = (r / pw) * 2, w0 = (r % pw) * 64;
    for (int i = tid; i < kWP * 4; i += kThreads) {  // dy: 128 px x 4 x 8 channels
      const int px = i >> 2, c = (i & 3) * 8;
      const long long p = ((long long)img * a.H + h0 + (px >> 6)) * a.W + w0 + (px & 63);
      cp_async16(&sA[buf][px][c], a.dy + p * a.Cdy + a.co_off + m0 + c, 16);
    }
    for (int i = tid; i < kWHalo * 4; i += kThreads) {  // x halo: 4 x 66 px x 4 x 8
      const int hp = i >> 2, c = (i & 3) * 8;
      const int hh = h0 - 1 + hp / 66, ww = w0 - 1 + hp % 66;
      const bool ok = hh >= 0 && hh < a.H && ww >= 0 && ww < a.W;
      const long long q = ok ? ((long long)img * a.H + hh) * a.W + ww : 0;
      cp_async16(&sB[buf][hp][c], a.x + q * a.Cx + a.ci_off + n0 + c, ok ? 16 : 0);
    }
  };
  if (pbeg < pend) load(pbeg, 0);
  cp_async_commit();
  for (int pt = pbeg; pt < pend; ++pt) {
    const int buf = (pt - pbeg) & 1;
    if (pt + 1 < pend) load(pt + 1, buf ^ 1);
    cp_async_commit();
    cp_async_wait<1>();  // patch pt has landed
    __syncthreads();
    if (with_bias) {
      const int cp = tid & 15, pg = tid >> 4;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const __nv_bfloat162 v =
            *reinterpret_cast<const __nv_bfloat162*>(&sA[buf][pg * 16 + i][cp * 2]);
        bsum0 += __low2float(v);
        bsum1 += __high2float(v);
      }
    }
#pragma unroll 1
    for (int ks = 0; ks < kWP / 16; ++ks) {
      const int rr = ks >> 2, c0 = (ks & 3) * 16;  // row of the patch, first column
      uint32_t af[4];
      ldmatrix_x4_t(af, &sA[buf][ks * 16 + (lane & 7) + ((lane >> 4) << 3)]
                             [wm * 16 + ((lane >> 3) & 1) * 8]);
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const int ky = t / 3, kx = t % 3;
        const int hrow = (rr + ky) * 66 + c0 + kx;  // halo pixel of the first of the 16
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          uint32_t bfr[2];
          ldmatrix_x2_t(bfr, &sB[buf][hrow + (lane & 15)][wn * 16 + nt * 8]);
          mma_bf16(acc[t][nt], af, bfr);
        }
      }
    }
    __syncthreads();  // buffer buf is free for the load two patches on
  }
  float* out = a.part + (size_t(tile) * nchunks + ck) * 9 * 1024;
#pragma unroll
  for (int t = 0; t < 9; ++t)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int co = wm * 16 + (lane >> 2) + (k >> 1) * 8;
        const int ci = wn * 16 + nt * 8 + (lane & 3) * 2 + (k & 1);
        out[t * 1024 + co * 32 + ci] = acc[t][nt][k];
      }
  if (with_bias) {  // the 8 pixel groups' sums in a fixed order (patch buffers are free)
    float* red = reinterpret_cast<float*>(wt_smem);
    red[(tid >> 4) * 32 + (tid & 15) * 2] = bsum0;
    red[(tid >> 4) * 32 + (tid & 15) * 2 + 1] = bsum1;
    __syncthreads();
    if (tid < 32) {
      float t = 0.f;
#pragma unroll
      for (int g = 0; g < 8; ++g) t += red[g * 32 + tid];
      a.part[bias_off + (size_t(tile / ntn) * nchunks + ck) * 32 + tid] = t;
    }
  }
}

// dw[tap][co][ci] += sum over the chunks of the nine-tap kernel's partials,
// and db[co] += sum over the chunks of its bias partials (entries n .. n +
// Cout of the loop).  A block takes 32 consecutive entries; its 8 warps sum
// every 8th chunk each (lane = entry, 128-byte rows), then warp 0 adds the 8
// warp sums in a fixed order: deterministic, no atomics.
__global__ void __launch_bounds__(256) wgrad_reduce_kernel(const float* part, size_t bias_off,
                                                           int nchunks, int ntiles, int ntn,
                                                           int Cout, int Cin, float* dw,
                                                           float* db) {
  __shared__ float red[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long n = (long long)ntiles * 9 * 1024;
  const long long total = n + (db ? Cout : 0);
  for (long long base = (long long)blockIdx.x * 32; base < total;
       base += (long long)gridDim.x * 32) {
    const long long i = base + lane;  // n and Cout are multiples of 32
    const float* p;
    size_t stride;
    if (base < n) {
      const int tile = int(i / (9 * 1024)), r = int(i % (9 * 1024));
      p = part + size_t(tile) * nchunks * 9 * 1024 + r;
      stride = 9 * 1024;
    } else {
      const int co = int(i - n);
      p = part + bias_off + size_t(co >> 5) * nchunks * 32 + (co & 31);
      stride = 32;
    }
    float s = 0.f;
    for (int c = warp; c < nchunks; c += 8) s += p[size_t(c) * stride];
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
      float t = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) t += red[w][lane];
      if (base < n) {
        const int tile = int(i / (9 * 1024)), r = int(i % (9 * 1024));
        const int tp = r / 1024, co = (tile / ntn) * 32 + (r % 1024) / 32,
                  ci = (tile % ntn) * 32 + r % 32;
        dw[(size_t(tp) * Cout + co) * Cin + ci] += t;
      } else {
        db[i - n] += t;
      }
    }
    __syncthreads();
  }
}

// ---- element-wise kernels -------------------------------------------------------------
// All of them move 8 channels (16 bytes) per thread and iteration; channel
// counts, strides and offsets are multiples of 8.
using V8 = uint4;  // 8 bf16

__device__ __forceinline__ void unpack8(const V8& v, float (&f)[8]) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __low2float(h[i]);
    f[2 * i + 1] = __high2float(h[i]);
  }
}
__device__ __forceinline__ V8 pack8(const float (&f)[8]) {
  V8 v;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
  return v;
}
__device__ __forceinline__ const V8& ld8(const bf16* p) { return *reinterpret_cast<const V8*>(p); }
__device__ __forceinline__ void st8(bf16* p, const V8& v) { *reinterpret_cast<V8*>(p) = v; }

// bias gradient db[c] += sum over pixels of g[p][off + c]: each thread owns
// one group of 8 channels and a stride of pixels; a tree in shared memory
// per block, the blocks' sums added in a fixed order (sum_partials)
__global__ void bias_grad_kernel(const bf16* g, int Cg, int off, int C, long long npix,
                                 float* part) {
  __shared__ float red[256][8];
  const int groups = C / 8;
  const int lanes = blockDim.x / groups;  // pixel lanes per block
  const int cg = threadIdx.x % groups, pl = threadIdx.x / groups;
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (pl < lanes)
#pragma unroll 4
    for (long long p = (long long)blockIdx.x * lanes + pl; p < npix; p += (long long)gridDim.x * lanes) {
      float f[8];
      unpack8(ld8(g + p * Cg + off + cg * 8), f);
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i] += f[i];
    }
#pragma unroll
  for (int i = 0; i < 8; ++i) red[threadIdx.x][i] = acc[i];
  __syncthreads();
  // tree over the pixel lanes (a power of two, set by the launcher), then one
  // atomic per value
  for (int half = lanes / 2; half > 0; half /= 2) {
    if (pl < half)
#pragma unroll
      for (int i = 0; i < 8; ++i) red[threadIdx.x][i] += red[threadIdx.x + half * groups][i];
    __syncthreads();
  }
  if (threadIdx.x < groups)  // this block's sums; summed over the blocks in a fixed order
#pragma unroll
    for (int i = 0; i < 8; ++i) part[size_t(blockIdx.x) * C + threadIdx.x * 8 + i] = red[threadIdx.x][i];
}

// g = 0 where act <= 0
__global__ void mask_kernel(bf16* g, int Cg, int goff, const bf16* act, int Ca, int aoff, int C,
                            long long npix) {
  const int groups = C / 8;
  const long long n = npix * groups;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / groups;
    const int c = int(i % groups) * 8;
    float gv[8], av[8];
    unpack8(ld8(g + p * Cg + goff + c), gv);
    unpack8(ld8(act + p * Ca + aoff + c), av);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (!(av[k] > 0.f)) gv[k] = 0.f;
    st8(g + p * Cg + goff + c, pack8(gv));
  }
}

// y[b][h/2][w/2][c] = mean of the 2x2 block of x
__global__ void avgpool_kernel(const bf16* x, int Cx, int xoff, bf16* y, int Cy, int yoff, int C,
                               int B, int H, int W) {
  pdl_trigger();
  pdl_wait();
  const int Ho = H / 2, Wo = W / 2, groups = C / 8;
  const long long n = (long long)B * Ho * Wo * groups;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = int(i % groups) * 8;
    const long long q = i / groups;
    const int wo = int(q % Wo), ho = int((q / Wo) % Ho);
    const long long b = q / ((long long)Wo * Ho);
    const long long p00 = (b * H + 2 * ho) * W + 2 * wo;
    float s[8], t[8];
    unpack8(ld8(x + p00 * Cx + xoff + c), s);
    unpack8(ld8(x + (p00 + 1) * Cx + xoff + c), t);
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] += t[k];
    unpack8(ld8(x + (p00 + W) * Cx + xoff + c), t);
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] += t[k];
    unpack8(ld8(x + (p00 + W + 1) * Cx + xoff + c), t);
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] = 0.25f * (s[k] + t[k]);
    st8(y + q * Cy + yoff + c, pack8(s));
  }
}

// g_skip = (g_skip + 0.25 g_pool[pooled position]) * (skip > 0)
__global__ void pool_bwd_add_mask_kernel(bf16* gs, const bf16* gp, const bf16* act, int Cs,
                                         int soff, int C, int B, int H, int W) {
  const int groups = C / 8;
  const long long n = (long long)B * H * W * groups;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = int(i % groups) * 8;
    const long long p = i / groups;
    const int w = int(p % W), h = int((p / W) % H);
    const long long b = p / ((long long)W * H);
    const long long q = (b * (H / 2) + h / 2) * (W / 2) + w / 2;
    float v[8], u[8], a[8];
    unpack8(ld8(gs + p * Cs + soff + c), v);
    unpack8(ld8(gp + q * C + c), u);
    unpack8(ld8(act + p * Cs + soff + c), a);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = a[k] > 0.f ? v[k] + 0.25f * u[k] : 0.f;
    st8(gs + p * Cs + soff + c, pack8(v));
  }
}

// nearest 2x upsampling: each source pixel's 8 channels go to its 2x2 block
__global__ void upsample_kernel(const bf16* x, bf16* y, int C, int B, int H, int W) {
  pdl_trigger();
  pdl_wait();
  const int Hs = H / 2, Ws = W / 2, groups = C / 8;
  const long long n = (long long)B * Hs * Ws * groups;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = int(i % groups) * 8;
    const long long q = i / groups;
    const int ws = int(q % Ws), hs = int((q / Ws) % Hs);
    const long long b = q / ((long long)Ws * Hs);
    const V8 v = ld8(x + q * C + c);
    const long long p00 = (b * H + 2 * hs) * W + 2 * ws;
    st8(y + p00 * C + c, v);
    st8(y + (p00 + 1) * C + c, v);
    st8(y + (p00 + W) * C + c, v);
    st8(y + (p00 + W + 1) * C + c, v);
  }
}

// gradient of the upsampling (sum of the 2x2 block), masked by act > 0
__global__ void upsample_bwd_mask_kernel(const bf16* g, bf16* gx, const bf16* act, int C, int B,
                                         int H, int W) {
  const int Ho = H / 2, Wo = W / 2, groups = C / 8;
  const long long n = (long long)B * Ho * Wo * groups;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = int(i % groups) * 8;
    const long long q = i / groups;
    const int wo = int(q % Wo), ho = int((q / Wo) % Ho);
    const long long b = q / ((long long)Wo * Ho);
    const long long p00 = (b * H + 2 * ho) * W + 2 * wo;
    float s[8], t[8], a[8];
    unpack8(ld8(g + p00 * C + c), s);
    unpack8(ld8(g + (p00 + 1) * C + c), t);
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] += t[k];
    unpack8(ld8(g + (p00 + W) * C + c), t);
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] += t[k];
    unpack8(ld8(g + (p00 + W + 1) * C + c), t);
    unpack8(ld8(act + q * C + c), a);
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] = a[k] > 0.f ? s[k] + t[k] : 0.f;
    st8(gx + q * C + c, pack8(s));
  }
}

// 1x1 head: y[p][o] = b[o] + sum_c x[p][c] w[o][c] (FP32 out); one pixel per
// thread, weights staged in shared memory; the output count O is a template
// parameter so that the accumulators stay in registers
template <int O>
__global__ void head_fwd_kernel(const bf16* x, int C, const float* w, const float* b, float* y,
                                long long npix) {
  __shared__ float sw[O * 256 + O];
  pdl_trigger();
  pdl_wait();
  for (int i = threadIdx.x; i < O * C; i += blockDim.x) sw[i] = w[i];
  if (threadIdx.x < O) sw[O * 256 + threadIdx.x] = b[threadIdx.x];
  __syncthreads();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    float acc[O];
#pragma unroll
    for (int o = 0; o < O; ++o) acc[o] = sw[O * 256 + o];
    for (int c = 0; c < C; c += 8) {
      float f[8];
      unpack8(ld8(x + p * C + c), f);
#pragma unroll
      for (int o = 0; o < O; ++o)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[o] = fmaf(f[k], sw[o * C + c + k], acc[o]);
    }
#pragma unroll
    for (int o = 0; o < O; ++o) y[p * O + o] = acc[o];
  }
}

// head gradient for a tile of 256 pixels per block: gx = (gy w) * (x > 0)
// (bf16, one pixel per thread); dw[o][c] += sum_p gy[p][o] x[p][c] and
// db[o] += sum_p gy[p][o] from the tile staged in shared memory
// head backward: gx[p][c] = (x[p][c] > 0) sum_o gy[p][o] w[o][c],
// dw[o][c] += sum_p gy[p][o] x[p][c], db[o] += sum_p gy[p][o].  A warp walks
// pixels one at a time with lane c on channel c (C <= 32), so every access of
// x and gx is one coalesced row and gy is a broadcast; the 8 warps' sums meet
// in shared memory in a fixed order, the blocks' sums are added in a fixed
// order too (sum_partials).
template <int O>
__global__ void __launch_bounds__(256) head_bwd_kernel(const bf16* x, int C, const float* w,
                                                       const float* gy, long long npix, bf16* gx,
                                                       float* part) {
  __shared__ float red[8][O][33];  // per warp: dw[o][c] at [o][c], db[o] at [o][32]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool on = lane < C;
  float wl[O], acc[O], accb[O];
#pragma unroll
  for (int o = 0; o < O; ++o) {
    wl[o] = on ? w[o * C + lane] : 0.f;
    acc[o] = accb[o] = 0.f;
  }
  const long long stride = (long long)gridDim.x * 8;
#pragma unroll 4
  for (long long p = (long long)blockIdx.x * 8 + warp; p < npix; p += stride) {
    const float xv = on ? __bfloat162float(x[p * C + lane]) : 0.f;
    float s = 0.f;
#pragma unroll
    for (int o = 0; o < O; ++o) {
      const float g = gy[p * O + o];
      s += g * wl[o];
      acc[o] += g * xv;
      accb[o] += g;
    }
    if (on) gx[p * C + lane] = __float2bfloat16(xv > 0.f ? s : 0.f);
  }
#pragma unroll
  for (int o = 0; o < O; ++o) {
    red[warp][o][lane] = acc[o];
    if (lane == 0) red[warp][o][32] = accb[o];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < O * 33; i += blockDim.x) {
    const int o = i / 33, c = i % 33;
    if (c < C || c == 32) {
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) t += red[k][o][c];
      // this block's partial: dw entries o C + c, then the O db entries
      part[size_t(blockIdx.x) * (O * C + O) + (c == 32 ? O * C + o : o * C + c)] = t;
    }
  }
}

// MSE: loss += sum (y - t)^2 / n; gy = 2 (y - t) / n (one atomic per block)
__global__ void mse_kernel(const float* y, const float* t, long long n, float* gy, float* loss) {
  __shared__ float ws[32];
  float s = 0.f;
  const float inv = 1.f / float(n);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    s += d * d;
    gy[i] = 2.f * d * inv;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(loss, s * inv);
  }
}

// the table entry of block b: the last segment whose first block is <= b
template <typename Seg>
__device__ __forceinline__ const Seg& seg_of(const Seg* segs, int nseg, long long b) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].blk0 <= b) lo = mid;
    else hi = mid - 1;
  }
  return segs[lo];
}

// Adam with bias correction over every parameter tensor of the network in one
// launch: each block updates kSegBlock consecutive values of one tensor,
// refreshes their bf16 copy and clears their gradient
__global__ void __launch_bounds__(256) adam_multi_kernel(const AdamSeg* segs, int nseg, float lr,
                                                         float b1, float b2, float eps, float c1,
                                                         float c2) {
  const AdamSeg sg = seg_of(segs, nseg, blockIdx.x);
  const long long i0 = (blockIdx.x - sg.blk0) * (long long)kSegBlock;
#pragma unroll
  for (int k = 0; k < kSegBlock / 256; ++k) {
    const long long i = i0 + k * 256 + threadIdx.x;
    if (i >= sg.n) break;
    const float gi = sg.g[i];
    const float mi = b1 * sg.m[i] + (1.f - b1) * gi;
    const float vi = b2 * sg.v[i] + (1.f - b2) * gi * gi;
    sg.m[i] = mi;
    sg.v[i] = vi;
    const float wi = sg.w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    sg.w[i] = wi;
    if (sg.wb) sg.wb[i] = __float2bfloat16(wi);
    sg.g[i] = 0.f;
  }
}

// wt[8 - tap][ci][co] = w[tap][co][ci] (the weights of the data gradient) for
// every convolution of the network in one launch
__global__ void __launch_bounds__(256) flip_multi_kernel(const FlipSeg* segs, int nseg) {
  const FlipSeg sg = seg_of(segs, nseg, blockIdx.x);
  const long long n = 9LL * sg.cout * sg.cin;
  const long long i0 = (blockIdx.x - sg.blk0) * (long long)kSegBlock;
#pragma unroll
  for (int k = 0; k < kSegBlock / 256; ++k) {
    const long long i = i0 + k * 256 + threadIdx.x;
    if (i >= n) break;
    const int ci = int(i % sg.cin);
    const int co = int((i / sg.cin) % sg.cout);
    const int tap = int(i / ((long long)sg.cin * sg.cout));
    sg.wt[(size_t(8 - tap) * sg.cin + ci) * sg.cout + co] = sg.w[i];
  }
}

int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return int(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

}  // namespace

cudaError_t conv3x3(const ConvArgs& a, cudaStream_t s) {
  if (a.head_done) *a.head_done = 0;
  if (a.pool_done) *a.pool_done = 0;
  if (a.tensor_path && a.err && conv3x3_tc_supported(a)) return conv3x3_tc(a, a.err, s);
  if (a.W % 64 || a.Cin % 16 || a.Cx % 8 || a.Cy % 8 || a.ci_off % 8 || a.co_off % 8)
    return cudaErrorInvalidValue;
  const long long npix = (long long)a.N * a.H * a.W;
  if (a.Cout % 64 == 0) {
    conv3x3_kernel<64><<<dim3(unsigned(npix / 64), a.Cout / 64), kThreads, 0, s>>>(a);
  } else if (a.Cout % 32 == 0) {
    conv3x3_kernel<32><<<dim3(unsigned(npix / 64), a.Cout / 32), kThreads, 0, s>>>(a);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// the nine-tap kernel's launch shape: 32 x 32 tiles, pixel patches per CTA
// chosen for about four CTAs per SM
namespace {
struct TapsShape {
  int ntiles, ntn, patches, chunk, nchunks;
};
bool taps_shape(int Cout, int Cin, int N, int H, int W, TapsShape* t) {
  if (Cout % 32 || Cin % 32 || W % 64 || H % 2) return false;
  t->ntn = Cin / 32;
  t->ntiles = (Cout / 32) * t->ntn;
  t->patches = N * (H / 2) * (W / 64);
  const long long want = 4 * 152;
  t->chunk = int((t->patches * (long long)t->ntiles + want - 1) / want);
  if (t->chunk < 1) t->chunk = 1;
  t->nchunks = (t->patches + t->chunk - 1) / t->chunk;
  return true;
}
// pixels per chunk of the per-tap kernel: the requested chunk, enlarged so
// that its grid (9 x chunks) stays within 65535
int pertap_chunk(long long npix, int chunk) {
  const long long max_chunks = 65535 / 9;
  if ((npix + chunk - 1) / chunk > max_chunks) {
    const long long c = (npix + max_chunks - 1) / max_chunks;
    chunk = int((c + 15) / 16 * 16);
  }
  return chunk;
}
// floats of the nine-tap kernel's weight partials; its bias partials follow
size_t taps_weight_floats(const TapsShape& t) { return size_t(t.ntiles) * t.nchunks * 9 * 1024; }
size_t taps_bias_floats(const TapsShape& t) {
  return size_t(t.ntiles / t.ntn) * t.nchunks * 32;
}
}  // namespace

size_t wgrad_scratch(int Cout, int Cin, int N, int H, int W, int chunk) {
  TapsShape t;
  if (taps_shape(Cout, Cin, N, H, W, &t)) return taps_weight_floats(t) + taps_bias_floats(t);
  const long long npix = (long long)N * H * W;
  const int c = pertap_chunk(npix, chunk);
  return size_t((npix + c - 1) / c) * 9 * Cout * Cin + bias_grad_scratch(Cout, npix);
}

cudaError_t wgrad3x3(const WgradArgs& args, cudaStream_t s) {
  WgradArgs a = args;
  TapsShape ts;
  const int N = int(a.npix / ((long long)a.H * a.W));
  if (a.part && taps_shape(a.Cout, a.Cin, N, a.H, a.W, &ts) &&
      taps_weight_floats(ts) + taps_bias_floats(ts) <= a.part_cap && a.Cdy % 8 == 0 &&
      a.Cx % 8 == 0 && a.co_off % 8 == 0 && a.ci_off % 8 == 0) {
    const int smem = 2 * (kWP + kWHalo) * kWLD * 2;
    cudaError_t e =
        cudaFuncSetAttribute(wgrad_taps_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const size_t bias_off = taps_weight_floats(ts);
    wgrad_taps_kernel<<<ts.ntiles * ts.nchunks, kThreads, smem, s>>>(a, ts.chunk, ts.nchunks,
                                                                      ts.patches, bias_off);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long groups = ((long long)ts.ntiles * 9 * 1024 + (a.db ? a.Cout : 0)) / 32;
    wgrad_reduce_kernel<<<unsigned(groups < 152 * 16 ? groups : 152 * 16), 256, 0, s>>>(
        a.part, bias_off, ts.nchunks, ts.ntiles, ts.ntn, a.Cout, a.Cin, a.dw, a.db);
    return cudaGetLastError();
  }
  if (a.W % 16 || a.Cout % 32 || a.Cin % 16 || a.chunk < 16 || a.chunk % 16)
    return cudaErrorInvalidValue;
  a.chunk = pertap_chunk(a.npix, a.chunk);
  const int chunks = int((a.npix + a.chunk - 1) / a.chunk);
  const unsigned gz = unsigned(9 * chunks);
  // the per-tap kernel's partials per chunk, then the bias partials: both
  // summed in a fixed order; without room for them, FP32 atomics
  const size_t wfloats = size_t(chunks) * 9 * a.Cout * a.Cin;
  const size_t bfloats = a.db ? bias_grad_scratch(a.Cout, a.npix) : 0;
  const bool partials = a.part && wfloats + bfloats <= a.part_cap;
  if (!partials) a.part = nullptr;
  constexpr int KP = 64, S = 4;
  auto go = [&](auto kern, int bm, int bn) {
    const int smem = S * KP * ((bm + 8) + (bn + 8)) * 2;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(a.Cout / bm, a.Cin / bn, gz), kThreads, smem, s>>>(a);
    return cudaGetLastError();
  };
  cudaError_t e;
  if (a.Cout % 64 == 0 && a.Cin % 32 == 0) e = go(wgrad3x3_kernel<64, 32, KP, S>, 64, 32);
  else if (a.Cin % 32 == 0) e = go(wgrad3x3_kernel<32, 32, KP, S>, 32, 32);
  else e = go(wgrad3x3_kernel<32, 16, KP, S>, 32, 16);
  if (e != cudaSuccess) return e;
  if (partials) {
    const long long n = 9LL * a.Cout * a.Cin;
    if ((e = sum_partials(a.part, n, chunks, int(n), a.dw, s)) != cudaSuccess) return e;
  }
  if (!a.db) return cudaSuccess;
  if (!partials) return cudaErrorInvalidValue;  // the bias gradient needs its scratch
  return bias_grad(a.dy, a.Cdy, a.co_off, a.Cout, a.npix, a.db, args.part + wfloats,
                   a.part_cap - wfloats, s);
}

bool v8(int a) { return a % 8 == 0; }

int bias_grad_blocks(int C, long long npix, int* lanes_out) {
  // pixel lanes per block: a power of two (the kernel's tree reduction),
  // about 16 pixels per lane
  const int groups = C / 8;
  int lanes = 1;
  while (lanes * 2 * groups <= 256) lanes *= 2;
  long long blocks = (npix + lanes * 16 - 1) / (lanes * 16);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  if (lanes_out) *lanes_out = lanes;
  return int(blocks);
}
size_t bias_grad_scratch(int C, long long npix) {
  return size_t(bias_grad_blocks(C, npix, nullptr)) * C;
}
cudaError_t bias_grad(const bf16* g, int Cg, int off, int C, long long npix, float* db,
                      float* part, size_t part_cap, cudaStream_t s) {
  if (!v8(C) || !v8(Cg) || !v8(off) || C > 2048 || !part) return cudaErrorInvalidValue;
  int lanes = 1;
  const int blocks = bias_grad_blocks(C, npix, &lanes);
  if (size_t(blocks) * C > part_cap) return cudaErrorInvalidValue;
  bias_grad_kernel<<<blocks, (C / 8) * lanes, 0, s>>>(g, Cg, off, C, npix, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return sum_partials(part, C, blocks, C, db, s);
}
cudaError_t relu_mask(bf16* g, int Cg, int goff, const bf16* act, int Ca, int aoff, int C,
                      long long npix, cudaStream_t s) {
  if (!v8(C) || !v8(Cg) || !v8(goff) || !v8(Ca) || !v8(aoff)) return cudaErrorInvalidValue;
  mask_kernel<<<blocks_for(npix * C / 8), 256, 0, s>>>(g, Cg, goff, act, Ca, aoff, C, npix);
  return cudaGetLastError();
}
cudaError_t avgpool2(const bf16* x, int Cx, int xoff, bf16* y, int Cy, int yoff, int C, int B,
                     int H, int W, cudaStream_t s) {
  if (!v8(C) || !v8(Cx) || !v8(xoff) || !v8(Cy) || !v8(yoff)) return cudaErrorInvalidValue;
  return launch_pdl(avgpool_kernel, dim3(blocks_for((long long)B * H * W * C / 32)), dim3(256), 0,
                    s, x, Cx, xoff, y, Cy, yoff, C, B, H, W);
}
cudaError_t avgpool2_bwd_add_mask(bf16* gs, const bf16* gp, const bf16* act, int Cs, int soff,
                                  int C, int B, int H, int W, cudaStream_t s) {
  if (!v8(C) || !v8(Cs) || !v8(soff)) return cudaErrorInvalidValue;
  pool_bwd_add_mask_kernel<<<blocks_for((long long)B * H * W * C / 8), 256, 0, s>>>(
      gs, gp, act, Cs, soff, C, B, H, W);
  return cudaGetLastError();
}
cudaError_t upsample2(const bf16* x, bf16* y, int C, int B, int H, int W, cudaStream_t s) {
  if (!v8(C)) return cudaErrorInvalidValue;
  return launch_pdl(upsample_kernel, dim3(blocks_for((long long)B * H * W * C / 32)), dim3(256), 0,
                    s, x, y, C, B, H, W);
}
cudaError_t upsample2_bwd_mask(const bf16* g, bf16* gx, const bf16* act, int C, int B, int H,
                               int W, cudaStream_t s) {
  if (!v8(C)) return cudaErrorInvalidValue;
  upsample_bwd_mask_kernel<<<blocks_for((long long)B * H * W * C / 32), 256, 0, s>>>(g, gx, act,
                                                                                    C, B, H, W);
  return cudaGetLastError();
}
cudaError_t head_fwd(const bf16* x, int C, const float* w, const float* b, float* y, int O,
                     long long npix, cudaStream_t s) {
  if (!v8(C) || O < 1 || O > 8 || C > 256) return cudaErrorInvalidValue;
  const dim3 g(blocks_for(npix)), bl(256);
  switch (O) {
    case 1: return launch_pdl(head_fwd_kernel<1>, g, bl, 0, s, x, C, w, b, y, npix);
    case 2: return launch_pdl(head_fwd_kernel<2>, g, bl, 0, s, x, C, w, b, y, npix);
    case 3: return launch_pdl(head_fwd_kernel<3>, g, bl, 0, s, x, C, w, b, y, npix);
    case 4: return launch_pdl(head_fwd_kernel<4>, g, bl, 0, s, x, C, w, b, y, npix);
    case 5: return launch_pdl(head_fwd_kernel<5>, g, bl, 0, s, x, C, w, b, y, npix);
    case 6: return launch_pdl(head_fwd_kernel<6>, g, bl, 0, s, x, C, w, b, y, npix);
    case 7: return launch_pdl(head_fwd_kernel<7>, g, bl, 0, s, x, C, w, b, y, npix);
    default: return launch_pdl(head_fwd_kernel<8>, g, bl, 0, s, x, C, w, b, y, npix);
  }
}
int head_bwd_blocks(long long npix) {
  long long blocks = (npix + 8 * 16 - 1) / (8 * 16);  // about 16 pixels per warp
  if (blocks > 152 * 8) blocks = 152 * 8;
  return int(blocks < 1 ? 1 : blocks);
}
size_t head_bwd_scratch(int C, int O, long long npix) {
  return size_t(head_bwd_blocks(npix)) * (size_t(O) * C + O);
}
cudaError_t head_bwd(const bf16* x, int C, const float* w, const float* gy, int O, long long npix,
                     bf16* gx, float* dw, float* db, float* part, size_t part_cap,
                     cudaStream_t s) {
  if (O < 1 || O > 8 || C > 32 || !v8(C) || !part) return cudaErrorInvalidValue;
  const int blocks = head_bwd_blocks(npix);
  if (size_t(blocks) * (O * C + O) > part_cap) return cudaErrorInvalidValue;
  const dim3 g{unsigned(blocks)}, bl{256};
  switch (O) {
    case 1: head_bwd_kernel<1><<<g, bl, 0, s>>>(x, C, w, gy, npix, gx, part); break;
    case 2: head_bwd_kernel<2><<<g, bl, 0, s>>>(x, C, w, gy, npix, gx, part); break;
    case 3: head_bwd_kernel<3><<<g, bl, 0, s>>>(x, C, w, gy, npix, gx, part); break;
    case 4: head_bwd_kernel<4><<<g, bl, 0, s>>>(x, C, w, gy, npix, gx, part); break;
    case 5: head_bwd_kernel<5><<<g, bl, 0, s>>>(x, C, w, gy, npix, gx, part); break;
    case 6: head_bwd_kernel<6><<<g, bl, 0, s>>>(x, C, w, gy, npix, gx, part); break;
    case 7: head_bwd_kernel<7><<<g, bl, 0, s>>>(x, C, w, gy, npix, gx, part); break;
    default: head_bwd_kernel<8><<<g, bl, 0, s>>>(x, C, w, gy, npix, gx, part); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long stride = (long long)O * C + O;
  if ((e = sum_partials(part, stride, blocks, O * C, dw, s)) != cudaSuccess) return e;
  return sum_partials(part + size_t(O) * C, stride, blocks, O, db, s);
}
cudaError_t mse(const float* y, const float* t, long long n, float* gy, float* loss,
                cudaStream_t s) {
  mse_kernel<<<blocks_for(n), 256, 0, s>>>(y, t, n, gy, loss);
  return cudaGetLastError();
}
cudaError_t adam_multi(const AdamSeg* segs, int nseg, long long blocks, float lr, float b1,
                       float b2, float eps, int t, cudaStream_t s) {
  if (nseg < 1 || blocks < 1 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  const float c1 = 1.f - powf(b1, float(t)), c2 = 1.f - powf(b2, float(t));
  adam_multi_kernel<<<unsigned(blocks), 256, 0, s>>>(segs, nseg, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}
cudaError_t flip_multi(const FlipSeg* segs, int nseg, long long blocks, cudaStream_t s) {
  if (nseg < 1 || blocks < 1 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  flip_multi_kernel<<<unsigned(blocks), 256, 0, s>>>(segs, nseg);
  return cudaGetLastError();
}

}  // namespace nn
}  // namespace lbk
