// Tensor-core 3x3 convolution of the U-Net surrogate on the 5th-generation
// tensor cores: implicit GEMM D[pixel][co] = sum over the nine taps and the
// input channels of x[pixel + shift(tap)][ci] w[tap][co][ci], then bias,
// ReLU, an optional mask, bf16 out.  The same kernel computes the data
// gradient on flipped / transposed weights.
//
// Persistent CTAs (one per SM) walk a strided list of output tiles of G
// sub-tiles of 128 pixels (one or two image rows each) x BN output channels,
// channel tiles innermost so that CTAs running side by side share their input
// rows in L2.  The G sub-tiles share the weight box and accumulate into G
// independent accumulators whose products are interleaved: with a narrow N
// one accumulator's chain of dependent products would leave the tensor pipe
// mostly idle.  Roles:
//   warp 0     TMA producer: per K step (one tap, BK input channels) a 4D box
//              of the NHWC input at the tap's shifted origin (zero fill
//              outside the image gives the convolution's zero padding) and a
//              3D box of the weights, into a stage of an S-deep ring that
//              runs on across tiles
//   warp 1     allocates tensor memory (two accumulators of BN FP32 columns);
//              one lane issues tcgen05.mma (kind::f16, bf16 x bf16 -> f32,
//              M = 128, N = BN, K = 16), frees each stage and hands each
//              finished accumulator to the epilogue through tcgen05.commit
//   warps 2-5  epilogue: tcgen05.ld of their 32-lane quarter of an
//              accumulator, bias / ReLU / mask, bf16 stores; then release the
//              accumulator, so that the next tile's products overlap them
// conv3x3_tc_halo_kernel (below) is the variant taken wherever the image
// width is a multiple of 128 and N <= 128: one input box per (channel chunk,
// ky) serves the three kx taps.
// Every wait on a barrier is bounded; on a timeout the kernel sets bit 2 of
// *err, lets the copies and products already issued finish, frees its tensor
// memory and returns (the host turns the bit into an error status).
#include <cuda.h>

#include <cstdint>
#include <cstdlib>

#include "tma.cuh"
#include "tma_host.h"
#include "unet.cuh"

namespace lbk {
namespace nn {
namespace {

constexpr int kTcThreads = 192;
constexpr int kTcSpin = 1 << 22;  // polls per barrier wait

// Shared-memory matrix descriptor of a K-major operand tile whose rows are
// exactly one swizzle span long (BK bf16), 8-row core groups SBO bytes apart.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t sbo, uint32_t mode) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFFu) >> 4);           // start address
  d |= uint64_t(1) << 16;                           // leading offset (unused: one span per row)
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;        // stride between 8-row groups
  d |= uint64_t(1) << 46;                           // descriptor version
  d |= uint64_t(mode) << 61;                        // swizzle mode
  return d;
}

// The same with the matrix starting `row` rows (of one swizzle span, rb
// bytes) into a 1024-byte aligned swizzled buffer.  The swizzle phase follows
// the absolute shared-memory address (as the TMA wrote it), so the start may
// sit at any row with the base-offset field left at 0 (measured: setting it
// to the row's phase, or starting at the aligned group with that phase,
// gives wrong products).
__device__ __forceinline__ uint64_t umma_desc_row(uint32_t saddr_aligned, int row, uint32_t rb,
                                                  uint32_t sbo, uint32_t mode) {
  return umma_desc(saddr_aligned + uint32_t(row) * rb, sbo, mode);
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(holder)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrives on `bar` once every tcgen05 operation this thread issued so far is done
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}
// 32 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcArgs {
  int H, W, BW;          // image size; tile width in pixels (128 or 64)
  int ci_off, nchunks;   // first input channel; K steps per tap
  int Cin;               // input channels
  int mtiles, ntiles_n;  // pixel tiles, channel tiles
  int Cy, co_off, relu;  // output channel stride / offset
  int Cout;              // output channels (bias entries)
  const float* bias;
  const bf16* mask;
  bf16* y;
  unsigned* err;
};

template <int BK, int BN, int G>
struct TcShape {
  static constexpr int A_BYTES = 128 * BK * 2;  // one 128-pixel sub-tile
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE = G * A_BYTES + B_BYTES;
  // one persistent CTA per SM: a ring as deep as ~200 KB of shared memory
  // allows (small stages need many copies in flight to cover their latency)
  static constexpr int S_FIT = 204800 / STAGE;
  static constexpr int S = S_FIT > 32 ? 32 : (S_FIT < 2 ? 2 : S_FIT);
  static constexpr int SMEM = S * STAGE + 1024;  // + alignment slack
  static_assert(SMEM <= 226 * 1024, "stage ring exceeds shared memory");
  static constexpr uint32_t SBO = 8 * BK * 2;
  static constexpr uint32_t MODE = BK == 64 ? 2 : (BK == 32 ? 4 : 6);  // 128 / 64 / 32 B swizzle
  // kind::f16 instruction descriptor: D f32, A and B bf16, both K-major, N, M = 128
  static constexpr uint32_t IDESC =
      (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(128 >> 4) << 24);
  static constexpr uint32_t ACC = G * BN;    // columns of one accumulator set
  static constexpr uint32_t TCOLS = 2 * ACC;  // double-buffered
  static_assert(TCOLS <= 512, "accumulators exceed tensor memory");
};

template <int BK, int BN, int G>
__global__ void __launch_bounds__(kTcThreads, 1)
    conv3x3_tc_kernel(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mw,
                      const TcArgs a) {
  using Sh = TcShape<BK, BN, G>;
  constexpr int S = Sh::S;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[S], empty[S], acc_full[2], acc_empty[2], fin;
  __shared__ uint32_t tmem_base;
  __shared__ float sbias[256];
  uint8_t* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ksteps = 9 * a.nchunks;
  const int ntiles = (a.mtiles / G) * a.ntiles_n;  // a tile: G x 128 pixels x BN channels
  pdl_trigger();

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp
    }
    mbar_init(&fin, 1);
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, Sh::TCOLS);
  pdl_wait();  // the previous kernel's outputs (and any weight update) are visible
  for (int i = threadIdx.x; i < a.Cout; i += blockDim.x) sbias[i] = a.bias ? a.bias[i] : 0.f;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // producer: coordinates once per tile, counters instead of divisions
    int st = 0, it = 0;
    uint32_t ph = 0;  // phase of the current pass over the ring
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const long long pix0 = (long long)(t / a.ntiles_n) * (128 * G);
      const int n0 = (t % a.ntiles_n) * BN;
      int wg[G], hg[G], ig[G];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const long long pg = pix0 + g * 128;
        wg[g] = int(pg % a.W) - 1;
        hg[g] = int((pg / a.W) % a.H) - 1;
        ig[g] = int(pg / ((long long)a.W * a.H));
      }
      int c0 = 0, kx = 0, ky = 0;
      for (int ks = 0; ks < ksteps; ++ks, ++it) {
        if (it >= S && !mbar_wait_bounded(&empty[st], ph ^ 1u, kTcSpin)) {
          atomicOr(a.err, 2u);
          ok = false;
          break;
        }
        uint8_t* sa = smem + st * Sh::STAGE;
        mbar_arrive_expect_tx(&full[st], Sh::STAGE);
#pragma unroll
        for (int g = 0; g < G; ++g)
          tma_load_4d(sa + g * Sh::A_BYTES, &mx, &full[st], a.ci_off + c0, wg[g] + kx, hg[g] + ky,
                      ig[g]);
        tma_load_3d(sa + G * Sh::A_BYTES, &mw, &full[st], c0, n0, ky * 3 + kx);
        c0 += BK;
        if (c0 == a.Cin) {
          c0 = 0;
          if (++kx == 3) {
            kx = 0;
            ++ky;
          }
        }
        if (++st == S) {
          st = 0;
          ph ^= 1u;
        }
      }
    }
    // every issued copy has landed before the CTA may finish
    for (int j = it > S ? it - S : 0; j < it; ++j)
      if (!mbar_wait_bounded(&full[j % S], uint32_t(j / S) & 1u, kTcSpin)) atomicOr(a.err, 2u);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: descriptors as offsets from a precomputed base (the start
    // address field holds address / 16; shared addresses stay below 256 KB)
    const uint64_t d0 = umma_desc(smem_addr(smem), Sh::SBO, Sh::MODE);
    int st = 0, tc = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tc) {
      const int buf = tc & 1;
      if (tc >= 2 && !mbar_wait_bounded(&acc_empty[buf], uint32_t((tc >> 1) - 1) & 1u, kTcSpin)) {
        atomicOr(a.err, 2u);
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + uint32_t(buf * Sh::ACC);
      for (int ks = 0; ks < ksteps; ++ks) {
        if (!mbar_wait_bounded(&full[st], ph, kTcSpin)) {
          atomicOr(a.err, 2u);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t ds = d0 + uint64_t((st * Sh::STAGE) >> 4);
        // the G sub-tiles accumulate independently: interleaving them keeps
        // several products in flight on the tensor pipe
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t db = ds + uint64_t((G * Sh::A_BYTES + kk * 32) >> 4);
#pragma unroll
          for (int g = 0; g < G; ++g)
            tc_mma(d + uint32_t(g * BN), ds + uint64_t((g * Sh::A_BYTES + kk * 32) >> 4), db,
                   Sh::IDESC, (ks | kk) != 0);
        }
        tc_commit(&empty[st]);
        if (++st == S) {
          st = 0;
          ph ^= 1u;
        }
      }
      if (ok) tc_commit(&acc_full[buf]);
    }
    // all products issued by this CTA are complete before its tensor memory is freed
    tc_commit(&fin);
    if (!mbar_wait_bounded(&fin, 0u, kTcSpin)) atomicOr(a.err, 2u);
  } else if (warp >= 2) {
    const int q = warp & 3;  // tensor-memory lanes 32q .. 32q + 31
    const int m = q * 32 + lane;
    int tc = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tc) {
      const int buf = tc & 1;
      bool ok = mbar_wait_bounded(&acc_full[buf], uint32_t(tc >> 1) & 1u, kTcSpin);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) atomicOr(a.err, 2u);
        break;
      }
      tc_fence_after();
      const long long pix0 = (long long)(t / a.ntiles_n) * (128 * G);
      const int n0 = (t % a.ntiles_n) * BN;
#pragma unroll 1
      for (int g = 0; g < G; ++g) {
        const long long pg = pix0 + g * 128;
        const int w0 = int(pg % a.W), h0 = int((pg / a.W) % a.H);
        const int img = int(pg / ((long long)a.W * a.H));
        const long long p = ((long long)img * a.H + h0 + m / a.BW) * a.W + w0 + (m % a.BW);
        bf16* yrow = a.y + p * a.Cy + a.co_off + n0;
        const bf16* mrow = a.mask ? a.mask + p * a.Cy + a.co_off + n0 : nullptr;
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
          uint32_t r[32];
          tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(buf * Sh::ACC + g * BN + c), r);
          uint4 mk[4];
          if (mrow)
#pragma unroll
            for (int v = 0; v < 4; ++v) mk[v] = reinterpret_cast<const uint4*>(mrow + c)[v];
          uint32_t out[16];
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            float v0 = __uint_as_float(r[j]) + sbias[n0 + c + j];
            float v1 = __uint_as_float(r[j + 1]) + sbias[n0 + c + j + 1];
            if (a.relu) {
              v0 = fmaxf(v0, 0.f);
              v1 = fmaxf(v1, 0.f);
            }
            if (mrow) {
              const __nv_bfloat162 mm = reinterpret_cast<const __nv_bfloat162*>(mk)[j / 2];
              if (!(__low2float(mm) > 0.f)) v0 = 0.f;
              if (!(__high2float(mm) > 0.f)) v1 = 0.f;
            }
            const __nv_bfloat162 o = __floats2bfloat162_rn(v0, v1);
            out[j / 2] = *reinterpret_cast<const uint32_t*>(&o);
          }
#pragma unroll
          for (int v = 0; v < 4; ++v)
            reinterpret_cast<uint4*>(yrow + c)[v] =
                make_uint4(out[4 * v], out[4 * v + 1], out[4 * v + 2], out[4 * v + 3]);
        }
      }
      // this warp's reads of the accumulator are done: hand it back
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, Sh::TCOLS);
  }
}

// ---- halo variant: one input box per (channel chunk, ky) serves the three kx taps
// Tiles of G image rows x 128 pixels (images of width a multiple of 128), BK
// input channels per K step.  A K step loads the G rows h0 + ky - 1 + g of the
// tile's columns w0 - 1 .. w0 + 128 (130 pixels, zero fill outside the
// image) and the weights of the taps (ky, kx = 0, 1, 2); sub-tile g's operand
// for tap kx is the 128 rows starting kx rows into row g of the box, so each
// input row is fetched once per ky instead of once per tap.
template <int BK, int BN, int G>
struct HaloShape {
  static constexpr int ROWS = 130;                 // pixels per box row
  static constexpr int RB = BK * 2;                // bytes per pixel row (one swizzle span)
  static constexpr int A_ROW = ROWS * RB;          // bytes of one image row of the box
  static constexpr int A_BYTES = G * A_ROW;
  static constexpr int B_TAP = BN * RB;            // bytes of one tap's weights
  static constexpr int B_OFF = (A_BYTES + 1023) / 1024 * 1024;
  static constexpr int STAGE = (B_OFF + 3 * B_TAP + 1023) / 1024 * 1024;
  static constexpr int TX_BYTES = A_BYTES + 3 * B_TAP;
  static constexpr int S_FIT = 204800 / STAGE;
  static constexpr int S = S_FIT > 16 ? 16 : (S_FIT < 2 ? 2 : S_FIT);
  static constexpr int SMEM = S * STAGE + 1024;
  static_assert(SMEM <= 226 * 1024, "stage ring exceeds shared memory");
  static constexpr uint32_t SBO = 8 * RB;
  static constexpr uint32_t MODE = BK == 64 ? 2 : (BK == 32 ? 4 : 6);  // 128 / 64 / 32 B swizzle
  static constexpr uint32_t IDESC =
      (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(128 >> 4) << 24);
  static constexpr uint32_t ACC = G * BN;
  static constexpr uint32_t TCOLS = 2 * ACC;
  static_assert(TCOLS <= 512, "accumulators exceed tensor memory");
};

struct HaloArgs {
  int H, W, rows_t, cols_t;  // image size; tiles per image column / row
  int ci_off, nchunks;       // first input channel; 64-channel chunks
  int ntiles, ntiles_n;      // tiles; channel tiles
  int Cy, co_off, relu, Cout;
  const float* bias;
  const bf16* mask;
  bf16* y;
  unsigned* err;
  // fused 1x1 head (null head_y: none): with one channel tile holding all
  // Cout channels of a pixel, head_y[p][o] = head_b[o] + sum_c head_w[o][c]
  // y[p][c] over the bf16 values stored, in channel order (the arithmetic of
  // the separate head kernel, so the result is the same)
  const float* head_w;
  const float* head_b;
  float* head_y;
  int head_out;
  // fused 2 x 2 average pooling of the output (null pool_y: none; G even and
  // no mask): pool_y [N][H/2][W/2][pool_Cy], channels pool_off + n0 + c
  bf16* pool_y;
  int pool_Cy, pool_off;
};

template <int BK, int BN, int G>
__global__ void __launch_bounds__(kTcThreads, 1)
    conv3x3_tc_halo_kernel(const __grid_constant__ CUtensorMap mx,
                           const __grid_constant__ CUtensorMap mw, const HaloArgs a) {
  using Sh = HaloShape<BK, BN, G>;
  constexpr int S = Sh::S;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[S], empty[S], acc_full[2], acc_empty[2], fin;
  __shared__ uint32_t tmem_base;
  __shared__ float sbias[256];
  __shared__ float shead[8 * BN + 8];
  uint8_t* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ksteps = 3 * a.nchunks;
  const bool head = a.head_y != nullptr;
  const bool pool = a.pool_y != nullptr;
  pdl_trigger();
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(&fin, 1);
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, Sh::TCOLS);
  pdl_wait();  // the previous kernel's outputs (and any weight update) are visible
  for (int i = threadIdx.x; i < a.Cout; i += blockDim.x) sbias[i] = a.bias ? a.bias[i] : 0.f;
  if (head)
    for (int i = threadIdx.x; i < a.head_out * (BN + 1); i += blockDim.x)
      shead[i] = i < a.head_out * BN ? a.head_w[i] : a.head_b[i - a.head_out * BN];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  // tile t -> (image, first row, first column, first output channel)
  auto tile_at = [&](int t, int& img, int& h0, int& w0, int& n0) {
    const int gm = t / a.ntiles_n;
    n0 = (t % a.ntiles_n) * BN;
    const int per_img = a.rows_t * a.cols_t;
    img = gm / per_img;
    const int r = gm % per_img;
    h0 = (r / a.cols_t) * G;
    w0 = (r % a.cols_t) * 128;
  };

  if (warp == 0 && lane == 0) {
    int st = 0, it = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
      int img, h0, w0, n0;
      tile_at(t, img, h0, w0, n0);
      int c0 = 0, ky = 0;
      for (int ks = 0; ks < ksteps; ++ks, ++it) {
        if (it >= S && !mbar_wait_bounded(&empty[st], ph ^ 1u, kTcSpin)) {
          atomicOr(a.err, 2u);
          ok = false;
          break;
        }
        uint8_t* sa = smem + st * Sh::STAGE;
        mbar_arrive_expect_tx(&full[st], Sh::TX_BYTES);
        tma_load_4d(sa, &mx, &full[st], a.ci_off + c0, w0 - 1, h0 + ky - 1, img);
        tma_load_4d(sa + Sh::B_OFF, &mw, &full[st], c0, n0, 0, ky);
        if (++ky == 3) {
          ky = 0;
          c0 += BK;
        }
        if (++st == S) {
          st = 0;
          ph ^= 1u;
        }
      }
    }
    for (int j = it > S ? it - S : 0; j < it; ++j)
      if (!mbar_wait_bounded(&full[j % S], uint32_t(j / S) & 1u, kTcSpin)) atomicOr(a.err, 2u);
  } else if (warp == 1 && lane == 0) {
    const uint32_t s0 = smem_addr(smem);
    int st = 0, tc = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++tc) {
      const int buf = tc & 1;
      if (tc >= 2 && !mbar_wait_bounded(&acc_empty[buf], uint32_t((tc >> 1) - 1) & 1u, kTcSpin)) {
        atomicOr(a.err, 2u);
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + uint32_t(buf * Sh::ACC);
      for (int ks = 0; ks < ksteps; ++ks) {
        if (!mbar_wait_bounded(&full[st], ph, kTcSpin)) {
          atomicOr(a.err, 2u);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = s0 + uint32_t(st * Sh::STAGE), sb = sa + Sh::B_OFF;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk)
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) {
            const uint64_t db =
                umma_desc(sb + uint32_t(kx * Sh::B_TAP + kk * 32), Sh::SBO, Sh::MODE);
#pragma unroll
            for (int g = 0; g < G; ++g)
              tc_mma(d + uint32_t(g * BN),
                     umma_desc_row(sa, g * Sh::ROWS + kx, Sh::RB, Sh::SBO, Sh::MODE) +
                         uint64_t((kk * 32) >> 4),
                     db, Sh::IDESC, (ks | kk | kx) != 0);
          }
        tc_commit(&empty[st]);
        if (++st == S) {
          st = 0;
          ph ^= 1u;
        }
      }
      if (ok) tc_commit(&acc_full[buf]);
    }
    tc_commit(&fin);
    if (!mbar_wait_bounded(&fin, 0u, kTcSpin)) atomicOr(a.err, 2u);
  } else if (warp >= 2) {
    const int q = warp & 3;
    const int m = q * 32 + lane;
    int tc = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++tc) {
      const int buf = tc & 1;
      bool ok = mbar_wait_bounded(&acc_full[buf], uint32_t(tc >> 1) & 1u, kTcSpin);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) atomicOr(a.err, 2u);
        break;
      }
      tc_fence_after();
      int img, h0, w0, n0;
      tile_at(t, img, h0, w0, n0);
      if constexpr (G % 2 == 0) {
        if (pool) {
          // rows in pairs: both rows' outputs are stored, and each even lane
          // also writes the 2 x 2 average of its pixel, its right neighbour's
          // (lane + 1) and the two below, in the order of the separate
          // pooling kernel ((x00 + x01) + x10 + x11) / 4 over the bf16 values
#pragma unroll 1
          for (int g0 = 0; g0 < G; g0 += 2) {
            const long long p0 = ((long long)img * a.H + h0 + g0) * a.W + w0 + m;
            bf16* y0 = a.y + p0 * a.Cy + a.co_off + n0;
            bf16* y1 = y0 + (long long)a.W * a.Cy;
            const long long pp = ((long long)img * (a.H / 2) + (h0 + g0) / 2) * (a.W / 2) +
                                 (w0 + m) / 2;
            bf16* yp = a.pool_y + pp * a.pool_Cy + a.pool_off + n0;
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
              uint32_t o0[16], o1[16];
#pragma unroll
              for (int rr = 0; rr < 2; ++rr) {
                uint32_t r[32];
                tmem_ld32(tmem + (uint32_t(q * 32) << 16) +
                              uint32_t(buf * Sh::ACC + (g0 + rr) * BN + c),
                          r);
                uint32_t* o = rr ? o1 : o0;
#pragma unroll
                for (int j = 0; j < 32; j += 2) {
                  float v0 = __uint_as_float(r[j]) + sbias[n0 + c + j];
                  float v1 = __uint_as_float(r[j + 1]) + sbias[n0 + c + j + 1];
                  if (a.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                  }
                  const __nv_bfloat162 ob = __floats2bfloat162_rn(v0, v1);
                  o[j / 2] = *reinterpret_cast<const uint32_t*>(&ob);
                }
              }
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                reinterpret_cast<uint4*>(y0 + c)[v] =
                    make_uint4(o0[4 * v], o0[4 * v + 1], o0[4 * v + 2], o0[4 * v + 3]);
                reinterpret_cast<uint4*>(y1 + c)[v] =
                    make_uint4(o1[4 * v], o1[4 * v + 1], o1[4 * v + 2], o1[4 * v + 3]);
              }
              uint32_t pk[16];
#pragma unroll
              for (int k = 0; k < 16; ++k) {
                const uint32_t n0v = __shfl_down_sync(0xffffffffu, o0[k], 1);
                const uint32_t n1v = __shfl_down_sync(0xffffffffu, o1[k], 1);
                const __nv_bfloat162 x00 = *reinterpret_cast<const __nv_bfloat162*>(&o0[k]);
                const __nv_bfloat162 x01 = *reinterpret_cast<const __nv_bfloat162*>(&n0v);
                const __nv_bfloat162 x10 = *reinterpret_cast<const __nv_bfloat162*>(&o1[k]);
                const __nv_bfloat162 x11 = *reinterpret_cast<const __nv_bfloat162*>(&n1v);
                float lo = __low2float(x00) + __low2float(x01);
                float hi = __high2float(x00) + __high2float(x01);
                lo += __low2float(x10);
                hi += __high2float(x10);
                lo = 0.25f * (lo + __low2float(x11));
                hi = 0.25f * (hi + __high2float(x11));
                const __nv_bfloat162 pb = __floats2bfloat162_rn(lo, hi);
                pk[k] = *reinterpret_cast<const uint32_t*>(&pb);
              }
              if ((lane & 1) == 0)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                  reinterpret_cast<uint4*>(yp + c)[v] =
                      make_uint4(pk[4 * v], pk[4 * v + 1], pk[4 * v + 2], pk[4 * v + 3]);
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[buf]);
          continue;
        }
      }
#pragma unroll 1
      for (int g = 0; g < G; ++g) {
        const long long p = ((long long)img * a.H + h0 + g) * a.W + w0 + m;
        bf16* yrow = a.y + p * a.Cy + a.co_off + n0;
        const bf16* mrow = a.mask ? a.mask + p * a.Cy + a.co_off + n0 : nullptr;
        float hacc[8];
        if (head)
#pragma unroll
          for (int o = 0; o < 8; ++o) hacc[o] = o < a.head_out ? shead[a.head_out * BN + o] : 0.f;
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
          uint32_t r[32];
          tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(buf * Sh::ACC + g * BN + c), r);
          uint4 mk[4];
          if (mrow)
#pragma unroll
            for (int v = 0; v < 4; ++v) mk[v] = reinterpret_cast<const uint4*>(mrow + c)[v];
          uint32_t out[16];
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            float v0 = __uint_as_float(r[j]) + sbias[n0 + c + j];
            float v1 = __uint_as_float(r[j + 1]) + sbias[n0 + c + j + 1];
            if (a.relu) {
              v0 = fmaxf(v0, 0.f);
              v1 = fmaxf(v1, 0.f);
            }
            if (mrow) {
              const __nv_bfloat162 mm = reinterpret_cast<const __nv_bfloat162*>(mk)[j / 2];
              if (!(__low2float(mm) > 0.f)) v0 = 0.f;
              if (!(__high2float(mm) > 0.f)) v1 = 0.f;
            }
            const __nv_bfloat162 o = __floats2bfloat162_rn(v0, v1);
            out[j / 2] = *reinterpret_cast<const uint32_t*>(&o);
          }
#pragma unroll
          for (int v = 0; v < 4; ++v)
            reinterpret_cast<uint4*>(yrow + c)[v] =
                make_uint4(out[4 * v], out[4 * v + 1], out[4 * v + 2], out[4 * v + 3]);
          if (head) {
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
              const __nv_bfloat162 hv = *reinterpret_cast<const __nv_bfloat162*>(&out[j / 2]);
              const float f0 = __low2float(hv), f1 = __high2float(hv);
#pragma unroll
              for (int o = 0; o < 8; ++o)
                if (o < a.head_out) {
                  hacc[o] = fmaf(f0, shead[o * BN + c + j], hacc[o]);
                  hacc[o] = fmaf(f1, shead[o * BN + c + j + 1], hacc[o]);
                }
            }
          }
        }
        if (head)
#pragma unroll
          for (int o = 0; o < 8; ++o)
            if (o < a.head_out) a.head_y[p * a.head_out + o] = hacc[o];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, Sh::TCOLS);
  }
}

template <int BK, int BN, int G>
cudaError_t launch_halo(const CUtensorMap& mx, const CUtensorMap& mw, const HaloArgs& t,
                        cudaStream_t s) {
  using Sh = HaloShape<BK, BN, G>;
  static int sms = 0;
  if (!sms) {
    cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_halo_kernel<BK, BN, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return e;
  }
  const unsigned grid = unsigned(t.ntiles < sms ? t.ntiles : sms);
  return launch_pdl(conv3x3_tc_halo_kernel<BK, BN, G>, dim3(grid), dim3(kTcThreads), Sh::SMEM, s,
                    mx, mw, t);
}

CUtensorMapSwizzle swizzle_for(int bk) {
  return bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                  : (bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
}

template <int BK, int BN, int G>
cudaError_t launch_tc(const CUtensorMap& mx, const CUtensorMap& mw, const TcArgs& t,
                      cudaStream_t s) {
  using Sh = TcShape<BK, BN, G>;
  static int sms = 0;
  if (!sms) {
    cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_kernel<BK, BN, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return e;
  }
  // one CTA per SM: the ring fills the shared memory, the accumulators the TMEM
  const long long tiles = (long long)(t.mtiles / G) * t.ntiles_n;
  const unsigned grid = unsigned(tiles < sms ? tiles : sms);
  return launch_pdl(conv3x3_tc_kernel<BK, BN, G>, dim3(grid), dim3(kTcThreads), Sh::SMEM, s, mx,
                    mw, t);
}

// G sub-tiles per tile (independent accumulators); the widest shapes stay
// within 227 KB of shared memory and 512 TMEM columns
template <int BK, int BN>
cudaError_t launch_g(int g, const CUtensorMap& mx, const CUtensorMap& mw, const TcArgs& t,
                     cudaStream_t s) {
  if (BN == 32 && BK < 64 && g == 8) return launch_tc<BK, BN, (BN == 32 && BK < 64) ? 8 : 1>(mx, mw, t, s);
  if (BN <= 64 && g == 4) return launch_tc<BK, BN, (BN <= 64) ? 4 : 1>(mx, mw, t, s);
  if (BN <= 128 && g == 2) return launch_tc<BK, BN, (BN <= 128) ? 2 : 1>(mx, mw, t, s);
  if (g == 1) return launch_tc<BK, BN, 1>(mx, mw, t, s);
  return cudaErrorInvalidValue;
}

template <int BK>
cudaError_t launch_bn(int bn, int g, const CUtensorMap& mx, const CUtensorMap& mw,
                      const TcArgs& t, cudaStream_t s) {
  switch (bn) {
    case 32: return launch_g<BK, 32>(g, mx, mw, t, s);
    case 64: return launch_g<BK, 64>(g, mx, mw, t, s);
    case 128: return launch_g<BK, 128>(g, mx, mw, t, s);
    case 256: return launch_g<BK, 256>(g, mx, mw, t, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool conv3x3_tc_supported(const ConvArgs& a) {
  const long long npix = (long long)a.N * a.H * a.W;
  const bool rows = a.W % 128 == 0 || (a.W == 64 && a.H % 2 == 0);
  return rows && npix % 128 == 0 && a.Cin % 16 == 0 && a.Cout % 32 == 0 && a.Cout <= 256 &&
         a.Cx % 8 == 0 &&
         a.Cy % 8 == 0 && a.ci_off % 8 == 0 && a.co_off % 8 == 0 && a.ci_off + a.Cin <= a.Cx &&
         a.co_off + a.Cout <= a.Cy;
}

// the halo variant: images of width a multiple of 128, output tiles of at
// most 128 channels (its three-tap weight box bounds N)
template <int BK>
cudaError_t launch_halo_bk(int BN, int G, const CUtensorMap& mx, const CUtensorMap& mw,
                           const HaloArgs& t, cudaStream_t s) {
  switch (BN * 16 + G) {
    case 32 * 16 + 8: return launch_halo<BK, 32, (BK < 64 ? 8 : 4)>(mx, mw, t, s);
    case 32 * 16 + 4: return launch_halo<BK, 32, 4>(mx, mw, t, s);
    case 32 * 16 + 2: return launch_halo<BK, 32, 2>(mx, mw, t, s);
    case 32 * 16 + 1: return launch_halo<BK, 32, 1>(mx, mw, t, s);
    case 64 * 16 + 4: return launch_halo<BK, 64, (BK < 64 ? 4 : 2)>(mx, mw, t, s);
    case 64 * 16 + 2: return launch_halo<BK, 64, 2>(mx, mw, t, s);
    case 64 * 16 + 1: return launch_halo<BK, 64, 1>(mx, mw, t, s);
    case 128 * 16 + 2: return launch_halo<BK, 128, (BK < 64 ? 2 : 1)>(mx, mw, t, s);
    case 128 * 16 + 1: return launch_halo<BK, 128, 1>(mx, mw, t, s);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t conv3x3_tc_halo(const ConvArgs& a, unsigned* err, cudaStream_t s, bool* used) {
  *used = false;
  if (const char* e = getenv("LBPF_CONV_HALO"))
    if (atoi(e) == 0) return cudaSuccess;
  if (a.W % 128 || a.Cin % 16) return cudaSuccess;
  // the widest channel chunk: splitting 64 channels into 32-wide chunks (to
  // fit 8 rows per tile instead of 4) measured slower
  const int BK = a.Cin % 64 == 0 ? 64 : (a.Cin % 32 == 0 ? 32 : 16);
  int BN = 128;
  while (BN > 32 && a.Cout % BN) BN >>= 1;
  if (a.Cout % BN) return cudaSuccess;
  // rows per tile: about 256 accumulator columns (within shared memory), as
  // many tiles as SMs where the image allows, G dividing the image height
  int G = 256 / BN;
  if (BK == 64 && G > 4) G = 4;
  if (BK == 64 && BN == 64) G = 2;
  if (BK == 64 && BN == 128) G = 1;
  const long long row_tiles = (long long)a.N * a.H * (a.W / 128);
  while (G > 1 && (a.H % G || (row_tiles / G) * (a.Cout / BN) < 152)) G >>= 1;
  if (a.H % G) return cudaSuccess;
  const CUtensorMapSwizzle sw = swizzle_for(BK);
  CUtensorMap mx, mw;
  {
    const uint64_t dims[4] = {uint64_t(a.Cx), uint64_t(a.W), uint64_t(a.H), uint64_t(a.N)};
    const uint64_t strides[3] = {uint64_t(a.Cx) * 2, uint64_t(a.W) * a.Cx * 2,
                                 uint64_t(a.H) * a.W * a.Cx * 2};
    const uint32_t box[4] = {uint32_t(BK), 130, uint32_t(G), 1};
    if (!encode_tiled(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(a.x), dims,
                      strides, box, sw))
      return cudaErrorInvalidValue;
  }
  {
    // weights [ky][kx][Cout][Cin] viewed as (Cin, Cout, kx, ky)
    const uint64_t dims[4] = {uint64_t(a.Cin), uint64_t(a.Cout), 3, 3};
    const uint64_t strides[3] = {uint64_t(a.Cin) * 2, uint64_t(a.Cout) * a.Cin * 2,
                                 3ull * a.Cout * a.Cin * 2};
    const uint32_t box[4] = {uint32_t(BK), uint32_t(BN), 3, 1};
    if (!encode_tiled(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(a.w), dims,
                      strides, box, sw))
      return cudaErrorInvalidValue;
  }
  HaloArgs t;
  t.H = a.H;
  t.W = a.W;
  t.rows_t = a.H / G;
  t.cols_t = a.W / 128;
  t.ci_off = a.ci_off;
  t.nchunks = a.Cin / BK;
  t.ntiles_n = a.Cout / BN;
  t.ntiles = a.N * t.rows_t * t.cols_t * t.ntiles_n;
  t.Cy = a.Cy;
  t.co_off = a.co_off;
  t.relu = a.relu;
  t.Cout = a.Cout;
  t.bias = a.bias;
  t.mask = a.mask;
  t.y = a.y;
  t.err = err;
  // the head rides along when one tile holds every channel of a pixel
  const bool fuse = a.head_y && BN == a.Cout && a.co_off == 0 && a.head_out >= 1 &&
                    a.head_out <= 8 && !a.mask;
  t.head_w = fuse ? a.head_w : nullptr;
  t.head_b = fuse ? a.head_b : nullptr;
  t.head_y = fuse ? a.head_y : nullptr;
  t.head_out = fuse ? a.head_out : 0;
  if (a.head_done) *a.head_done = fuse ? 1 : 0;
  // the pooling of the next level rides along when a tile holds row pairs
  const bool fpool = a.pool_y && G % 2 == 0 && !a.mask && a.H % 2 == 0 && a.pool_Cy % 8 == 0 &&
                     a.pool_off % 8 == 0 && !fuse;
  t.pool_y = fpool ? a.pool_y : nullptr;
  t.pool_Cy = a.pool_Cy;
  t.pool_off = a.pool_off;
  if (a.pool_done) *a.pool_done = fpool ? 1 : 0;
  *used = true;
  switch (BK) {
    case 64: return launch_halo_bk<64>(BN, G, mx, mw, t, s);
    case 32: return launch_halo_bk<32>(BN, G, mx, mw, t, s);
    default: return launch_halo_bk<16>(BN, G, mx, mw, t, s);
  }
}

cudaError_t conv3x3_tc(const ConvArgs& a, unsigned* err, cudaStream_t s) {
  if (!conv3x3_tc_supported(a) || !err) return cudaErrorInvalidValue;
  {
    bool used = false;
    const cudaError_t e = conv3x3_tc_halo(a, err, s, &used);
    if (used || e != cudaSuccess) return e;
  }
  const long long npix = (long long)a.N * a.H * a.W;
  const int BK = a.Cin % 64 == 0 ? 64 : (a.Cin % 32 == 0 ? 32 : 16);
  // the widest N the channels allow: a tcgen05.mma costs about the same time
  // whatever its N, so wide tiles beat more tiles even when some SMs idle
  int BN = 256;
  while (BN > 32 && a.Cout % BN) BN >>= 1;
  if (const char* e = getenv("LBPF_CONV_MAX_BN")) {
    const int cap = atoi(e);
    while (BN > 32 && BN > cap) BN >>= 1;
  }
  const int BW = a.W % 128 == 0 ? 128 : 64;
  // sub-tiles per tile: about 256 accumulator columns per K step, as many
  // tiles as SMs where the image allows, G dividing the pixel tiles
  const long long mt = npix / 128;
  int G = 256 / BN;
  const int gmax = BN == 32 ? (BK < 64 ? 8 : 4) : (BN == 64 ? 4 : (BN == 128 ? 2 : 1));
  if (G > gmax) G = gmax;
  while (G > 1 && (mt % G || (mt / G) * (a.Cout / BN) < 152)) G >>= 1;
  if (const char* e = getenv("LBPF_CONV_G")) {
    const int want = atoi(e);
    while (G > 1 && G > want) G >>= 1;
  }
  CUtensorMap mx, mw;
  {
    const uint64_t dims[4] = {uint64_t(a.Cx), uint64_t(a.W), uint64_t(a.H), uint64_t(a.N)};
    const uint64_t strides[3] = {uint64_t(a.Cx) * 2, uint64_t(a.W) * a.Cx * 2,
                                 uint64_t(a.H) * a.W * a.Cx * 2};
    const uint32_t box[4] = {uint32_t(BK), uint32_t(BW), uint32_t(128 / BW), 1};
    if (!encode_tiled(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(a.x), dims,
                      strides, box, swizzle_for(BK)))
      return cudaErrorInvalidValue;
  }
  {
    const uint64_t dims[3] = {uint64_t(a.Cin), uint64_t(a.Cout), 9};
    const uint64_t strides[2] = {uint64_t(a.Cin) * 2, uint64_t(a.Cout) * a.Cin * 2};
    const uint32_t box[3] = {uint32_t(BK), uint32_t(BN), 1};
    if (!encode_tiled(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(a.w), dims,
                      strides, box, swizzle_for(BK)))
      return cudaErrorInvalidValue;
  }
  TcArgs t;
  t.H = a.H;
  t.W = a.W;
  t.BW = BW;
  t.ci_off = a.ci_off;
  t.nchunks = a.Cin / BK;
  t.Cy = a.Cy;
  t.co_off = a.co_off;
  t.relu = a.relu;
  t.bias = a.bias;
  t.mask = a.mask;
  t.y = a.y;
  t.err = err;
  t.mtiles = int(npix / 128);
  t.ntiles_n = a.Cout / BN;
  t.Cout = a.Cout;
  t.Cin = a.Cin;
  switch (BK) {
    case 64: return launch_bn<64>(BN, G, mx, mw, t, s);
    case 32: return launch_bn<32>(BN, G, mx, mw, t, s);
    default: return launch_bn<16>(BN, G, mx, mw, t, s);
  }
}

}  // namespace nn
}  // namespace lbk
