// Tensor-core 3x3 convolution of the U-Net surrogate on the 5th-generation
// tensor cores: implicit GEMM D[pixel][co] = sum over the nine taps and the
// input channels of x[pixel + shift(tap)][ci] w[tap][co][ci], then bias,
// ReLU, an optional mask, bf16 out.  The same kernel computes the data
// gradient on flipped / transposed weights.
//
// One CTA computes a tile of 128 pixels (one or two image rows) x BN output
// channels with the FP32 accumulator in tensor memory:
//   warp 0     TMA producer: per K step (one tap, BK input channels) a 4D box
//              of the NHWC input at the tap's shifted origin (zero fill
//              outside the image gives the convolution's zero padding) and a
//              3D box of the weights, into a stage of an S-deep ring
//   warp 1     allocates tensor memory; one lane issues tcgen05.mma
//              (kind::f16, bf16 x bf16 -> f32, M = 128, N = BN, K = 16) and
//              frees each stage through tcgen05.commit
//   warps 2-5  epilogue: tcgen05.ld of their 32-lane quarter of the
//              accumulator, bias / ReLU / mask, bf16 stores
// Every wait on a barrier is bounded; on a timeout the kernel sets bit 2 of
// *err, lets the copies and products already issued finish, frees its tensor
// memory and returns (the host turns the bit into an error status).
#include <cuda.h>

#include <cstdint>

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
  int Cy, co_off, relu;  // output channel stride / offset
  const float* bias;
  const bf16* mask;
  bf16* y;
  unsigned* err;
};

template <int BK, int BN>
struct TcShape {
  static constexpr int A_BYTES = 128 * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  // deep enough to cover latency, small enough for two CTAs per SM
  static constexpr int S = STAGE <= 24576 ? 4 : (STAGE <= 36864 ? 3 : 2);
  static constexpr int SMEM = S * STAGE + 1024;  // + alignment slack
  static constexpr uint32_t SBO = 8 * BK * 2;
  static constexpr uint32_t MODE = BK == 64 ? 2 : (BK == 32 ? 4 : 6);  // 128 / 64 / 32 B swizzle
  // kind::f16 instruction descriptor: D f32, A and B bf16, both K-major, N, M = 128
  static constexpr uint32_t IDESC =
      (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(128 >> 4) << 24);
  static constexpr uint32_t TCOLS = BN < 32 ? 32 : BN;
};

template <int BK, int BN>
__global__ void __launch_bounds__(kTcThreads, 1)
    conv3x3_tc_kernel(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mw,
                      const TcArgs a) {
  using Sh = TcShape<BK, BN>;
  constexpr int S = Sh::S;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[S], empty[S], accum;
  __shared__ uint32_t tmem_base;
  uint8_t* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long pix0 = (long long)blockIdx.x * 128;
  const int n0 = blockIdx.y * BN;
  const int w0 = int(pix0 % a.W), h0 = int((pix0 / a.W) % a.H);
  const int img = int(pix0 / ((long long)a.W * a.H));
  const int ksteps = 9 * a.nchunks;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accum, 1);
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, Sh::TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int ks = 0; ks < ksteps; ++ks) {
      const int st = ks % S, use = ks / S;
      if (ks >= S && !mbar_wait_bounded(&empty[st], uint32_t(use - 1) & 1u, kTcSpin)) {
        atomicOr(a.err, 2u);
        break;
      }
      const int tap = ks / a.nchunks, c0 = (ks % a.nchunks) * BK;
      const int ky = tap / 3, kx = tap % 3;
      uint8_t* sa = smem + st * Sh::STAGE;
      mbar_arrive_expect_tx(&full[st], Sh::STAGE);
      tma_load_4d(sa, &mx, &full[st], a.ci_off + c0, w0 + kx - 1, h0 + ky - 1, img);
      tma_load_3d(sa + Sh::A_BYTES, &mw, &full[st], c0, n0, tap);
      issued = ks + 1;
    }
    // every issued copy has landed before the CTA may finish
    for (int ks = issued > S ? issued - S : 0; ks < issued; ++ks)
      if (!mbar_wait_bounded(&full[ks % S], uint32_t(ks / S) & 1u, kTcSpin)) atomicOr(a.err, 2u);
  } else if (warp == 1 && lane == 0) {
    for (int ks = 0; ks < ksteps; ++ks) {
      const int st = ks % S;
      if (!mbar_wait_bounded(&full[st], uint32_t(ks / S) & 1u, kTcSpin)) {
        atomicOr(a.err, 2u);
        break;
      }
      tc_fence_after();
      const uint32_t sa = smem_addr(smem + st * Sh::STAGE), sb = sa + Sh::A_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)
        tc_mma(tmem, umma_desc(sa + kk * 32, Sh::SBO, Sh::MODE),
               umma_desc(sb + kk * 32, Sh::SBO, Sh::MODE), Sh::IDESC, (ks | kk) != 0);
      tc_commit(&empty[st]);
    }
    tc_commit(&accum);  // also after an abort: the products issued so far complete
  } else if (warp >= 2) {
    bool ok = mbar_wait_bounded(&accum, 0u, kTcSpin);
    ok = __all_sync(0xffffffffu, ok);
    tc_fence_after();
    if (!ok) {
      if (lane == 0) atomicOr(a.err, 2u);
    } else {
      const int q = warp & 3;  // tensor-memory lanes 32q .. 32q + 31
      const int m = q * 32 + lane;
      const long long p =
          ((long long)img * a.H + h0 + m / a.BW) * a.W + w0 + (m % a.BW);
      bf16* yrow = a.y + p * a.Cy + a.co_off + n0;
      const bf16* mrow = a.mask ? a.mask + p * a.Cy + a.co_off + n0 : nullptr;
#pragma unroll 1
      for (int c = 0; c < BN; c += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(c), r);
        uint4 mk[4];
        if (mrow)
#pragma unroll
          for (int v = 0; v < 4; ++v) mk[v] = reinterpret_cast<const uint4*>(mrow + c)[v];
        uint32_t out[16];
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
          float v0 = __uint_as_float(r[j]), v1 = __uint_as_float(r[j + 1]);
          if (a.bias) {
            v0 += a.bias[n0 + c + j];
            v1 += a.bias[n0 + c + j + 1];
          }
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
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, Sh::TCOLS);
  }
}

CUtensorMapSwizzle swizzle_for(int bk) {
  return bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                  : (bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
}

template <int BK, int BN>
cudaError_t launch_tc(const ConvArgs& c, const CUtensorMap& mx, const CUtensorMap& mw,
                      const TcArgs& t, unsigned grid_x, cudaStream_t s) {
  using Sh = TcShape<BK, BN>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_kernel<BK, BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  conv3x3_tc_kernel<BK, BN>
      <<<dim3(grid_x, unsigned(c.Cout / BN)), kTcThreads, Sh::SMEM, s>>>(mx, mw, t);
  return cudaGetLastError();
}

template <int BK>
cudaError_t launch_bn(int bn, const ConvArgs& c, const CUtensorMap& mx, const CUtensorMap& mw,
                      const TcArgs& t, unsigned gx, cudaStream_t s) {
  switch (bn) {
    case 32: return launch_tc<BK, 32>(c, mx, mw, t, gx, s);
    case 64: return launch_tc<BK, 64>(c, mx, mw, t, gx, s);
    case 128: return launch_tc<BK, 128>(c, mx, mw, t, gx, s);
    case 256: return launch_tc<BK, 256>(c, mx, mw, t, gx, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool conv3x3_tc_supported(const ConvArgs& a) {
  const long long npix = (long long)a.N * a.H * a.W;
  const bool rows = a.W % 128 == 0 || (a.W == 64 && a.H % 2 == 0);
  return rows && npix % 128 == 0 && a.Cin % 16 == 0 && a.Cout % 32 == 0 && a.Cx % 8 == 0 &&
         a.Cy % 8 == 0 && a.ci_off % 8 == 0 && a.co_off % 8 == 0 && a.ci_off + a.Cin <= a.Cx &&
         a.co_off + a.Cout <= a.Cy;
}

cudaError_t conv3x3_tc(const ConvArgs& a, unsigned* err, cudaStream_t s) {
  if (!conv3x3_tc_supported(a) || !err) return cudaErrorInvalidValue;
  const long long npix = (long long)a.N * a.H * a.W;
  const int BK = a.Cin % 64 == 0 ? 64 : (a.Cin % 32 == 0 ? 32 : 16);
  int BN = 256;
  while (BN > 32 && a.Cout % BN) BN >>= 1;
  // small grids: split the channels further so that every SM gets work
  while (BN > 32 && (npix / 128) * (a.Cout / BN) < 2 * 152) BN >>= 1;
  const int BW = a.W % 128 == 0 ? 128 : 64;
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
  const unsigned gx = unsigned(npix / 128);
  switch (BK) {
    case 64: return launch_bn<64>(BN, a, mx, mw, t, gx, s);
    case 32: return launch_bn<32>(BN, a, mx, mw, t, gx, s);
    default: return launch_bn<16>(BN, a, mx, mw, t, gx, s);
  }
}

}  // namespace nn
}  // namespace lbk
