// BF16 U-Net surrogate of the coupled step (training and inference on the
// project's own kernels, unet.cu) and its use as a block propagator with the
// LB solver as fallback and judge.
//
// Network (levels L, base channels C0, channels C_l = C0 2^l):
//   encoder level l: conv3x3(in -> C_l) ReLU, conv3x3(C_l -> C_l) ReLU [= skip_l];
//                    2x2 average pooling feeds level l + 1
//   decoder level l: nearest 2x upsampling of the level below, conv3x3(C_{l+1} -> C_l)
//                    ReLU [= up_l], concatenation [up_l | skip_l], conv3x3(2C_l -> C_l)
//                    ReLU, conv3x3(C_l -> C_l) ReLU
//   head: 1x1 convolution (C0 -> out channels), FP32, predicting the residual
// Activations and weights are bf16 (weights keep an FP32 master copy for
// Adam); every GEMM accumulates in FP32.  Inputs are padded to 16 channels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbpf.h"
#include "lbpf_handle.cuh"
#include "unet.cuh"

using lbk::nn::bf16;

namespace {

// one 3x3 convolution layer
struct ConvLayer {
  int cin = 0, cout = 0;
  size_t nw = 0;
  float *w = nullptr, *b = nullptr, *gw = nullptr, *gb = nullptr;
  float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
  bf16 *wb = nullptr, *wt = nullptr;  // bf16 weights and their flip-transpose
};

struct Act {  // NHWC bf16 buffer
  bf16* p = nullptr;
  int c = 0, h = 0, w = 0;
};

// SplitMix64-driven uniform numbers for the weight initialisation
uint64_t mix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

struct lbpf_unet {
  lbpf_unet_cfg cfg;
  cudaStream_t stream = nullptr;
  int L = 0;
  std::vector<int> C, H, W;
  std::vector<ConvLayer> enc_a, enc_b, up, dec_a, dec_b;
  // head
  float *hw = nullptr, *hb = nullptr, *ghw = nullptr, *ghb = nullptr;
  float *mhw = nullptr, *vhw = nullptr, *mhb = nullptr, *vhb = nullptr;
  // activations and their gradients
  Act xin;                                   // packed input, 16 channels
  std::vector<Act> ea, cat, pool, u, da, db;  // per level
  Act bottom;                                // encoder output of the last level
  std::vector<Act> g_ea, g_cat, g_pool, g_u, g_da, g_db;
  Act g_bottom;
  float *y = nullptr, *gy = nullptr, *loss = nullptr;
  unsigned* d_err = nullptr;  // bit 2: a tensor-core kernel timed out
  float* wpart = nullptr;     // partial sums of the weight, bias and head gradients
  size_t wpart_cap = 0;       // ... in floats
  // tables of the one-launch Adam step (every parameter tensor) and
  // flip-transpose (every convolution), in device memory
  lbk::nn::AdamSeg* adam_segs = nullptr;
  lbk::nn::FlipSeg* flip_segs = nullptr;
  int n_adam = 0, n_flip = 0;
  long long adam_blocks = 0, flip_blocks = 0;
  int tensor_path = 1;        // convolutions on the tcgen05 kernel where possible
  // block propagator scratch (allocated on first use): network input x,
  // output y, current planes F (phi, U, ux, uy, rho), predicted planes F1
  // (phi, U, ux, uy, phi(t-1)), FP64 sums and interface crossings
  float *px = nullptr, *py = nullptr, *pF = nullptr, *pF1 = nullptr;
  float *tx = nullptr, *tt = nullptr;  // training minibatch (lbpf_surrogate_train)
  double *psum = nullptr, *pcross = nullptr;
  double* ppart = nullptr;  // partial sums of the prediction's FP64 reduction
  // the prediction phase of a block as a CUDA graph per buffer parity, with
  // the key it was captured for; results land in pinned host memory
  cudaGraphExec_t pgraph[2] = {nullptr, nullptr};
  const void* pkey_pops[2] = {nullptr, nullptr};
  lbpf_surrogate_cfg pkey_cfg[2];
  cudaStream_t pkey_stream[2] = {nullptr, nullptr};
  double* hres = nullptr;  // [0..2] sums, [3..10] crossings (predicted, current), [11] error word
  std::vector<void*> allocs;
  size_t bytes = 0;
  int t = 0;  // Adam step
  char msg[256] = {0};
};

namespace {

constexpr int kWgradChunk = 4096;  // pixels per chunk of the per-tap weight gradient

int ufail(lbpf_unet* n, int code, const char* fmt, ...) {
  if (!n) return code;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(n->msg, sizeof(n->msg), fmt, ap);
  va_end(ap);
  return code;
}

#define UCK(n, call)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return ufail(n, LBPF_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                   __LINE__);                                                             \
  } while (0)

template <typename Tp>
cudaError_t dalloc(lbpf_unet* n, Tp** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(Tp) + 16);
  if (e != cudaSuccess) return e;
  n->allocs.push_back(q);
  n->bytes += count * sizeof(Tp);
  *p = static_cast<Tp*>(q);
  return cudaMemset(q, 0, count * sizeof(Tp));
}

cudaError_t act(lbpf_unet* n, Act* a, int c, int h, int w) {
  a->c = c;
  a->h = h;
  a->w = w;
  return dalloc(n, &a->p, size_t(n->cfg.batch) * h * w * c);
}

// He-uniform initialisation in FP32, seeded
cudaError_t make_conv(lbpf_unet* n, ConvLayer* l, int cin, int cout, int real_cin,
                      uint64_t seed) {
  l->cin = cin;
  l->cout = cout;
  l->nw = size_t(9) * cout * cin;
  cudaError_t e;
  float** f32[] = {&l->w, &l->gw, &l->mw, &l->vw};
  for (float** p : f32)
    if ((e = dalloc(n, p, l->nw)) != cudaSuccess) return e;
  float** b32[] = {&l->b, &l->gb, &l->mb, &l->vb};
  for (float** p : b32)
    if ((e = dalloc(n, p, size_t(cout))) != cudaSuccess) return e;
  if ((e = dalloc(n, &l->wb, l->nw)) != cudaSuccess) return e;
  if ((e = dalloc(n, &l->wt, l->nw)) != cudaSuccess) return e;
  std::vector<float> hw(l->nw, 0.f);
  std::vector<bf16> hb(l->nw);
  const float bound = std::sqrt(6.0f / float(9 * real_cin));
  for (size_t i = 0; i < l->nw; ++i) {
    const int ci = int(i % cin);
    if (ci >= real_cin) continue;  // padded input channels stay zero
    const double u = double(mix(seed ^ (i * 0x9E3779B97F4A7C15ull)) >> 11) * 0x1.0p-53;
    hw[i] = float((2.0 * u - 1.0) * bound);
  }
  for (size_t i = 0; i < l->nw; ++i) hb[i] = __float2bfloat16(hw[i]);
  if ((e = cudaMemcpy(l->w, hw.data(), l->nw * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  return cudaMemcpy(l->wb, hb.data(), l->nw * 2, cudaMemcpyHostToDevice);
}

// head: the 1x1 head to fuse into this layer's epilogue where the kernel can
// (*head_done says whether it did)
int conv_fwd(lbpf_unet* n, const ConvLayer& l, const Act& x, int xoff, const Act& y, int yoff,
             int* head_done = nullptr, const Act* pool = nullptr, int* pool_done = nullptr) {
  lbk::nn::ConvArgs a{};
  a.x = x.p;
  a.Cx = x.c;
  a.ci_off = xoff;
  a.Cin = l.cin;
  a.w = l.wb;
  a.bias = l.b;
  a.y = y.p;
  a.Cy = y.c;
  a.co_off = yoff;
  a.Cout = l.cout;
  a.N = n->cfg.batch;
  a.H = x.h;
  a.W = x.w;
  a.relu = 1;
  a.mask = nullptr;
  a.tensor_path = n->tensor_path;
  a.err = n->d_err;
  if (head_done) {
    a.head_w = n->hw;
    a.head_b = n->hb;
    a.head_y = n->y;
    a.head_out = n->cfg.out_ch;
    a.head_done = head_done;
  }
  if (pool && pool_done) {  // the next level's pooled input, channels 0 .. Cout
    a.pool_y = pool->p;
    a.pool_Cy = pool->c;
    a.pool_off = 0;
    a.pool_done = pool_done;
  }
  UCK(n, lbk::nn::conv3x3(a, n->stream));
  return LBPF_OK;
}

// backward of one layer whose input is x[xoff..] and whose pre-activation
// gradient is g[goff..]: weight and bias gradients, and (if gx) the input
// gradient, optionally masked by `mask` (same layout as gx).
int conv_bwd(lbpf_unet* n, const ConvLayer& l, const Act& x, int xoff, const Act& g, int goff,
             const Act* gx, int gxoff, const Act* mask) {
  const long long npix = (long long)n->cfg.batch * x.h * x.w;
  lbk::nn::WgradArgs wa{};
  wa.x = x.p;
  wa.Cx = x.c;
  wa.ci_off = xoff;
  wa.Cin = l.cin;
  wa.dy = g.p;
  wa.Cdy = g.c;
  wa.co_off = goff;
  wa.Cout = l.cout;
  wa.dw = l.gw;
  wa.db = l.gb;
  wa.npix = npix;
  wa.H = x.h;
  wa.W = x.w;
  wa.chunk = kWgradChunk;
  wa.part = n->wpart;
  wa.part_cap = n->wpart_cap;
  UCK(n, lbk::nn::wgrad3x3(wa, n->stream));  // weight and bias gradients
  if (gx) {
    lbk::nn::ConvArgs a{};
    a.x = g.p;
    a.Cx = g.c;
    a.ci_off = goff;
    a.Cin = l.cout;
    a.w = l.wt;
    a.bias = nullptr;
    a.y = gx->p;
    a.Cy = gx->c;
    a.co_off = gxoff;
    a.Cout = l.cin;
    a.N = n->cfg.batch;
    a.H = x.h;
    a.W = x.w;
    a.relu = 0;
    a.mask = mask ? mask->p : nullptr;
    a.tensor_path = n->tensor_path;
    a.err = n->d_err;
    UCK(n, lbk::nn::conv3x3(a, n->stream));
  }
  return LBPF_OK;
}

std::vector<ConvLayer*> all_layers(lbpf_unet* n) {
  std::vector<ConvLayer*> v;
  for (auto* vec : {&n->enc_a, &n->enc_b, &n->up, &n->dec_a, &n->dec_b})
    for (auto& l : *vec) v.push_back(&l);
  return v;
}

// forward pass on the packed input n->xin; output n->y (FP32 NHWC, out_ch)
int forward(lbpf_unet* n) {
  const int L = n->L;
  int rc;
  for (int l = 0; l < L; ++l) {
    const Act& in = l == 0 ? n->xin : n->pool[l];
    if ((rc = conv_fwd(n, n->enc_a[l], in, 0, n->ea[l], 0))) return rc;
    if (l < L - 1) {
      // the 2 x 2 pooling into the next level rides in the epilogue where it can
      int pooled = 0;
      if ((rc = conv_fwd(n, n->enc_b[l], n->ea[l], 0, n->cat[l], n->C[l], nullptr, &n->pool[l + 1],
                         &pooled)))
        return rc;
      if (!pooled)
        UCK(n, lbk::nn::avgpool2(n->cat[l].p, n->cat[l].c, n->C[l], n->pool[l + 1].p, n->C[l], 0,
                                 n->C[l], n->cfg.batch, n->H[l], n->W[l], n->stream));
    } else {
      if ((rc = conv_fwd(n, n->enc_b[l], n->ea[l], 0, n->bottom, 0))) return rc;
    }
  }
  const Act* d = &n->bottom;
  int head_done = 0;
  for (int l = L - 2; l >= 0; --l) {
    UCK(n, lbk::nn::upsample2(d->p, n->u[l].p, n->C[l + 1], n->cfg.batch, n->H[l], n->W[l],
                              n->stream));
    if ((rc = conv_fwd(n, n->up[l], n->u[l], 0, n->cat[l], 0))) return rc;
    if ((rc = conv_fwd(n, n->dec_a[l], n->cat[l], 0, n->da[l], 0))) return rc;
    // the last convolution carries the 1x1 head in its epilogue where it can
    if ((rc = conv_fwd(n, n->dec_b[l], n->da[l], 0, n->db[l], 0, l == 0 ? &head_done : nullptr)))
      return rc;
    d = &n->db[l];
  }
  if (!head_done) {
    const long long npix = (long long)n->cfg.batch * n->H[0] * n->W[0];
    UCK(n, lbk::nn::head_fwd(L > 1 ? n->db[0].p : n->bottom.p, n->C[0], n->hw, n->hb, n->y,
                             n->cfg.out_ch, npix, n->stream));
  }
  return LBPF_OK;
}

// loss and gradients for targets t (FP32 NHWC, out_ch); gradients accumulate
int backward(lbpf_unet* n, const float* t) {
  const int L = n->L, B = n->cfg.batch;
  const long long npix = (long long)B * n->H[0] * n->W[0];
  int rc;
  UCK(n, lbk::nn::flip_multi(n->flip_segs, n->n_flip, n->flip_blocks, n->stream));
  UCK(n, cudaMemsetAsync(n->loss, 0, sizeof(float), n->stream));
  UCK(n, lbk::nn::mse(n->y, t, npix * n->cfg.out_ch, n->gy, n->loss, n->stream));
  const Act& top = L > 1 ? n->db[0] : n->bottom;
  Act& g_top = L > 1 ? n->g_db[0] : n->g_bottom;
  UCK(n, lbk::nn::head_bwd(top.p, n->C[0], n->hw, n->gy, n->cfg.out_ch, npix, g_top.p, n->ghw,
                           n->ghb, n->wpart, n->wpart_cap, n->stream));
  // decoder, from the top level down to the bottom
  for (int l = 0; l < L - 1; ++l) {
    if ((rc = conv_bwd(n, n->dec_b[l], n->da[l], 0, n->g_db[l], 0, &n->g_da[l], 0, &n->da[l])))
      return rc;
    if ((rc = conv_bwd(n, n->dec_a[l], n->cat[l], 0, n->g_da[l], 0, &n->g_cat[l], 0, nullptr)))
      return rc;
    UCK(n, lbk::nn::relu_mask(n->g_cat[l].p, n->g_cat[l].c, 0, n->cat[l].p, n->cat[l].c, 0,
                              n->C[l], (long long)B * n->H[l] * n->W[l], n->stream));
    if ((rc = conv_bwd(n, n->up[l], n->u[l], 0, n->g_cat[l], 0, &n->g_u[l], 0, nullptr))) return rc;
    const Act& below = l + 1 < L - 1 ? n->db[l + 1] : n->bottom;
    Act& g_below = l + 1 < L - 1 ? n->g_db[l + 1] : n->g_bottom;
    UCK(n, lbk::nn::upsample2_bwd_mask(n->g_u[l].p, g_below.p, below.p, n->C[l + 1], B, n->H[l],
                                       n->W[l], n->stream));
  }
  // encoder, from the bottom level up
  for (int l = L - 1; l >= 0; --l) {
    const Act* gb;
    int gboff;
    const Act* eb_out;
    if (l == L - 1) {
      gb = &n->g_bottom;
      gboff = 0;
      eb_out = &n->bottom;
    } else {
      // skip gradient = from the concatenation + from the pooling path, masked
      UCK(n, lbk::nn::avgpool2_bwd_add_mask(n->g_cat[l].p, n->g_pool[l + 1].p, n->cat[l].p,
                                            n->cat[l].c, n->C[l], n->C[l], B, n->H[l], n->W[l],
                                            n->stream));
      gb = &n->g_cat[l];
      gboff = n->C[l];
      eb_out = &n->cat[l];
    }
    (void)eb_out;
    if ((rc = conv_bwd(n, n->enc_b[l], n->ea[l], 0, *gb, gboff, &n->g_ea[l], 0, &n->ea[l])))
      return rc;
    const Act& in = l == 0 ? n->xin : n->pool[l];
    if ((rc = conv_bwd(n, n->enc_a[l], in, 0, n->g_ea[l], 0, l == 0 ? nullptr : &n->g_pool[l], 0,
                       nullptr)))
      return rc;
  }
  return LBPF_OK;
}

// the device error word after a synchronisation: a tensor-core kernel timed out
int check_err(lbpf_unet* n) {
  unsigned e = 0;
  UCK(n, cudaMemcpyAsync(&e, n->d_err, sizeof(e), cudaMemcpyDeviceToHost, n->stream));
  UCK(n, cudaStreamSynchronize(n->stream));
  if (e) return ufail(n, LBPF_ETIMEDOUT, "a tensor-core convolution gave up waiting (code %u)", e);
  return LBPF_OK;
}

int adam_all(lbpf_unet* n, float lr) {
  ++n->t;
  UCK(n, lbk::nn::adam_multi(n->adam_segs, n->n_adam, n->adam_blocks, lr, 0.9f, 0.999f, 1e-8f,
                             n->t, n->stream));
  return LBPF_OK;
}

// the device tables of adam_all and of the weights' flip-transpose
cudaError_t build_seg_tables(lbpf_unet* n) {
  using lbk::nn::kSegBlock;
  std::vector<lbk::nn::AdamSeg> as;
  std::vector<lbk::nn::FlipSeg> fs;
  long long ab = 0, fb = 0;
  auto add = [&](float* w, float* g, float* m, float* v, bf16* wb, long long cnt) {
    as.push_back({w, g, m, v, wb, cnt, ab});
    ab += (cnt + kSegBlock - 1) / kSegBlock;
  };
  for (ConvLayer* l : all_layers(n)) {
    add(l->w, l->gw, l->mw, l->vw, l->wb, (long long)l->nw);
    add(l->b, l->gb, l->mb, l->vb, nullptr, l->cout);
    fs.push_back({l->wb, l->wt, l->cout, l->cin, fb});
    fb += (9LL * l->cout * l->cin + kSegBlock - 1) / kSegBlock;
  }
  add(n->hw, n->ghw, n->mhw, n->vhw, nullptr, (long long)n->cfg.out_ch * n->C[0]);
  add(n->hb, n->ghb, n->mhb, n->vhb, nullptr, n->cfg.out_ch);
  cudaError_t e = dalloc(n, &n->adam_segs, as.size());
  if (e == cudaSuccess) e = dalloc(n, &n->flip_segs, fs.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(n->adam_segs, as.data(), as.size() * sizeof(as[0]), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(n->flip_segs, fs.data(), fs.size() * sizeof(fs[0]), cudaMemcpyHostToDevice);
  n->n_adam = int(as.size());
  n->n_flip = int(fs.size());
  n->adam_blocks = ab;
  n->flip_blocks = fb;
  return e;
}

// pack FP32 NHWC (in_ch <= 16) into the bf16 16-channel input buffer: one
// pixel per thread, its 16 outputs written as two 16-byte stores
__global__ void pack_input_kernel(const float* x, int cin, int vec4, bf16* out, long long npix) {
  lbk::nn::pdl_trigger();
  lbk::nn::pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    __align__(16) bf16 v[16];
    if (vec4) {  // four 16-byte aligned channels (the propagator's phi, U, ux, uy)
      const float4 f = reinterpret_cast<const float4*>(x)[p];
      v[0] = __float2bfloat16(f.x);
      v[1] = __float2bfloat16(f.y);
      v[2] = __float2bfloat16(f.z);
      v[3] = __float2bfloat16(f.w);
#pragma unroll
      for (int c = 4; c < 16; ++c) v[c] = __float2bfloat16(0.f);
    } else {
#pragma unroll
      for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16(c < cin ? x[p * cin + c] : 0.f);
    }
    uint4* o = reinterpret_cast<uint4*>(out + p * 16);
    o[0] = reinterpret_cast<const uint4*>(v)[0];
    o[1] = reinterpret_cast<const uint4*>(v)[1];
  }
}

int pack_input(lbpf_unet* n, const float* x) {
  const long long npix = (long long)n->cfg.batch * n->H[0] * n->W[0];
  long long blocks = (npix + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  // four channels are read as one float4 where x is 16-byte aligned
  const int vec4 = n->cfg.in_ch == 4 && (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
  UCK(n, lbk::nn::launch_pdl(pack_input_kernel, dim3(unsigned(blocks)), dim3(256), 0, n->stream,
                             x, n->cfg.in_ch, vec4, n->xin.p, npix));
  return LBPF_OK;
}

// parameter views, in a fixed order: per layer (w, b) in all_layers order, then the head
struct ParamView {
  float* p;
  float* g;
  size_t n;
};
std::vector<ParamView> params(lbpf_unet* n) {
  std::vector<ParamView> v;
  for (ConvLayer* l : all_layers(n)) {
    v.push_back({l->w, l->gw, l->nw});
    v.push_back({l->b, l->gb, size_t(l->cout)});
  }
  v.push_back({n->hw, n->ghw, size_t(n->cfg.out_ch) * n->C[0]});
  v.push_back({n->hb, n->ghb, size_t(n->cfg.out_ch)});
  return v;
}

__global__ void to_bf16_kernel(const float* w, bf16* wb, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16(w[i]);
}

// predicted planes: f' = f + res_scale y; phi(t-1)' = phi' - (phi' - phi) / n_block
__global__ void apply_kernel(const float* F, const float* y, const lbk::Vec4 rs, float inv_nb,
                             long long n, float* F1) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      v[c] = F[c * n + i] + rs.v[c] * y[i * 4 + c];
      F1[c * n + i] = v[c];
    }
    F1[4 * n + i] = v[0] - (v[0] - F[i]) * inv_nb;
  }
}

// phi = 0 crossings of a field plane along the four axis rays from (icx, icy):
// the first change from phi >= 0 to phi < 0, linearly interpolated, as a
// distance from the origin; -1 where there is none (the definition of
// lbpf_diag.iface_pos)
__global__ void plane_crossing_kernel(const float* phi, int nx, int ny, int bcx, int bcy, int icx,
                                      int icy, double* out) {
  // one warp per ray, 32 positions per round
  const int r = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (r >= 4) return;
  const int axis = r / 2, dir = (r & 1) ? -1 : 1;
  const int n = axis == 0 ? nx : ny, bc = axis == 0 ? bcx : bcy;
  const int start = axis == 0 ? icx : icy;
  auto at = [&](int d) -> float {  // phi at distance d along the ray (d in range)
    int v = start + dir * d;
    if (bc == LBPF_BC_PERIODIC) v = ((v % n) + n) % n;
    return axis == 0 ? phi[(long long)icy * nx + v] : phi[(long long)v * nx + icx];
  };
  double res = -1.0;
  if (at(0) >= 0.f) {
    int limit = bc == LBPF_BC_PERIODIC ? n / 2 : n;  // distances 1 .. limit - 1
    if (bc != LBPF_BC_PERIODIC) {
      const int room = dir > 0 ? n - 1 - start : start;  // positions inside the domain
      if (room + 1 < limit) limit = room + 1;
    }
    for (int base = 1; base < limit; base += 32) {
      const int d = base + lane;
      const bool neg = d < limit && at(d) < 0.f;
      const unsigned m = __ballot_sync(0xffffffffu, neg);
      if (m) {
        const int dd = base + __ffs(m) - 1;
        const double p = at(dd), prev = at(dd - 1);
        res = double(dd - 1) + prev / (prev - p);
        break;
      }
    }
  }
  if (lane == 0) out[r] = res;
}

// U += k (1 - clamp(phi, -1, 1)) / 2 on the predicted planes
__global__ void correct_kernel(float* F1, long long n, float k) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float ph = fminf(fmaxf(F1[i], -1.f), 1.f);
    F1[n + i] += k * 0.5f * (1.f - ph);
  }
}

__global__ void target_kernel(const float* x0, const float* x1, const lbk::Vec4 g, long long n4,
                              float* t) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x)
    t[i] = (x1[i] - x0[i]) * g.v[i & 3];
}

// One minibatch of the training loop: pairs idx[0..B) of X / T ([n][H][W][4],
// channels phi, U, ux, uy), mirrored as `flip` says (1: rows, uy negated;
// 2: columns, ux negated), into xb / tb ([B][H][W][4]).  A copy up to the
// sign: the values are those of the stored pairs exactly.
__global__ void gather_pairs_kernel(const float* __restrict__ X, const float* __restrict__ T,
                                    const int* __restrict__ idx, int flip, int H, int W,
                                    long long n, float* __restrict__ xb, float* __restrict__ tb) {
  const long long hw4 = (long long)H * W * 4;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / hw4, r = e % hw4;
    int i = int(r / (W * 4)), j = int((r / 4) % W);
    const int c = int(r & 3);
    if (flip == 1) i = H - 1 - i;
    if (flip == 2) j = W - 1 - j;
    const float sg = (flip == 1 && c == 3) || (flip == 2 && c == 2) ? -1.f : 1.f;
    const long long src = (long long)idx[b] * hw4 + ((long long)i * W + j) * 4 + c;
    xb[e] = sg * X[src];
    tb[e] = sg * T[src];
  }
}

int grid_of(long long n) {
  long long b = (n + 255) / 256;
  return int(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

int sfail(lbpf* h, int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(h->msg, sizeof(h->msg), fmt, ap);
  va_end(ap);
  return code;
}

#define SCK(h, call)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return sfail(h, LBPF_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                   __LINE__);                                                             \
  } while (0)

int check_cfg(const lbpf_surrogate_cfg* c) {
  if (!c || c->steps_per_block < 1 || c->judge_every < 0 || !(c->drift_tol >= 0.0) ||
      !(c->iface_tol >= 0.0) || !(c->iface_budget >= 0.0) || !(c->iface_rel_tol >= 0.0))
    return LBPF_EINVAL;
  for (int k = 0; k < 4; ++k)
    if (!(std::isfinite(c->shift[k]) && std::isfinite(c->scale[k]) && c->scale[k] != 0.f &&
          std::isfinite(c->res_scale[k])))
      return LBPF_EINVAL;
  return LBPF_OK;
}

lbk::Vec4 vec4(const float* v) {
  lbk::Vec4 r;
  for (int k = 0; k < 4; ++k) r.v[k] = v[k];
  return r;
}

// largest |a_r - b_r| over the rays valid (>= 0) in both; -1 if none
double ray_diff(const double* a, const double* b) {
  double m = -1.0;
  for (int r = 0; r < 4; ++r)
    if (a[r] >= 0.0 && b[r] >= 0.0) m = std::fmax(m, std::fabs(a[r] - b[r]));
  return m;
}

}  // namespace

extern "C" {

lbpf_status lbpf_unet_create(const lbpf_unet_cfg* cfg, void* stream, lbpf_unet_t** out) {
  if (!cfg || !out) return LBPF_EINVAL;
  *out = nullptr;
  const int L = cfg->levels;
  if (L < 1 || L > 6 || cfg->base_ch < 32 || cfg->base_ch % 32 || cfg->in_ch < 1 ||
      cfg->in_ch > 16 || cfg->out_ch < 1 || cfg->out_ch > 4 || cfg->batch < 1 ||
      cfg->height < 1 || cfg->width < 1 || cfg->base_ch > 32) {
    fprintf(stderr, "lbpf_unet_create: unsupported configuration\n");
    return LBPF_EINVAL;
  }
  if ((cfg->width >> (L - 1)) % 64 != 0 || (cfg->height >> (L - 1)) < 1 ||
      cfg->width % (1 << (L - 1)) || cfg->height % (1 << (L - 1))) {
    fprintf(stderr,
            "lbpf_unet_create: width / 2^(levels-1) must be a multiple of 64 and height "
            "divisible by 2^(levels-1)\n");
    return LBPF_EINVAL;
  }
  lbpf_unet* n = new (std::nothrow) lbpf_unet();
  if (!n) return LBPF_ENOMEM;
  n->cfg = *cfg;
  n->stream = static_cast<cudaStream_t>(stream);
  n->L = L;
  for (int l = 0; l < L; ++l) {
    n->C.push_back(cfg->base_ch << l);
    n->H.push_back(cfg->height >> l);
    n->W.push_back(cfg->width >> l);
  }
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  uint64_t sd = cfg->seed;
  n->enc_a.resize(L);
  n->enc_b.resize(L);
  n->up.resize(L > 1 ? L - 1 : 0);
  n->dec_a.resize(L > 1 ? L - 1 : 0);
  n->dec_b.resize(L > 1 ? L - 1 : 0);
  for (int l = 0; l < L; ++l) {
    const int cin = l == 0 ? 16 : n->C[l - 1];
    chk(make_conv(n, &n->enc_a[l], cin, n->C[l], l == 0 ? cfg->in_ch : cin, mix(sd += 101)));
    chk(make_conv(n, &n->enc_b[l], n->C[l], n->C[l], n->C[l], mix(sd += 101)));
  }
  for (int l = 0; l < L - 1; ++l) {
    chk(make_conv(n, &n->up[l], n->C[l + 1], n->C[l], n->C[l + 1], mix(sd += 101)));
    chk(make_conv(n, &n->dec_a[l], 2 * n->C[l], n->C[l], 2 * n->C[l], mix(sd += 101)));
    chk(make_conv(n, &n->dec_b[l], n->C[l], n->C[l], n->C[l], mix(sd += 101)));
  }
  const size_t nh = size_t(cfg->out_ch) * n->C[0];
  float** hp[] = {&n->hw, &n->ghw, &n->mhw, &n->vhw};
  for (float** p : hp) chk(dalloc(n, p, nh));
  float** hbp[] = {&n->hb, &n->ghb, &n->mhb, &n->vhb};
  for (float** p : hbp) chk(dalloc(n, p, size_t(cfg->out_ch)));
  if (e == cudaSuccess) {
    std::vector<float> h(nh);
    const float bound = std::sqrt(6.0f / float(n->C[0])) * 0.1f;  // small head: start near 0
    for (size_t i = 0; i < nh; ++i)
      h[i] = float((2.0 * (double(mix(cfg->seed ^ (777 + i)) >> 11) * 0x1.0p-53) - 1.0) * bound);
    chk(cudaMemcpy(n->hw, h.data(), nh * 4, cudaMemcpyHostToDevice));
  }
  n->ea.resize(L);
  n->g_ea.resize(L);
  n->pool.resize(L);
  n->g_pool.resize(L);
  n->cat.resize(L);
  n->g_cat.resize(L);
  n->u.resize(L);
  n->g_u.resize(L);
  n->da.resize(L);
  n->g_da.resize(L);
  n->db.resize(L);
  n->g_db.resize(L);
  chk(act(n, &n->xin, 16, n->H[0], n->W[0]));
  for (int l = 0; l < L; ++l) {
    chk(act(n, &n->ea[l], n->C[l], n->H[l], n->W[l]));
    chk(act(n, &n->g_ea[l], n->C[l], n->H[l], n->W[l]));
    if (l > 0) {
      chk(act(n, &n->pool[l], n->C[l - 1], n->H[l], n->W[l]));
      chk(act(n, &n->g_pool[l], n->C[l - 1], n->H[l], n->W[l]));
    }
    if (l < L - 1) {
      chk(act(n, &n->cat[l], 2 * n->C[l], n->H[l], n->W[l]));
      chk(act(n, &n->g_cat[l], 2 * n->C[l], n->H[l], n->W[l]));
      chk(act(n, &n->u[l], n->C[l + 1], n->H[l], n->W[l]));
      chk(act(n, &n->g_u[l], n->C[l + 1], n->H[l], n->W[l]));
      chk(act(n, &n->da[l], n->C[l], n->H[l], n->W[l]));
      chk(act(n, &n->g_da[l], n->C[l], n->H[l], n->W[l]));
      chk(act(n, &n->db[l], n->C[l], n->H[l], n->W[l]));
      chk(act(n, &n->g_db[l], n->C[l], n->H[l], n->W[l]));
    }
  }
  chk(act(n, &n->bottom, n->C[L - 1], n->H[L - 1], n->W[L - 1]));
  chk(act(n, &n->g_bottom, n->C[L - 1], n->H[L - 1], n->W[L - 1]));
  const size_t ny = size_t(cfg->batch) * n->H[0] * n->W[0] * cfg->out_ch;
  chk(dalloc(n, &n->y, ny));
  chk(dalloc(n, &n->gy, ny));
  chk(dalloc(n, &n->loss, 1));
  chk(dalloc(n, &n->d_err, 1));
  {  // scratch of the gradients' partial sums: the largest need of a layer's
     // weight and bias gradients and of the head's backward (used one after
     // another on the network's stream)
    size_t need = lbk::nn::head_bwd_scratch(n->C[0], cfg->out_ch,
                                            (long long)cfg->batch * n->H[0] * n->W[0]);
    auto take = [&](const ConvLayer& cl, int l) {
      need = std::max(need, lbk::nn::wgrad_scratch(cl.cout, cl.cin, cfg->batch, n->H[l], n->W[l],
                                                   kWgradChunk));
    };
    for (int l = 0; l < L; ++l) {
      take(n->enc_a[l], l);
      take(n->enc_b[l], l);
    }
    for (int l = 0; l < L - 1; ++l) {
      take(n->up[l], l);
      take(n->dec_a[l], l);
      take(n->dec_b[l], l);
    }
    if (need) chk(dalloc(n, &n->wpart, need));
    n->wpart_cap = need;
  }
  chk(build_seg_tables(n));
  if (e != cudaSuccess) {
    fprintf(stderr, "lbpf_unet_create: %s\n", cudaGetErrorString(e));
    lbpf_unet_destroy(n);
    return LBPF_ENOMEM;
  }
  *out = n;
  return LBPF_OK;
}

lbpf_status lbpf_unet_forward(lbpf_unet_t* n, const float* x, float* y) {
  if (!n || !x || !y) return LBPF_EINVAL;
  int rc;
  if ((rc = pack_input(n, x))) return rc;
  if ((rc = forward(n))) return rc;
  const size_t ny = size_t(n->cfg.batch) * n->H[0] * n->W[0] * n->cfg.out_ch;
  UCK(n, cudaMemcpyAsync(y, n->y, ny * 4, cudaMemcpyDeviceToDevice, n->stream));
  return LBPF_OK;
}

lbpf_status lbpf_unet_grad(lbpf_unet_t* n, const float* x, const float* t, float* loss_host) {
  if (!n || !x || !t) return LBPF_EINVAL;
  int rc;
  for (const ParamView& v : params(n)) UCK(n, cudaMemsetAsync(v.g, 0, v.n * 4, n->stream));
  if ((rc = pack_input(n, x)) || (rc = forward(n)) || (rc = backward(n, t))) return rc;
  if (loss_host) UCK(n, cudaMemcpyAsync(loss_host, n->loss, 4, cudaMemcpyDeviceToHost, n->stream));
  return check_err(n);
}

lbpf_status lbpf_unet_set_tensor_path(lbpf_unet_t* n, int use_tcgen05) {
  if (!n) return LBPF_EINVAL;
  n->tensor_path = use_tcgen05 ? 1 : 0;
  return LBPF_OK;
}

lbpf_status lbpf_unet_status(lbpf_unet_t* n) { return n ? check_err(n) : LBPF_EINVAL; }

lbpf_status lbpf_unet_train_step(lbpf_unet_t* n, const float* x, const float* t, float lr,
                         float* loss_dev) {
  if (!n || !x || !t) return LBPF_EINVAL;
  int rc;
  if ((rc = pack_input(n, x)) || (rc = forward(n)) || (rc = backward(n, t)) ||
      (rc = adam_all(n, lr)))
    return rc;
  if (loss_dev)
    UCK(n, cudaMemcpyAsync(loss_dev, n->loss, 4, cudaMemcpyDeviceToDevice, n->stream));
  return LBPF_OK;
}

lbpf_status lbpf_surrogate_train(lbpf_unet_t* n, const float* X, const float* T, int64_t n_pairs,
                         int steps, const int32_t* idx, const int32_t* flip, const float* lr,
                         int log_every, float* loss_log) {
  if (!n || !X || !T || n_pairs < 1 || steps < 0 || (steps > 0 && (!idx || !lr)) ||
      log_every < 1)
    return LBPF_EINVAL;
  const lbpf_unet_cfg& c = n->cfg;
  if (c.in_ch != 4 || c.out_ch != 4)
    return ufail(n, LBPF_EINVAL, "lbpf_surrogate_train: the network must map 4 fields to 4");
  const int B = c.batch, H = n->H[0], W = n->W[0];
  for (long long k = 0; k < (long long)steps * B; ++k)
    if (idx[k] < 0 || idx[k] >= n_pairs)
      return ufail(n, LBPF_EINVAL, "lbpf_surrogate_train: pair index %d outside [0, %lld)",
                   int(idx[k]), (long long)n_pairs);
  for (int k = 0; flip && k < steps; ++k)
    if (flip[k] < 0 || flip[k] > 2)
      return ufail(n, LBPF_EINVAL, "lbpf_surrogate_train: flip %d of step %d not 0, 1 or 2",
                   int(flip[k]), k);
  for (int k = 0; k < steps; ++k)
    if (!(lr[k] >= 0.f && std::isfinite(lr[k])))
      return ufail(n, LBPF_EINVAL, "lbpf_surrogate_train: learning rate of step %d", k);
  if (steps == 0) return LBPF_OK;
  const int nlog = steps / log_every + (steps % log_every ? 1 : 0);
  const long long nb = (long long)B * H * W * 4;
  if (!n->tx) {  // minibatch buffers, kept with the network
    UCK(n, dalloc(n, &n->tx, size_t(nb)));
    UCK(n, dalloc(n, &n->tt, size_t(nb)));
  }
  int* d_idx = nullptr;
  float* d_log = nullptr;
  auto release = [&]() {
    if (d_idx) cudaFree(d_idx);
    if (d_log) cudaFree(d_log);
  };
  cudaError_t e = cudaMalloc(&d_idx, sizeof(int) * size_t(steps) * B);
  if (e == cudaSuccess) e = cudaMalloc(&d_log, sizeof(float) * size_t(nlog));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_idx, idx, sizeof(int) * size_t(steps) * B, cudaMemcpyHostToDevice,
                        n->stream);
  if (e != cudaSuccess) {
    release();
    return ufail(n, LBPF_ECUDA, "lbpf_surrogate_train: %s", cudaGetErrorString(e));
  }
  int rc = LBPF_OK, k = 0;
  for (int st = 0; st < steps && rc == LBPF_OK; ++st) {
    gather_pairs_kernel<<<grid_of(nb), 256, 0, n->stream>>>(X, T, d_idx + size_t(st) * B,
                                                           flip ? flip[st] : 0, H, W, nb, n->tx,
                                                           n->tt);
    if ((e = cudaGetLastError()) != cudaSuccess) {
      rc = ufail(n, LBPF_ECUDA, "gather_pairs_kernel: %s", cudaGetErrorString(e));
      break;
    }
    rc = lbpf_unet_train_step(n, n->tx, n->tt, lr[st], nullptr);
    if (rc == LBPF_OK && ((st + 1) % log_every == 0 || st == steps - 1) &&
        (e = cudaMemcpyAsync(d_log + k++, n->loss, 4, cudaMemcpyDeviceToDevice, n->stream)) !=
            cudaSuccess)
      rc = ufail(n, LBPF_ECUDA, "loss log: %s", cudaGetErrorString(e));
  }
  if (rc == LBPF_OK && loss_log &&
      (e = cudaMemcpyAsync(loss_log, d_log, sizeof(float) * size_t(nlog), cudaMemcpyDeviceToHost,
                           n->stream)) != cudaSuccess)
    rc = ufail(n, LBPF_ECUDA, "loss log: %s", cudaGetErrorString(e));
  if ((e = cudaStreamSynchronize(n->stream)) != cudaSuccess && rc == LBPF_OK)
    rc = ufail(n, LBPF_ECUDA, "lbpf_surrogate_train: %s", cudaGetErrorString(e));
  release();
  return rc == LBPF_OK ? check_err(n) : rc;
}

size_t lbpf_unet_param_count(const lbpf_unet_t* n) {
  if (!n) return 0;
  size_t s = 0;
  for (const ParamView& v : params(const_cast<lbpf_unet*>(n))) s += v.n;
  return s;
}

lbpf_status lbpf_unet_params(lbpf_unet_t* n, int which, float* host, size_t count, int set) {
  if (!n || !host || count != lbpf_unet_param_count(n) || which < 0 || which > 1 ||
      (set && which != 0))
    return LBPF_EINVAL;
  size_t off = 0;
  for (const ParamView& v : params(n)) {
    float* src = which == 0 ? v.p : v.g;
    if (set)
      UCK(n, cudaMemcpyAsync(src, host + off, v.n * 4, cudaMemcpyHostToDevice, n->stream));
    else
      UCK(n, cudaMemcpyAsync(host + off, src, v.n * 4, cudaMemcpyDeviceToHost, n->stream));
    off += v.n;
  }
  if (set)
    for (ConvLayer* l : all_layers(n)) {
      long long blocks = ((long long)l->nw + 255) / 256;
      if (blocks > 4096) blocks = 4096;
      to_bf16_kernel<<<int(blocks), 256, 0, n->stream>>>(l->w, l->wb, (long long)l->nw);
      UCK(n, cudaGetLastError());
    }
  UCK(n, cudaStreamSynchronize(n->stream));
  return LBPF_OK;
}

lbpf_status lbpf_surrogate_target(const lbpf_surrogate_cfg* cfg, const float* x0, const float* x1,
                          int64_t npix, float* t, void* stream) {
  if (check_cfg(cfg) || !x0 || !x1 || !t || npix < 0) return LBPF_EINVAL;
  lbk::Vec4 g;
  for (int k = 0; k < 4; ++k) g.v[k] = cfg->res_scale[k] != 0.f ? cfg->scale[k] / cfg->res_scale[k] : 0.f;
  if (npix == 0) return LBPF_OK;
  target_kernel<<<grid_of(npix * 4), 256, 0, static_cast<cudaStream_t>(stream)>>>(x0, x1, g,
                                                                                   npix * 4, t);
  return cudaGetLastError() == cudaSuccess ? LBPF_OK : LBPF_ECUDA;
}

lbpf_status lbpf_surrogate_sample(lbpf_t* h, const lbpf_surrogate_cfg* cfg, float* x) {
  if (!h || !x || check_cfg(cfg)) return LBPF_EINVAL;
  if (h->status != LBPF_OK) return h->status;
  if (!h->initialized) return sfail(h, LBPF_ESTATE, "sample before init");
  if (h->m.dim != 2) return sfail(h, LBPF_EINVAL, "the block propagator is 2D only");
  SCK(h, lbk::launch_surrogate_gather(h->m, h->pops[h->cur], h->cur, vec4(cfg->shift), vec4(cfg->scale), x,
                                      nullptr, h->stream));
  return LBPF_OK;
}

}  // extern "C"

namespace {

// The prediction phase of a block, queued on s: read-out of the state and its
// interface positions, the network, the predicted planes, their FP64 sums and
// interface positions, and the copy of those results to pinned host memory.
int queue_prediction(lbpf* h, lbpf_unet* net, const lbpf_surrogate_cfg* cfg, cudaStream_t s) {
  const long long n = (long long)h->m.nx * h->m.ny;
  const int nb = cfg->steps_per_block;
  SCK(h, lbk::launch_surrogate_gather(h->m, h->pops[h->cur], h->cur, vec4(cfg->shift), vec4(cfg->scale),
                                      net->px, net->pF, s));
  plane_crossing_kernel<<<1, 128, 0, s>>>(net->pF, h->m.nx, h->m.ny, h->m.bc[0], h->m.bc[1], h->icx,
                                         h->icy, net->pcross + 4);
  SCK(h, cudaGetLastError());
  int rc;
  if ((rc = lbpf_unet_forward(net, net->px, net->py))) return sfail(h, rc, "network: %s", net->msg);
  apply_kernel<<<grid_of(n), 256, 0, s>>>(net->pF, net->py, vec4(cfg->res_scale), 1.0f / nb, n,
                                          net->pF1);
  SCK(h, cudaGetLastError());
  // the prediction's FP64 sums, into this network's own scratch: two
  // propagators on unordered streams do not share it
  SCK(h, lbk::launch_field_sums(net->pF1, net->pF1 + 4 * n, net->pF1 + n, net->pF + 4 * n, n, 0,
                                net->ppart, lbk::field_sums_blocks(n), net->psum, s));
  plane_crossing_kernel<<<1, 128, 0, s>>>(net->pF1, h->m.nx, h->m.ny, h->m.bc[0], h->m.bc[1], h->icx,
                                         h->icy, net->pcross);
  SCK(h, cudaGetLastError());
  SCK(h, cudaMemcpyAsync(net->hres, net->psum, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  SCK(h, cudaMemcpyAsync(net->hres + 3, net->pcross, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  SCK(h, cudaMemcpyAsync(net->hres + 11, net->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  return LBPF_OK;
}

// the graph of the prediction phase for the current buffer parity, captured
// on first use and again whenever the state buffers, stream or settings change
int prediction_graph(lbpf* h, lbpf_unet* net, const lbpf_surrogate_cfg* cfg,
                     cudaGraphExec_t* out) {
  const int c = h->cur;
  if (net->pgraph[c] && net->pkey_pops[c] == h->pops[c] && net->pkey_stream[c] == h->stream &&
      std::memcmp(&net->pkey_cfg[c], cfg, sizeof(*cfg)) == 0) {
    *out = net->pgraph[c];
    return LBPF_OK;
  }
  if (net->pgraph[c]) {
    cudaGraphExecDestroy(net->pgraph[c]);
    net->pgraph[c] = nullptr;
  }
  // one uncaptured pass first: the first calls of some kernels set attributes
  // and look up device symbols, which must not happen inside a capture
  int rc = queue_prediction(h, net, cfg, h->stream);
  if (rc) return rc;
  SCK(h, cudaStreamSynchronize(h->stream));
  cudaStream_t cs = nullptr;
  SCK(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const cudaStream_t saved = net->stream;
  net->stream = cs;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = queue_prediction(h, net, cfg, cs);
    e = cudaStreamEndCapture(cs, &g);
  }
  net->stream = saved;
  cudaStreamDestroy(cs);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return sfail(h, LBPF_ECUDA, "prediction capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&net->pgraph[c], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return sfail(h, LBPF_ECUDA, "prediction graph: %s", cudaGetErrorString(e));
  net->pkey_pops[c] = h->pops[c];
  net->pkey_stream[c] = h->stream;
  net->pkey_cfg[c] = *cfg;
  *out = net->pgraph[c];
  return LBPF_OK;
}

}  // namespace

extern "C" {

lbpf_status lbpf_surrogate_advance(lbpf_t* h, lbpf_unet_t* net, const lbpf_surrogate_cfg* cfg,
                           int blocks, lbpf_surrogate_report* rep) {
  if (!h || !net || check_cfg(cfg) || blocks < 0) return LBPF_EINVAL;
  if (h->status != LBPF_OK) return h->status;
  if (!h->initialized) return sfail(h, LBPF_ESTATE, "advance before init");
  if (h->m.dim != 2) return sfail(h, LBPF_EINVAL, "the block propagator is 2D only");
  if (h->m.solid)
    return sfail(h, LBPF_EINVAL, "the block propagator was not trained with solid nodes");
  const lbpf_unet_cfg& nc = net->cfg;
  if (nc.batch != 1 || nc.in_ch != 4 || nc.out_ch != 4 || nc.height != h->m.ny ||
      nc.width != h->m.nx)
    return sfail(h, LBPF_EINVAL, "network must be batch 1, 4 -> 4 channels, %d x %d", h->m.ny,
                 h->m.nx);
  const long long n = (long long)h->m.nx * h->m.ny;
  if (!net->px) {
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) {
      if (e == cudaSuccess) e = r;
    };
    chk(dalloc(net, &net->px, size_t(4 * n)));
    chk(dalloc(net, &net->py, size_t(4 * n)));
    chk(dalloc(net, &net->pF, size_t(5 * n)));
    chk(dalloc(net, &net->pF1, size_t(5 * n)));
    chk(dalloc(net, &net->psum, 4));
    chk(dalloc(net, &net->ppart, size_t(3 * lbk::field_sums_blocks(n))));
    chk(dalloc(net, &net->pcross, 8));
    chk(cudaMallocHost(&net->hres, 16 * sizeof(double)));
    if (e != cudaSuccess)
      return sfail(h, LBPF_ENOMEM, "propagator scratch: %s", cudaGetErrorString(e));
  }
  lbpf_surrogate_report r{};
  r.max_iface_err = -1.0;
  r.max_iface_est = -1.0;
  const cudaStream_t s = h->stream;
  const cudaStream_t saved = net->stream;
  net->stream = s;  // the network's kernels run in order with the simulation's
  struct Restore {
    lbpf_unet* n;
    cudaStream_t st;
    ~Restore() { n->stream = st; }
  } restore{net, saved};
  double I0 = 0.0;
  SCK(h, cudaMemcpyAsync(&I0, h->d_diag + 16, sizeof(double), cudaMemcpyDeviceToHost, s));
  SCK(h, cudaStreamSynchronize(s));
  const int nb = cfg->steps_per_block;
  const double tol = cfg->iface_tol;
  // Controller state.  An LB block's outcome (its interface displacement and,
  // if it was judging, the error of the prediction made from the same start)
  // is read at the start of the next block, from that block's own read-out.
  // acc: per ray, the signed sum over every committed block of the predicted
  // displacement minus the displacement the LB showed in its last block: an
  // estimate of how far the committed trajectory has drifted from the LB's
  // (bounded by iface_budget when that is set).
  bool trusted = false, have_ref = false;
  bool lb_pending = false, judge_pending = false, pending_ok = false;
  double dref[4] = {0, 0, 0, 0}, lb_start[4] = {0, 0, 0, 0}, pred_pending[4] = {0, 0, 0, 0};
  double acc[4] = {0, 0, 0, 0};
  double dref_max = 0.0;  // the most recent LB block's largest displacement over the rays
  const double rel = cfg->iface_rel_tol;
  int rc;
  for (int b = 0; b <= blocks; ++b) {
    const bool last = b == blocks;  // only resolves the outcome of the final block
    cudaGraphExec_t g = nullptr;
    if ((rc = prediction_graph(h, net, cfg, &g))) return rc;
    SCK(h, cudaGraphLaunch(g, s));
    SCK(h, cudaStreamSynchronize(s));
    const double* res = net->hres;
    unsigned nerr = 0;
    std::memcpy(&nerr, res + 11, sizeof(nerr));
    if (nerr) return sfail(h, LBPF_ETIMEDOUT, "a tensor-core convolution gave up waiting");
    const double* posP = res + 3;
    const double* pos0 = res + 7;
    if (lb_pending) {
      dref_max = 0.0;
      for (int k = 0; k < 4; ++k) {
        dref[k] = (pos0[k] >= 0 && lb_start[k] >= 0) ? pos0[k] - lb_start[k] : -1e300;
        if (dref[k] > -1e300) dref_max = std::fmax(dref_max, std::fabs(dref[k]));
      }
      have_ref = true;
      if (judge_pending) {
        const double err = ray_diff(pred_pending, pos0);
        r.max_iface_err = std::fmax(r.max_iface_err, err);
        trusted = pending_ok && err >= 0.0 && err <= tol && (rel <= 0.0 || err <= rel * dref_max);
      }
      lb_pending = false;
    }
    if (last) break;
    const double drift = std::fabs(res[0] - I0) / std::fmax(std::fabs(I0), 1e-300);
    r.max_drift = std::fmax(r.max_drift, std::isfinite(drift) ? drift : 1e300);
    double cand[4] = {acc[0], acc[1], acc[2], acc[3]};
    double est = -1.0, est_acc = 0.0;
    if (have_ref)
      for (int k = 0; k < 4; ++k)
        if (posP[k] >= 0 && pos0[k] >= 0 && dref[k] > -1e300) {
          const double e = (posP[k] - pos0[k]) - dref[k];
          est = std::fmax(est, std::fabs(e));
          cand[k] = acc[k] + e;
          est_acc = std::fmax(est_acc, std::fabs(cand[k]));
        }
    const bool drift_ok = drift <= cfg->drift_tol;
    const bool judge = !trusted || !have_ref || (cfg->judge_every > 0 && b % cfg->judge_every == 0);
    const bool fails = !drift_ok || !(est >= 0.0 && est <= tol) ||
                       (cfg->iface_budget > 0.0 && !(est_acc <= cfg->iface_budget)) ||
                       (rel > 0.0 && !(est <= rel * dref_max));
    if (judge || fails) {
      if ((rc = lbpf_step(h, nb))) return rc;
      lb_pending = true;
      judge_pending = judge;
      pending_ok = drift_ok;
      for (int k = 0; k < 4; ++k) {
        lb_start[k] = pos0[k];
        pred_pending[k] = posP[k];
      }
      if (judge) {
        ++r.judged_blocks;
      } else {
        trusted = false;
        ++r.fallback_blocks;
      }
    } else {
      // conservative correction: the accepted prediction's solute deficit is
      // spread over the liquid in proportion to (1 - phi)/2, so that a
      // committed state keeps sum(U + phi(t-1)) as the LB does
      const double liquid = double(n) - res[2];
      const float k = liquid > 0.5 ? float((I0 - res[0]) / liquid) : 0.f;
      correct_kernel<<<grid_of(n), 256, 0, s>>>(net->pF1, n, k);
      SCK(h, cudaGetLastError());
      SCK(h, lbk::launch_surrogate_commit(h->m, net->pF1, net->pF + 4 * n, h->pops[h->cur],
                                          h->phi[h->cur], s));
      h->step += nb;
      for (int k = 0; k < 4; ++k) acc[k] = cand[k];
      r.max_iface_est = std::fmax(r.max_iface_est, est);
      r.max_drift_committed = std::fmax(r.max_drift_committed, drift);
      r.iface_acc = est_acc;
      ++r.surrogate_blocks;
    }
    ++r.blocks;
  }
  if (rep) *rep = r;
  return LBPF_OK;
}

size_t lbpf_unet_device_bytes(const lbpf_unet_t* n) { return n ? n->bytes : 0; }
const char* lbpf_unet_last_error(const lbpf_unet_t* n) { return n ? n->msg : "null handle"; }

void lbpf_unet_destroy(lbpf_unet_t* n) {
  if (!n) return;
  cudaStreamSynchronize(n->stream);
  for (auto& g : n->pgraph)
    if (g) cudaGraphExecDestroy(g);
  if (n->hres) cudaFreeHost(n->hres);
  for (void* p : n->allocs) cudaFree(p);
  delete n;
}

}  // extern "C"
