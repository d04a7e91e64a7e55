// Internal declarations shared by the translation units of liblbpf.so.
// Nothing here is part of the C ABI (include/lbpf.h is).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "batch_schedule.h"

namespace lbk {

enum { BC_PERIODIC = 0, BC_INOUT = 1, BC_WALL = 2 };
enum { ST_FP32 = 0, ST_FP64 = 1, ST_FP16 = 2, ST_BF16 = 3 };

// Model constants in one arithmetic type.  The kernels read the copy in their
// own type: converting a double constant inside the per-node code would run
// on the FP64 pipe, which on GB300 is narrow enough to bound the whole step.
template <typename R>
struct Coef {
  R omega_f, guo, tauU_slope, inv_tau0, tpc, lambda, eps, ck0, sk0, aniso_fac, kdrag;
  R body[3];
  R u_in, U_in, ref_f, ref_g, ref_h;
  R chm_wb, chm_wh;  // central Hermite MRT: trace and higher-order rates
};

// Derived model constants (FP64 on the host; the kernels use cf / cd).  Device layout: every population is its own array of
// `plane` elements, node (x, y, z) at (z * ny + y) * px + x, px a multiple
// of 32 elements so that every row starts 128-byte aligned.  Population
// arrays of one buffer are consecutive: f (qf of them, 0 without flow),
// then g (qs), then h (qs).
struct Model {
  int dim, nx, ny, nz;
  int px;
  long long plane;
  int bc[3];
  int flow, fold, storage, qf, qs;
  double omega_f;      // 1 / tau_f                                   (Eq. 8)
  double guo;          // 1 - 1/(2 tau_f)                              (Eq. 5)
  double tauU_slope;   // tau_U(liquid) - 1/2                          (Eq. 18)
  double inv_tau0;     // 1 / tau0                                     (Eq. 19)
  double tpc;          // W0^2 / (cs^2 tau0), the a_s^2 slope of tau_phi (Eq. 23)
                       // and the c.N coefficient of h^eq (Eq. 21)
  double lambda;       //                                              (Eq. 20)
  double eps;          //                                              (Eq. 3)
  double ck0, sk0;     // cos(k theta0), sin(k theta0)
  double aniso_fac;    // 1 (variational N) or 2 (literal factor)
  double kdrag;        // h tau_f / (4 W0^2)                           (Eq. 6)
  double w0;           // interface width W0
  double body[3];
  double u_in, U_in;   // inflow ghost state
  double ref_f, ref_g, ref_h;  // reference moments of the stored deviations (1, U_ref, -1)
  Coef<float> cf;   // the constants above in FP32 ...
  Coef<double> cd;  // ... and in FP64 (filled by finalize())
  // 16-bit storage (2D and 3D): g is stored relative to a per-node U instead
  // of the global U_ref.  uring: two FP16 planes of `plane` values; for the
  // populations of buffer c, plane c holds each node's reference, while the
  // step that reads them writes the node's new U into plane c and encodes the
  // populations it pushes against the destination's value in plane c ^ 1.
  // The reference only has to be the same number at encoding and decoding,
  // so FP16 loses nothing.
  int chm;              // flow collision: 0 BGK, 1 central Hermite MRT
  double chm_wb, chm_wh;
  int rel_g;
  __half* uring;
  // Solid nodes (walls, obstacles): one byte per node at (z * ny + y) * px +
  // x, 1 = solid; null when there are none.  solid_tiles: in 2D one byte per
  // 32 x 4 tile of the step (row-major over the tiles), in 3D one per column
  // chunk of the z-marching step; 1 = the tile or chunk or its one-node halo
  // holds a solid node
  const unsigned char* solid;
  const unsigned char* solid_tiles;
};

// The stored-g reference of the populations in buffer c (null when g is
// stored relative to the global U_ref).
inline const __half* uref_plane(const Model& m, int c) {
  return m.rel_g ? m.uring + size_t(c) * size_t(m.plane) : nullptr;
}

// Fill m.cf and m.cd from the FP64 fields; call after every change of those.
inline void finalize(Model& m) {
  auto fill = [&](auto& c) {
    using R = std::remove_reference_t<decltype(c.omega_f)>;
    c.omega_f = R(m.omega_f);
    c.guo = R(m.guo);
    c.tauU_slope = R(m.tauU_slope);
    c.inv_tau0 = R(m.inv_tau0);
    c.tpc = R(m.tpc);
    c.lambda = R(m.lambda);
    c.eps = R(m.eps);
    c.ck0 = R(m.ck0);
    c.sk0 = R(m.sk0);
    c.aniso_fac = R(m.aniso_fac);
    c.kdrag = R(m.kdrag);
    for (int d = 0; d < 3; ++d) c.body[d] = R(m.body[d]);
    c.u_in = R(m.u_in);
    c.U_in = R(m.U_in);
    c.ref_f = R(m.ref_f);
    c.ref_g = R(m.ref_g);
    c.ref_h = R(m.ref_h);
    c.chm_wb = R(m.chm_wb);
    c.chm_wh = R(m.chm_wh);
  };
  fill(m.cf);
  fill(m.cd);
}

template <typename R>
__host__ __device__ __forceinline__ const Coef<R>& coef(const Model& m);
template <>
__host__ __device__ __forceinline__ const Coef<float>& coef<float>(const Model& m) {
  return m.cf;
}
template <>
__host__ __device__ __forceinline__ const Coef<double>& coef<double>(const Model& m) {
  return m.cd;
}

// Base pointer of every population array of one buffer (f, then g, then h).
// Passed by value as a kernel parameter, so that each access is one
// constant-bank base plus a 32-bit node offset.
struct PopPtrs {
  void* p[27];
};
// TMA descriptors of the 2D or 3D step for both population buffers (index = the
// parity of the source buffer) and the launch shape of the persistent kernel.
struct StepMaps {
  CUtensorMap fg[2], h[2], ring[2];
  CUtensorMap uown, uhal;  // 2D 16-bit: the U planes (tile box, halo box; plane = coordinate)
  int ctas = 0, smem = 0, ready = 0;
  int ctas_v[4] = {0, 0, 0, 0};  // 2D: CTAs of the variant MASK + 2 CHM
};

// Launchers (each returns the launch error).
cudaError_t prepare_step2d(const Model& m, void* const pops[2], void* const rings[2],
                           StepMaps* out);
cudaError_t launch_step2d(const Model& m, const StepMaps& maps, int c, const void* src, void* dst,
                          const void* ring_prev, void* ring_cur, unsigned* err, cudaStream_t s);
inline PopPtrs pop_ptrs(const Model& m, void* buf, size_t elem_bytes) {
  PopPtrs r{};
  const int q = m.qf + 2 * m.qs;
  for (int a = 0; a < q && a < 27; ++a)
    r.p[a] = static_cast<char*>(buf) + size_t(a) * size_t(m.plane) * elem_bytes;
  return r;
}
cudaError_t prepare_step3d(const Model& m, void* const pops[2], void* const rings[2],
                           StepMaps* out);
cudaError_t launch_step3d(const Model& m, const StepMaps& maps, int c, const void* src, void* dst,
                          const void* ring_prev, void* ring_cur, unsigned* err, cudaStream_t s);

// ---- batched 2D step ---------------------------------------------------------------
// One instance of a batch for one buffer parity: its TMA descriptors (64-byte
// aligned, read by the TMA from global memory), model and buffers.
struct alignas(128) BatchDesc {
  CUtensorMap fg, h, ring, uown, uhal;
  Model m;
  const void* src;
  void* dst;
  float* ring_cur;
  unsigned* err;
  int ntx, c;  // tiles per row of the instance; buffer parity
};
struct BatchMember {  // what the batch needs of one instance
  Model m;
  void* pops[2];
  void* rings[2];
  unsigned* err;
};
struct BatchPlan {  // device tables of one compiled variant
  BatchDesc* desc[2] = {nullptr, nullptr};
  BatchSeg* segs = nullptr;   // the runs of every CTA, CTA after CTA
  int* cta_seg = nullptr;     // CTA b works through segs[cta_seg[b] .. cta_seg[b + 1])
  unsigned char* solid_tiles = nullptr;  // per-tile solid flags of this variant's tiles
  int total_tiles = 0, variant = 0, storage = 0, flow = 0, ctas = 0, smem = 0;
  int grid = 0;   // CTAs of one launch (those with work, all resident at once)
  int order = 0;  // tile order of the schedule (batch_schedule)
  int mask = 0, chm = 0;  // some instance has solid nodes; the flow collides by CHM
  size_t bytes = 0;
};
int batch_variant_count();
int batch_variant_rows(int v);
int batch_variant_stages(int v);
// the tile orders a plan can take (batch_schedule): 0 large instances
// interleaved, 1 instance after instance
constexpr int kBatchOrders = 2;
cudaError_t batch_plan_build(const BatchMember* members, int count, int storage, int flow, int v,
                             int order, BatchPlan* plan);
cudaError_t batch_plan_launch(const BatchPlan& plan, int c, cudaStream_t s);
// the kernel variants of one storage type (setup: occupancy and shared memory
// into *ctas, *smem; else one launch of the step: grid CTAs working through
// their runs of tiles)
#define LBPF_BATCH_DISPATCH(NAME)                                                            \
  cudaError_t NAME(int flow, int v, bool mask, bool chm, bool setup, int* ctas, int* smem,   \
                   const BatchDesc* d, const BatchSeg* segs, const int* cta_seg, int grid,   \
                   cudaStream_t s);
LBPF_BATCH_DISPATCH(batch_dispatch_fp32)
LBPF_BATCH_DISPATCH(batch_dispatch_fp16)
LBPF_BATCH_DISPATCH(batch_dispatch_bf16)
#undef LBPF_BATCH_DISPATCH
void batch_plan_free(BatchPlan* plan);

// Seeded initial state (FP64 arithmetic, stored in the population type).
struct SeedArgs {
  double cx, cy, cz, radius, u0, noise_amp;
  unsigned long long seed;
};
cudaError_t launch_init_seed(const Model& m, const SeedArgs& a, void* pops, void* phi_prev,
                             cudaStream_t s);
// Convex polygon seed (2D): facets of outward unit normals (nx, ny) at
// distances d from (cx, cy).
constexpr int kMaxFacets = 12;
struct PolygonArgs {
  double cx, cy;
  int k;
  double nx[kMaxFacets], ny[kMaxFacets], d[kMaxFacets];
  double u0, noise_amp;
  unsigned long long seed;
};
cudaError_t launch_init_polygon(const Model& m, const PolygonArgs& a, void* pops, void* phi_prev,
                                cudaStream_t s);
// Copy the state of the solid nodes from buffer c to buffer c ^ 1 (both
// population buffers, phi rings and, for 16-bit 2D storage, g-reference
// planes hold the same frozen state).
cudaError_t launch_solid_sync(const Model& m, void* const pops[2], void* const rings[2], int c,
                              cudaStream_t s);
// The per-tile flags of m.solid for the 2D step's tiles, into `flags`
// (solid_tile_count(m) bytes).
size_t solid_tile_count(const Model& m);
cudaError_t launch_solid_tiles(const Model& m, unsigned char* flags, cudaStream_t s);
// 3D: one flag per column chunk of the z-marching step
size_t solid_chunk_count(const Model& m);
cudaError_t launch_solid_chunks(const Model& m, unsigned char* flags, cudaStream_t s);
// Support values of the phi = 0 contour of a 2D state (phi from the h
// populations) along up to kMaxFacets + 4 unit directions, into out[0 ..
// kMaxDirs] on the device: out[j] the order-preserving integer key of max over
// the contour points p of p . dir_j (facet_key_value turns it back into the
// double; key 0: no point), out[kMaxDirs] the number of contour points.
constexpr int kMaxDirs = kMaxFacets + 4;
struct FacetDirs {
  int n;
  double dx[kMaxDirs], dy[kMaxDirs];
};
cudaError_t launch_facet_support(const Model& m, const void* pops, const FacetDirs& dirs,
                                 unsigned long long* out, cudaStream_t s);
double facet_key_value(unsigned long long key);
// Equilibrium state from device FP64 fields (rho/ux/uy/uz may be null).
cudaError_t launch_init_fields(const Model& m, const double* phi, const double* U,
                               const double* rho, const double* ux, const double* uy,
                               const double* uz, void* pops, void* phi_prev, cudaStream_t s);
// Moments of the state into a packed device buffer: the fields selected by
// `mask` (LBPF_FIELD_* bits 0..6) one after another, N values each, as
// double (fp64) or float.
cudaError_t launch_fields(const Model& m, const void* pops, const void* phi_prev, int c,
                          unsigned mask, int fp64, void* out, cudaStream_t s);

// Learned block propagator (2D only).  gather: network input x[i][c] =
// (f_c - shift_c) / scale_c of f = (phi, U, ux, uy), i = y nx + x, and the
// unnormalised planes F[c][i] of (phi, U, ux, uy, rho).  commit: the state
// becomes the equilibrium of the planes F1 = (phi, U, ux, uy, phi(t-1)) with
// density rho.
struct Vec4 {
  float v[4];
};
cudaError_t launch_surrogate_gather(const Model& m, const void* pops, int c, const Vec4& shift,
                                    const Vec4& scale, float* x, float* F, cudaStream_t s);
cudaError_t launch_surrogate_commit(const Model& m, const float* F1, const float* rho, void* pops,
                                    void* phi_prev, cudaStream_t s);

// FP64 diagnostics.  partials: scratch of diag_partials_bytes(m) bytes.
// out[0..4] = sum(U + phi_prev), sum(rho), sum((1+phihat)/2), max|u|,
// nonfinite count; out[5..10] = interface crossings from (icx, icy, icz).
size_t diag_partials_bytes(const Model& m);
cudaError_t launch_diag(const Model& m, const void* pops, const void* phi_prev, int c,
                        double* partials, double* out, int icx, int icy, int icz, cudaStream_t s);

// FP64 sums of caller-held fields (n values each, float or double; rho may be
// null for 1): out[0] = sum(U + phi_prev), out[1] = sum(rho), out[2] =
// sum((1 + clamp(phi))/2), by the deterministic two-pass reduction.
// partials: scratch of field_sums_blocks(n) x 3 doubles, owned by the caller
// (the allocation-free entry point passes its file-scope array).
int field_sums_blocks(int64_t n);
cudaError_t launch_field_sums(const void* phi, const void* phi_prev, const void* U,
                              const void* rho, int64_t n, int fp64, double* partials,
                              int blocks, double* out, cudaStream_t s);

}  // namespace lbk
