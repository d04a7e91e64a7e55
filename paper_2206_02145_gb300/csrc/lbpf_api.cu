// Host side of the C ABI declared in include/lbpf.h: parameter validation,
// device memory, the step loop with its CUDA-graph replay, state export and
// restore, field read-out and FP64 diagnostics.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbpf.h"
#include "lbpf_handle.cuh"

using lbk::Model;

struct lbpf_batch {
  std::vector<lbpf*> kids;
  std::vector<int> gens;
  lbk::BatchPlan plans[8];
  int nplans = 0, chosen = -1;
  float tune_ms[8] = {0};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int cur = 0;
  int status = LBPF_OK;
  char msg[256] = {0};
};

namespace {

constexpr int kGraphSteps = 64;  // even, so a replay keeps the buffer parity
constexpr int kTailMin = 4;      // shorter remainders are launched one by one

int fail(lbpf* h, int code, const char* fmt, ...) {
  if (!h) return code;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(h->msg, sizeof(h->msg), fmt, ap);
  va_end(ap);
  if (code == LBPF_ECUDA || code == LBPF_ENONFINITE || code == LBPF_ETIMEDOUT) h->status = code;
  return code;
}

#define CK(h, call)                                                                     \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(h, LBPF_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                            \
  } while (0)

// Rows of `width` bytes between pitched buffers; one contiguous copy when
// both pitches equal the width (grids whose x size fills the padded row), so
// that the transfer runs as a single large DMA rather than row by row.
cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width,
                      size_t rows, cudaMemcpyKind kind, cudaStream_t s) {
  if (dpitch == width && spitch == width)
    return cudaMemcpyAsync(dst, src, width * rows, kind, s);
  return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, kind, s);
}

long long nodes(const lbpf_params& p) {
  return (long long)p.nx * p.ny * (p.dim == 3 ? p.nz : 1);
}

int validate(const lbpf_params* p, char* why, size_t n) {
  auto bad = [&](const char* s) {
    snprintf(why, n, "%s", s);
    return LBPF_EINVAL;
  };
  if (p->dim != 2 && p->dim != 3) return bad("dim must be 2 or 3");
  if (p->nx < 4 || p->ny < 4 || (p->dim == 3 && p->nz < 4)) return bad("every grid dimension must be >= 4");
  // node offsets are 32-bit: at most 2^31 - 1 (padded) nodes per array
  if ((double)((p->nx + 31) / 32 * 32) * p->ny * (p->dim == 3 ? p->nz : 1) > 2147483647.0)
    return bad("grid too large (more than 2^31 nodes per population array)");
  for (int d = 0; d < 3; ++d)
    if (p->bc[d] < 0 || p->bc[d] > 2) return bad("unknown boundary condition");
  if (p->bc[1] == LBPF_BC_INLET_OUTLET || p->bc[2] == LBPF_BC_INLET_OUTLET)
    return bad("INLET_OUTLET is only available on x");
  if (p->storage < 0 || p->storage > 3) return bad("unknown storage");
  if (!(p->tau_phi0 > 0.5) || !(p->tau_u_liquid > 0.5)) return bad("relaxation times must exceed 1/2");
  if (p->flow && !(p->tau_f > 0.5)) return bad("tau_f must exceed 1/2");
  if (!(p->w0 > 0.0)) return bad("W0 must be positive");
  if (!(p->eps_aniso >= 0.0 && p->eps_aniso < 1.0)) return bad("eps must be in [0, 1)");
  if (p->fold < 0 || p->fold > 12) return bad("fold must be 0..12");
  if (p->dim == 3 && p->fold != 0) return bad("3D supports the cubic form only (fold = 0)");
  if (!(std::fabs(p->u_inlet) <= 0.1)) return bad("|u_inlet| must be <= 0.1 (low Mach)");
  if (!std::isfinite(p->lambda) || !std::isfinite(p->theta0) || !std::isfinite(p->h_drag) ||
      !std::isfinite(p->u0_inlet))
    return bad("non-finite parameter");
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(p->body_force[d])) return bad("non-finite body force");
  if (p->collision != LBPF_COLL_BGK && p->collision != LBPF_COLL_CHM)
    return bad("unknown collision");
  if (p->collision == LBPF_COLL_CHM) {
    if (!p->flow) return bad("the central Hermite MRT is a collision of the flow lattice");
    for (double w : {p->chm_omega_bulk, p->chm_omega_high})
      if (!(w == 0.0 || (w > 0.0 && w < 2.0))) return bad("CHM rates must be in (0, 2) or 0");
  }
  return LBPF_OK;
}

Model derive(const lbpf_params& p) {
  Model m{};
  m.dim = p.dim;
  m.nx = p.nx;
  m.ny = p.ny;
  m.nz = p.dim == 3 ? p.nz : 1;
  m.px = (p.nx + 31) / 32 * 32;
  m.plane = (long long)m.px * m.ny * m.nz;
  for (int d = 0; d < 3; ++d) m.bc[d] = p.bc[d];
  if (p.dim == 2) m.bc[2] = LBPF_BC_PERIODIC;
  m.flow = p.flow ? 1 : 0;
  m.fold = p.fold;
  m.storage = p.storage;
  m.qf = p.flow ? (p.dim == 2 ? 9 : 19) : 0;
  m.qs = p.dim == 2 ? 9 : 7;
  const double cs2 = p.dim == 2 ? 1.0 / 3.0 : 0.25;  // lattice of g and h
  const double tau0 = p.w0 * p.w0 / (cs2 * (p.tau_phi0 - 0.5));  // Eq. 23 at a_s = 1
  m.omega_f = p.flow ? 1.0 / p.tau_f : 0.0;
  m.guo = p.flow ? 1.0 - 0.5 / p.tau_f : 0.0;
  m.tauU_slope = p.tau_u_liquid - 0.5;
  m.inv_tau0 = 1.0 / tau0;
  m.tpc = p.w0 * p.w0 / (cs2 * tau0);
  if (p.lambda >= 0.0) {
    m.lambda = p.lambda;
  } else {
    const double D = cs2 * (p.tau_u_liquid - 0.5);
    m.lambda = D * tau0 / (0.6267 * p.w0 * p.w0);  // thin-interface value, a2 = 0.6267
  }
  m.eps = p.eps_aniso;
  m.ck0 = std::cos(p.fold * p.theta0);
  m.sk0 = std::sin(p.fold * p.theta0);
  m.aniso_fac = p.aniso_literal ? 2.0 : 1.0;
  m.kdrag = p.flow ? p.h_drag * p.tau_f / (4.0 * p.w0 * p.w0) : 0.0;
  m.w0 = p.w0;
  for (int d = 0; d < 3; ++d) m.body[d] = p.flow ? p.body_force[d] : 0.0;
  m.u_in = p.flow ? p.u_inlet : 0.0;
  m.U_in = p.u0_inlet;
  m.ref_f = 1.0;
  m.ref_g = 0.0;
  m.ref_h = -1.0;
  // 16-bit storage keeps g relative to a per-node U (two FP16 planes,
  // allocated by lbpf_create)
  m.rel_g = (p.storage == LBPF_FP16_SHIFTED || p.storage == LBPF_BF16_SHIFTED) ? 1 : 0;
  m.uring = nullptr;
  m.solid = nullptr;
  m.solid_tiles = nullptr;
  m.chm = p.collision == LBPF_COLL_CHM ? 1 : 0;
  m.chm_wb = p.chm_omega_bulk > 0.0 ? p.chm_omega_bulk : 1.0;
  m.chm_wh = p.chm_omega_high > 0.0 ? p.chm_omega_high : 1.0;
  lbk::finalize(m);
  return m;
}

bool is16(const Model& m) { return m.storage == lbk::ST_FP16 || m.storage == lbk::ST_BF16; }

int check_handle(lbpf* h) {
  if (!h) return LBPF_EINVAL;
  if (h->status != LBPF_OK) return h->status;
  return LBPF_OK;
}

int check_device_error(lbpf* h) {
  unsigned e = 0;
  CK(h, cudaMemcpyAsync(&e, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  if (e & 2u) return fail(h, LBPF_ETIMEDOUT, "a step kernel gave up waiting for its tile loads");
  if (e & 1u) return fail(h, LBPF_ENONFINITE, "a non-finite phi, U or rho appeared in the step");
  return LBPF_OK;
}

int launch_one(lbpf* h, cudaStream_t s) {
  const int c = h->cur;
  cudaError_t e = h->m.dim == 2
                      ? lbk::launch_step2d(h->m, h->maps, c, h->pops[c], h->pops[c ^ 1],
                                           h->phi[c], h->phi[c ^ 1], h->d_err, s)
                      : lbk::launch_step3d(h->m, h->maps, c, h->pops[c], h->pops[c ^ 1],
                                           h->phi[c], h->phi[c ^ 1], h->d_err, s);
  if (e != cudaSuccess) return fail(h, LBPF_ECUDA, "step launch: %s", cudaGetErrorString(e));
  h->cur ^= 1;
  return LBPF_OK;
}

// Capture n launches starting from buffer parity `parity` into *out.
int capture_steps(lbpf* h, int n, int parity, cudaGraphExec_t* out) {
  if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  const int saved = h->cur;
  h->cur = parity;
  cudaGraph_t g = nullptr;
  CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = LBPF_OK;
  for (int i = 0; i < n && rc == LBPF_OK; ++i) rc = launch_one(h, h->cap_stream);
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  h->cur = saved;
  if (rc != LBPF_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(h, LBPF_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(h, LBPF_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return LBPF_OK;
}

// Capture kGraphSteps launches starting from buffer parity 0.
int build_graph(lbpf* h) {
  if (h->graph) return LBPF_OK;
  int rc = capture_steps(h, kGraphSteps, 0, &h->graph);
  if (rc) return rc;
  h->graph_steps = kGraphSteps;
  return LBPF_OK;
}

// The graph of n (< kGraphSteps) steps from the current parity: found among
// the cached ones or captured (replacing the oldest).
int tail_graph(lbpf* h, int n, cudaGraphExec_t* out) {
  for (int i = 0; i < lbpf::kTailGraphs; ++i)
    if (h->tail_graph[i] && h->tail_n[i] == n && h->tail_parity[i] == h->cur) {
      *out = h->tail_graph[i];
      return LBPF_OK;
    }
  const int i = h->tail_next;
  h->tail_next = (i + 1) % lbpf::kTailGraphs;
  if (h->tail_graph[i]) cudaGraphExecDestroy(h->tail_graph[i]);
  h->tail_graph[i] = nullptr;
  int rc = capture_steps(h, n, h->cur, &h->tail_graph[i]);
  if (rc) return rc;
  h->tail_n[i] = n;
  h->tail_parity[i] = h->cur;
  *out = h->tail_graph[i];
  return LBPF_OK;
}

// The graphs bake the model constants in; drop them when they change.
void drop_graph(lbpf* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  h->graph_steps = 0;
  for (int i = 0; i < lbpf::kTailGraphs; ++i) {
    if (h->tail_graph[i]) cudaGraphExecDestroy(h->tail_graph[i]);
    h->tail_graph[i] = nullptr;
    h->tail_n[i] = 0;
  }
}

int ensure_fields_buffer(lbpf* h, size_t bytes) {
  if (h->fields_cap >= bytes) return LBPF_OK;
  if (h->d_fields) {
    cudaFree(h->d_fields);
    h->dev_bytes -= h->fields_cap;
    h->d_fields = nullptr;
    h->fields_cap = 0;
  }
  cudaError_t e = cudaMalloc(&h->d_fields, bytes);
  if (e != cudaSuccess) return fail(h, LBPF_ENOMEM, "field buffer: %s", cudaGetErrorString(e));
  h->fields_cap = bytes;
  h->dev_bytes += bytes;
  return LBPF_OK;
}

// plane c of the per-node g reference (16-bit 2D storage)
__half* uref_dev(lbpf* h, int c) { return h->m.uring + size_t(c) * size_t(h->m.plane); }

// After the state of buffer cur was replaced: the solid nodes' frozen state
// into the other buffer as well.
int sync_solids(lbpf* h) {
  if (!h->m.solid) return LBPF_OK;
  CK(h, lbk::launch_solid_sync(h->m, h->pops, h->phi, h->cur, h->stream));
  return LBPF_OK;
}

void store_I0(lbpf* h) {
  // solute total at init, kept on the device for the drift of lbpf_diagnostics
  lbk::launch_diag(h->m, h->pops[h->cur], h->phi[h->cur], h->cur, h->d_partials, h->d_diag,
                    h->icx, h->icy, h->icz, h->stream);
  cudaMemcpyAsync(h->d_diag + 16, h->d_diag, sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
}

constexpr char kMagic[8] = {'L', 'B', 'P', 'F', 'S', 'T', '0', '2'};

struct StateHeader {
  char magic[8];
  int64_t step;
  int32_t dim, nx, ny, nz, storage, flow, q, elem;
  double ref_g;  // reference U of the stored g deviations
  // where the diagnostics measure from: the node the interface rays start at
  // (the seed centre) and the solute total Sum(U + phi_lag) at initialisation
  // (the base of solute_drift_rel), so that a restored run reports what the
  // uninterrupted one does
  int32_t icx, icy, icz, pad0;
  double solute0;
  char pad[48];
};
static_assert(sizeof(StateHeader) == 128, "state header must be 128 bytes");

}  // namespace

extern "C" {

lbpf_status lbpf_params_default(lbpf_params* p) {
  if (!p) return LBPF_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->dim = 2;
  p->nx = p->ny = 128;
  p->nz = 1;
  p->fold = 4;
  p->tau_phi0 = 0.8;
  p->tau_u_liquid = 0.8;
  p->tau_f = 0.6;
  p->w0 = 2.0;
  p->lambda = -1.0;
  p->eps_aniso = 0.05;
  p->h_drag = 2.757;
  return LBPF_OK;
}

lbpf_status lbpf_create(const lbpf_params* p, void* stream, lbpf_t** out) {
  if (!p || !out) return LBPF_EINVAL;
  *out = nullptr;
  char why[160];
  if (validate(p, why, sizeof(why)) != LBPF_OK) {
    fprintf(stderr, "lbpf_create: %s\n", why);
    return LBPF_EINVAL;
  }
  lbpf* h = new (std::nothrow) lbpf();
  if (!h) return LBPF_ENOMEM;
  h->p = *p;
  if (h->p.dim == 2) h->p.nz = 1;
  h->m = derive(h->p);
  h->stream = static_cast<cudaStream_t>(stream);
  h->es = h->m.storage == lbk::ST_FP64 ? 8 : (is16(h->m) ? 2 : 4);
  h->rs = h->m.storage == lbk::ST_FP64 ? 8 : 4;
  const size_t q = size_t(h->m.qf + 2 * h->m.qs);
  const size_t pop_bytes = q * size_t(h->m.plane) * h->es;
  const size_t ring_bytes = size_t(h->m.plane) * h->rs;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&h->pops[i], pop_bytes);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&h->phi[i], ring_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_err, 256);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_partials, lbk::diag_partials_bytes(h->m));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_diag, 32 * sizeof(double));
  const size_t uring_bytes = h->m.rel_g ? 2 * size_t(h->m.plane) * sizeof(__half) : 0;
  if (e == cudaSuccess && uring_bytes) e = cudaMalloc(&h->m.uring, uring_bytes);
  if (e != cudaSuccess) {
    fprintf(stderr, "lbpf_create: %s\n", cudaGetErrorString(e));
    lbpf_destroy(h);
    return LBPF_ENOMEM;
  }
  h->dev_bytes = 2 * pop_bytes + 2 * ring_bytes + uring_bytes + 256 +
                 lbk::diag_partials_bytes(h->m) + 32 * sizeof(double);
  e = cudaMemsetAsync(h->d_err, 0, 256, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_diag, 0, 32 * sizeof(double), h->stream);
  if (e != cudaSuccess) {
    fprintf(stderr, "lbpf_create: %s\n", cudaGetErrorString(e));
    lbpf_destroy(h);
    return LBPF_ECUDA;
  }
  {
    e = h->m.dim == 2 ? lbk::prepare_step2d(h->m, h->pops, h->phi, &h->maps)
                      : lbk::prepare_step3d(h->m, h->pops, h->phi, &h->maps);
    if (e != cudaSuccess) {
      fprintf(stderr, "lbpf_create: step setup: %s\n", cudaGetErrorString(e));
      lbpf_destroy(h);
      return LBPF_ECUDA;
    }
  }
  h->icx = h->m.nx / 2;
  h->icy = h->m.ny / 2;
  h->icz = h->m.nz / 2;
  *out = h;
  return LBPF_OK;
}

lbpf_status lbpf_init_seed(lbpf_t* h, const lbpf_seed* s) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!s || !(s->radius >= 0.0) || !std::isfinite(s->u0) || !std::isfinite(s->noise_amp) ||
      !std::isfinite(s->cx) || !std::isfinite(s->cy) || !std::isfinite(s->cz))
    return fail(h, LBPF_EINVAL, "invalid seed");
  h->m.ref_g = s->u0;
  lbk::finalize(h->m);
  drop_graph(h);
  ++h->gen;
  lbk::SeedArgs a{s->cx, s->cy, s->cz, s->radius, s->u0, s->noise_amp, s->seed};
  h->cur = 0;
  h->step = 0;
  CK(h, lbk::launch_init_seed(h->m, a, h->pops[0], h->phi[0], h->stream));
  if ((rc = sync_solids(h))) return rc;
  auto clampi = [](double v, int n) {
    long long i = std::llround(v);
    return int(i < 0 ? 0 : (i >= n ? n - 1 : i));
  };
  h->icx = clampi(s->cx, h->m.nx);
  h->icy = clampi(s->cy, h->m.ny);
  h->icz = h->m.dim == 3 ? clampi(s->cz, h->m.nz) : 0;
  h->initialized = true;
  store_I0(h);
  CK(h, cudaGetLastError());
  return LBPF_OK;
}

lbpf_status lbpf_init_polygon(lbpf_t* h, const lbpf_polygon_seed* s) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (h->m.dim != 2) return fail(h, LBPF_EINVAL, "polygon seeds are 2D");
  if (!s || s->nfacets < 3 || s->nfacets > LBPF_MAX_FACETS || !std::isfinite(s->cx) ||
      !std::isfinite(s->cy) || !std::isfinite(s->u0) || !std::isfinite(s->noise_amp))
    return fail(h, LBPF_EINVAL, "invalid polygon seed");
  lbk::PolygonArgs a{};
  a.cx = s->cx;
  a.cy = s->cy;
  a.k = s->nfacets;
  for (int i = 0; i < s->nfacets; ++i) {
    const double len = std::hypot(s->nx[i], s->ny[i]);
    if (!(std::fabs(len - 1.0) <= 1e-9) || !std::isfinite(s->dist[i]))
      return fail(h, LBPF_EINVAL, "facet %d: normal not of unit length or distance not finite", i);
    a.nx[i] = s->nx[i];
    a.ny[i] = s->ny[i];
    a.d[i] = s->dist[i];
  }
  a.u0 = s->u0;
  a.noise_amp = s->noise_amp;
  a.seed = s->seed;
  h->m.ref_g = s->u0;
  lbk::finalize(h->m);
  drop_graph(h);
  ++h->gen;
  h->cur = 0;
  h->step = 0;
  CK(h, lbk::launch_init_polygon(h->m, a, h->pops[0], h->phi[0], h->stream));
  if ((rc = sync_solids(h))) return rc;
  auto clampi = [](double v, int n) {
    long long i = std::llround(v);
    return int(i < 0 ? 0 : (i >= n ? n - 1 : i));
  };
  h->icx = clampi(s->cx, h->m.nx);
  h->icy = clampi(s->cy, h->m.ny);
  h->icz = 0;
  h->initialized = true;
  store_I0(h);
  CK(h, cudaGetLastError());
  return LBPF_OK;
}

lbpf_status lbpf_init_fields(lbpf_t* h, const double* phi, const double* U, const double* rho,
                     const double* ux, const double* uy, const double* uz) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!phi || !U) return fail(h, LBPF_EINVAL, "phi and U are required");
  const size_t n = size_t(nodes(h->p));
  const double* src[6] = {phi, U, rho, ux, uy, uz};
  double* dev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* block = nullptr;
  CK(h, cudaMalloc(&block, 6 * n * sizeof(double)));
  for (int k = 0; k < 6; ++k) {
    if (!src[k]) continue;
    dev[k] = block + k * n;
    cudaError_t e = cudaMemcpyAsync(dev[k], src[k], n * sizeof(double), cudaMemcpyHostToDevice,
                                    h->stream);
    if (e != cudaSuccess) {
      cudaFree(block);
      return fail(h, LBPF_ECUDA, "init_fields copy: %s", cudaGetErrorString(e));
    }
  }
  // g is stored as the deviation from w_a times the mean initial U
  {
    double mean = 0.0;
    for (size_t i = 0; i < n; ++i) mean += U[i];
    h->m.ref_g = mean / double(n);
  }
  lbk::finalize(h->m);
  drop_graph(h);
  ++h->gen;
  h->cur = 0;
  h->step = 0;
  cudaError_t e = lbk::launch_init_fields(h->m, dev[0], dev[1], dev[2], dev[3], dev[4], dev[5],
                                           h->pops[0], h->phi[0], h->stream);
  if (e == cudaSuccess && h->m.solid) e = lbk::launch_solid_sync(h->m, h->pops, h->phi, 0, h->stream);
  cudaError_t e2 = cudaStreamSynchronize(h->stream);
  cudaFree(block);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return fail(h, LBPF_ECUDA, "init_fields: %s",
                cudaGetErrorString(e != cudaSuccess ? e : e2));
  h->initialized = true;
  store_I0(h);
  CK(h, cudaGetLastError());
  return LBPF_OK;
}

lbpf_status lbpf_step(lbpf_t* h, int n) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (n < 0) return fail(h, LBPF_EINVAL, "n must be >= 0");
  if (!h->initialized) return fail(h, LBPF_ESTATE, "step before init");
  int left = n;
  if (left >= kGraphSteps) {
    if (h->cur == 1) {
      if ((rc = launch_one(h, h->stream))) return rc;
      --left;
    }
    if (left >= kGraphSteps) {
      if ((rc = build_graph(h))) return rc;
      while (left >= h->graph_steps) {
        CK(h, cudaGraphLaunch(h->graph, h->stream));
        left -= h->graph_steps;
      }
    }
  }
  if (left >= kTailMin) {
    // the rest as one graph of its own (cached per count and parity)
    cudaGraphExec_t g = nullptr;
    if ((rc = tail_graph(h, left, &g))) return rc;
    CK(h, cudaGraphLaunch(g, h->stream));
    h->cur ^= left & 1;
    left = 0;
  }
  for (; left > 0; --left)
    if ((rc = launch_one(h, h->stream))) return rc;
  h->step += n;
  return LBPF_OK;
}

size_t lbpf_state_bytes(const lbpf_t* h) {
  if (!h) return 0;
  const size_t n = size_t(nodes(h->p));
  const size_t q = size_t(h->m.qf + 2 * h->m.qs);
  return sizeof(StateHeader) + q * n * h->es + n * h->rs + (h->m.rel_g ? 2 * n * 2 : 0);
}

lbpf_status lbpf_read_fields(lbpf_t* h, unsigned mask, void* host_dst, size_t bytes, int as_fp64) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!host_dst) return fail(h, LBPF_EINVAL, "null destination");
  if (!h->initialized) return fail(h, LBPF_ESTATE, "read before init");
  const size_t n = size_t(nodes(h->p));
  if (mask & LBPF_FIELD_STATE) {
    if (mask != LBPF_FIELD_STATE) return fail(h, LBPF_EINVAL, "STATE must be requested alone");
    if (bytes != lbpf_state_bytes(h)) return fail(h, LBPF_EINVAL, "state buffer size mismatch");
    StateHeader hd{};
    std::memcpy(hd.magic, kMagic, 8);
    hd.step = h->step;
    hd.dim = h->m.dim;
    hd.nx = h->m.nx;
    hd.ny = h->m.ny;
    hd.nz = h->m.nz;
    hd.storage = h->m.storage;
    hd.flow = h->m.flow;
    hd.q = h->m.qf + 2 * h->m.qs;
    hd.elem = int32_t(h->es);
    hd.ref_g = h->m.ref_g;
    hd.icx = h->icx;
    hd.icy = h->icy;
    hd.icz = h->icz;
    CK(h, cudaMemcpyAsync(&hd.solute0, h->d_diag + 16, sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
    char* dst = static_cast<char*>(host_dst);
    const size_t rows = size_t(hd.q) * h->m.ny * h->m.nz;
    CK(h, copy_rows(dst + sizeof(hd), h->m.nx * h->es, h->pops[h->cur], h->m.px * h->es,
                    h->m.nx * h->es, rows, cudaMemcpyDeviceToHost, h->stream));
    CK(h, copy_rows(dst + sizeof(hd) + size_t(hd.q) * n * h->es, h->m.nx * h->rs,
                    h->phi[h->cur], h->m.px * h->rs, h->m.nx * h->rs, size_t(h->m.ny) * h->m.nz,
                    cudaMemcpyDeviceToHost, h->stream));
    if (h->m.rel_g) {  // g references: the current buffer's, then the other one
      char* ud = dst + sizeof(hd) + size_t(hd.q) * n * h->es + n * h->rs;
      for (int k = 0; k < 2; ++k)
        CK(h, copy_rows(ud + k * n * 2, h->m.nx * 2, uref_dev(h, h->cur ^ k), h->m.px * 2,
                        h->m.nx * 2, size_t(h->m.ny) * h->m.nz, cudaMemcpyDeviceToHost,
                        h->stream));
    }
    rc = check_device_error(h);  // synchronises: hd.solute0 has arrived
    std::memcpy(dst, &hd, sizeof(hd));
    return rc;
  }
  const unsigned fm = mask & 0x7Fu;
  if (fm == 0 || mask != fm) return fail(h, LBPF_EINVAL, "unknown field bits");
  const int nf = __builtin_popcount(fm);
  const size_t es = as_fp64 ? 8 : 4;
  if (bytes != size_t(nf) * n * es) return fail(h, LBPF_EINVAL, "field buffer size mismatch");
  if ((rc = ensure_fields_buffer(h, bytes))) return rc;
  CK(h, lbk::launch_fields(h->m, h->pops[h->cur], h->phi[h->cur], h->cur, fm, as_fp64,
                            h->d_fields, h->stream));
  CK(h, cudaMemcpyAsync(host_dst, h->d_fields, bytes, cudaMemcpyDeviceToHost, h->stream));
  return check_device_error(h);
}

lbpf_status lbpf_write_state(lbpf_t* h, const void* host_src, size_t bytes) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!host_src || bytes != lbpf_state_bytes(h))
    return fail(h, LBPF_EINVAL, "state buffer size mismatch");
  StateHeader hd;
  std::memcpy(&hd, host_src, sizeof(hd));
  if (std::memcmp(hd.magic, kMagic, 8) != 0 || hd.dim != h->m.dim || hd.nx != h->m.nx ||
      hd.ny != h->m.ny || hd.nz != h->m.nz || hd.storage != h->m.storage || hd.flow != h->m.flow ||
      hd.q != h->m.qf + 2 * h->m.qs || hd.elem != int32_t(h->es) || hd.step < 0 ||
      hd.icx < 0 || hd.icx >= h->m.nx || hd.icy < 0 || hd.icy >= h->m.ny || hd.icz < 0 ||
      hd.icz >= h->m.nz || !std::isfinite(hd.solute0))
    return fail(h, LBPF_EINVAL, "state does not match this handle");
  const size_t n = size_t(nodes(h->p));
  const char* src = static_cast<const char*>(host_src);
  h->cur = 0;
  const size_t rows = size_t(hd.q) * h->m.ny * h->m.nz;
  CK(h, copy_rows(h->pops[0], h->m.px * h->es, src + sizeof(hd), h->m.nx * h->es,
                  h->m.nx * h->es, rows, cudaMemcpyHostToDevice, h->stream));
  CK(h, copy_rows(h->phi[0], h->m.px * h->rs, src + sizeof(hd) + size_t(hd.q) * n * h->es,
                  h->m.nx * h->rs, h->m.nx * h->rs, size_t(h->m.ny) * h->m.nz,
                  cudaMemcpyHostToDevice, h->stream));
  if (h->m.rel_g) {
    const char* us = src + sizeof(hd) + size_t(hd.q) * n * h->es + n * h->rs;
    for (int k = 0; k < 2; ++k)
      CK(h, copy_rows(uref_dev(h, k), h->m.px * 2, us + k * n * 2, h->m.nx * 2, h->m.nx * 2,
                      size_t(h->m.ny) * h->m.nz, cudaMemcpyHostToDevice, h->stream));
  }
  if ((rc = sync_solids(h))) return rc;
  h->step = hd.step;
  if (h->m.ref_g != hd.ref_g) drop_graph(h);
  h->m.ref_g = hd.ref_g;
  lbk::finalize(h->m);
  ++h->gen;
  h->icx = hd.icx;
  h->icy = hd.icy;
  h->icz = hd.icz;
  CK(h, cudaMemcpyAsync(h->d_diag + 16, &hd.solute0, sizeof(double), cudaMemcpyHostToDevice,
                        h->stream));
  h->initialized = true;
  CK(h, cudaStreamSynchronize(h->stream));
  return LBPF_OK;
}

lbpf_status lbpf_diagnostics(lbpf_t* h, lbpf_diag* out) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!out) return fail(h, LBPF_EINVAL, "null output");
  if (!h->initialized) return fail(h, LBPF_ESTATE, "diagnostics before init");
  CK(h, lbk::launch_diag(h->m, h->pops[h->cur], h->phi[h->cur], h->cur, h->d_partials,
                          h->d_diag, h->icx, h->icy, h->icz, h->stream));
  double v[17];
  CK(h, cudaMemcpyAsync(v, h->d_diag, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
  if ((rc = check_device_error(h))) return rc;
  std::memset(out, 0, sizeof(*out));
  out->step = h->step;
  out->solute_total = v[0];
  out->mass_total = v[1];
  out->solid_volume = v[2];
  out->max_u = v[3];
  out->nonfinite = (int64_t)v[4];
  out->solute_drift_rel = v[16] != 0.0 ? (v[0] - v[16]) / std::fabs(v[16]) : 0.0;
  out->r_eq = h->m.dim == 3 ? std::cbrt(3.0 * v[2] / (4.0 * M_PI)) : std::sqrt(v[2] / M_PI);
  for (int k = 0; k < 6; ++k) out->iface_pos[k] = v[5 + k];
  if (out->nonfinite > 0)
    return fail(h, LBPF_ENONFINITE, "%lld nodes hold non-finite values", (long long)out->nonfinite);
  return LBPF_OK;
}

lbpf_status lbpf_facets_enqueue(lbpf_t* h, int k, const double* nx, const double* ny) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!nx || !ny) return fail(h, LBPF_EINVAL, "null argument");
  if (!h->initialized) return fail(h, LBPF_ESTATE, "facets before init");
  if (h->m.dim != 2) return fail(h, LBPF_EINVAL, "facet measurement is 2D");
  if (k < 4 || k > LBPF_MAX_FACETS || k % 2)
    return fail(h, LBPF_EINVAL, "facet count must be even, 4..%d", LBPF_MAX_FACETS);
  for (int i = 0; i < k; ++i) {
    const int o = (i + k / 2) % k, nb = (i + 1) % k;
    if (!(std::fabs(std::hypot(nx[i], ny[i]) - 1.0) <= 1e-9))
      return fail(h, LBPF_EINVAL, "facet %d: normal not of unit length", i);
    if (!(std::fabs(nx[i] + nx[o]) <= 1e-9 && std::fabs(ny[i] + ny[o]) <= 1e-9))
      return fail(h, LBPF_EINVAL, "facet %d: normal %d is not its opposite", i, o);
    if (!(nx[i] * ny[nb] - ny[i] * nx[nb] > 1e-6))
      return fail(h, LBPF_EINVAL, "facets %d, %d: normals not in counter-clockwise order", i, nb);
  }
  const size_t nres = sizeof(unsigned long long) * (lbk::kMaxDirs + 1);
  if (!h->d_facets) {
    cudaError_t e = cudaMalloc(&h->d_facets, nres);
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_facets, nres);
    if (e != cudaSuccess) return fail(h, LBPF_ENOMEM, "facet results: %s", cudaGetErrorString(e));
    h->dev_bytes += nres;
  }
  // directions: the k normals, then +x, -x, +y, -y for the extents
  lbk::FacetDirs d{};
  d.n = k + 4;
  for (int i = 0; i < k; ++i) {
    d.dx[i] = h->facet_nx[i] = nx[i];
    d.dy[i] = h->facet_ny[i] = ny[i];
  }
  const double ax[4] = {1.0, -1.0, 0.0, 0.0}, ay[4] = {0.0, 0.0, 1.0, -1.0};
  for (int j = 0; j < 4; ++j) {
    d.dx[k + j] = ax[j];
    d.dy[k + j] = ay[j];
  }
  h->facet_k = 0;
  CK(h, lbk::launch_facet_support(h->m, h->pops[h->cur], d, h->d_facets, h->stream));
  CK(h, cudaMemcpyAsync(h->h_facets, h->d_facets, nres, cudaMemcpyDeviceToHost, h->stream));
  h->facet_k = k;
  return LBPF_OK;
}

lbpf_status lbpf_facets_collect(lbpf_t* h, lbpf_facets* out) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!out) return fail(h, LBPF_EINVAL, "null argument");
  if (!h->facet_k) return fail(h, LBPF_ESTATE, "no facet measurement enqueued");
  if ((rc = check_device_error(h))) return rc;
  const int k = h->facet_k;
  const double* nx = h->facet_nx;
  const double* ny = h->facet_ny;
  double v[lbk::kMaxDirs];  // the k supports, then max x, -min x, max y, -min y
  for (int j = 0; j < k + 4; ++j) v[j] = lbk::facet_key_value(h->h_facets[j]);
  h->facet_k = 0;
  const double nan = std::nan("");
  std::memset(out, 0, sizeof(*out));
  out->nfacets = k;
  out->points = (long long)h->h_facets[lbk::kMaxDirs];
  if (out->points == 0) {
    for (int i = 0; i < LBPF_MAX_FACETS; ++i)
      out->support[i] = out->side_cx[i] = out->side_cy[i] = out->L[i] = nan;
    out->cx = out->cy = out->L_avg = out->Q = out->width = out->height = out->aspect = nan;
    return LBPF_OK;
  }
  // side i runs between its meets with the supporting lines of sides i - 1
  // and i + 1; its centre is the midpoint
  double ex[LBPF_MAX_FACETS], ey[LBPF_MAX_FACETS];  // end shared by sides i and i + 1
  for (int i = 0; i < k; ++i) {
    const int j = (i + 1) % k;
    const double det = nx[i] * ny[j] - ny[i] * nx[j];
    ex[i] = (v[i] * ny[j] - ny[i] * v[j]) / det;
    ey[i] = (nx[i] * v[j] - v[i] * nx[j]) / det;
    out->support[i] = v[i];
  }
  for (int i = 0; i < k; ++i) {
    const int p = (i + k - 1) % k;
    out->side_cx[i] = 0.5 * (ex[p] + ex[i]);
    out->side_cy[i] = 0.5 * (ey[p] + ey[i]);
  }
  // centre: the point nearest (least squares) to the lines joining the
  // centres of opposite sides; their mean if those lines cannot fix a point
  double a11 = 0.0, a12 = 0.0, a22 = 0.0, r1 = 0.0, r2 = 0.0;
  int lines = 0;
  for (int i = 0; i < k / 2; ++i) {
    const int o = i + k / 2;
    double ux = out->side_cx[o] - out->side_cx[i], uy = out->side_cy[o] - out->side_cy[i];
    const double len = std::hypot(ux, uy);
    if (!(len > 0.0)) continue;
    ux /= len;
    uy /= len;
    const double m11 = 1.0 - ux * ux, m12 = -ux * uy, m22 = 1.0 - uy * uy;
    a11 += m11;
    a12 += m12;
    a22 += m22;
    r1 += m11 * out->side_cx[i] + m12 * out->side_cy[i];
    r2 += m12 * out->side_cx[i] + m22 * out->side_cy[i];
    ++lines;
  }
  const double det = a11 * a22 - a12 * a12;
  if (lines >= 2 && std::fabs(det) > 1e-12) {
    out->cx = (r1 * a22 - a12 * r2) / det;
    out->cy = (a11 * r2 - a12 * r1) / det;
  } else {
    out->cx = out->cy = 0.0;
    for (int i = 0; i < k; ++i) {
      out->cx += out->side_cx[i] / k;
      out->cy += out->side_cy[i] / k;
    }
  }
  double sum = 0.0, lo = INFINITY, hi = -INFINITY;
  for (int i = 0; i < k; ++i) {
    out->L[i] = v[i] - (nx[i] * out->cx + ny[i] * out->cy);
    sum += out->L[i];
    lo = std::fmin(lo, out->L[i]);
    hi = std::fmax(hi, out->L[i]);
  }
  for (int i = k; i < LBPF_MAX_FACETS; ++i)
    out->support[i] = out->side_cx[i] = out->side_cy[i] = out->L[i] = nan;
  out->L_avg = sum / k;
  out->Q = hi / lo;
  out->width = v[k] + v[k + 1];    // max x - min x
  out->height = v[k + 2] + v[k + 3];
  out->aspect = out->height > 0.0 ? out->width / out->height : nan;
  return LBPF_OK;
}

lbpf_status lbpf_measure_facets(lbpf_t* h, int k, const double* nx, const double* ny,
                        lbpf_facets* out) {
  int rc = lbpf_facets_enqueue(h, k, nx, ny);
  return rc ? rc : lbpf_facets_collect(h, out);
}

lbpf_status lbpf_growth_fit(const double* t, const double* L, int n, double* slope, double* intercept,
                    double* r2) {
  if (!t || !L || !slope || !intercept || !r2 || n < 2) return LBPF_EINVAL;
  double tm = 0.0, Lm = 0.0;
  for (int i = 0; i < n; ++i) {
    if (!std::isfinite(t[i]) || !std::isfinite(L[i])) return LBPF_EINVAL;
    tm += t[i];
    Lm += L[i];
  }
  tm /= n;
  Lm /= n;
  double stt = 0.0, stl = 0.0;
  for (int i = 0; i < n; ++i) {
    stt += (t[i] - tm) * (t[i] - tm);
    stl += (t[i] - tm) * (L[i] - Lm);
  }
  if (!(stt > 0.0)) return LBPF_EINVAL;
  const double b = stl / stt, a = Lm - b * tm;
  double res = 0.0, tot = 0.0;  // Eqs. 27, 28
  for (int i = 0; i < n; ++i) {
    const double e = L[i] - (a + b * t[i]);
    res += e * e;
    tot += (L[i] - Lm) * (L[i] - Lm);
  }
  *slope = b;
  *intercept = a;
  *r2 = tot > 0.0 ? 1.0 - res / tot : std::nan("");  // Eq. 26
  return LBPF_OK;
}

lbpf_status lbpf_set_solid(lbpf_t* h, const uint8_t* mask) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!mask) {
    h->m.solid = nullptr;
    h->m.solid_tiles = nullptr;
    drop_graph(h);
    ++h->gen;
    return LBPF_OK;
  }
  const int nx = h->m.nx, ny = h->m.ny, nz = h->m.nz, px = h->m.px;
  const size_t rows = size_t(ny) * nz;  // rows of nx nodes (y fastest, then z)
  if (h->m.bc[0] == LBPF_BC_INLET_OUTLET)
    for (size_t r = 0; r < rows; ++r)
      if (mask[r * nx] || mask[r * nx + nx - 1])
        return fail(h, LBPF_EINVAL, "the inlet and outlet columns must be fluid (row %zu)", r);
  std::vector<unsigned char> host(size_t(px) * rows, 0);
  for (size_t r = 0; r < rows; ++r)
    for (int x = 0; x < nx; ++x) host[r * px + x] = mask[r * nx + x] ? 1 : 0;
  const size_t nt =
      h->m.dim == 3 ? lbk::solid_chunk_count(h->m) : lbk::solid_tile_count(h->m);
  if (!h->d_solid) {
    cudaError_t e = cudaMalloc(&h->d_solid, host.size());
    if (e == cudaSuccess) e = cudaMalloc(&h->d_solid_tiles, nt);
    if (e != cudaSuccess) return fail(h, LBPF_ENOMEM, "solid mask: %s", cudaGetErrorString(e));
    h->dev_bytes += host.size() + nt;
  }
  CK(h, cudaMemcpyAsync(h->d_solid, host.data(), host.size(), cudaMemcpyHostToDevice, h->stream));
  h->m.solid = h->d_solid;
  h->m.solid_tiles = h->d_solid_tiles;
  CK(h, h->m.dim == 3 ? lbk::launch_solid_chunks(h->m, h->d_solid_tiles, h->stream)
                      : lbk::launch_solid_tiles(h->m, h->d_solid_tiles, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));  // the host copy goes out of scope
  drop_graph(h);
  ++h->gen;
  if (h->initialized && (rc = sync_solids(h))) return rc;
  return LBPF_OK;
}

lbpf_status lbpf_set_stream(lbpf_t* h, void* stream) {
  if (!h) return LBPF_EINVAL;
  h->stream = static_cast<cudaStream_t>(stream);
  return LBPF_OK;
}

size_t lbpf_device_bytes(const lbpf_t* h) { return h ? h->dev_bytes : 0; }

const char* lbpf_last_error(const lbpf_t* h) { return h ? h->msg : "null handle"; }

void lbpf_destroy(lbpf_t* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  drop_graph(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (int i = 0; i < 2; ++i) {
    if (h->pops[i]) cudaFree(h->pops[i]);
    if (h->phi[i]) cudaFree(h->phi[i]);
  }
  if (h->m.uring) cudaFree(h->m.uring);
  if (h->d_err) cudaFree(h->d_err);
  if (h->d_partials) cudaFree(h->d_partials);
  if (h->d_diag) cudaFree(h->d_diag);
  if (h->d_fields) cudaFree(h->d_fields);
  if (h->d_facets) cudaFree(h->d_facets);
  if (h->d_solid) cudaFree(h->d_solid);
  if (h->d_solid_tiles) cudaFree(h->d_solid_tiles);
  if (h->h_facets) cudaFreeHost(h->h_facets);
  delete h;
}

}  // extern "C"

// ---- batched sweep ------------------------------------------------------------------
namespace {

constexpr int kTuneWarm = 2, kTuneTimed = 4;

int bfail(lbpf_batch* b, int code, const char* fmt, ...) {
  if (!b) return code;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b->msg, sizeof(b->msg), fmt, ap);
  va_end(ap);
  if (code == LBPF_ECUDA || code == LBPF_ENONFINITE || code == LBPF_ETIMEDOUT) b->status = code;
  return code;
}

#define BCK(b, call)                                                                       \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return bfail(b, LBPF_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                   __LINE__);                                                              \
  } while (0)

void batch_drop_graph(lbpf_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

// (Re)build the device tables of every compiled variant from the instances.
int batch_build(lbpf_batch* b) {
  batch_drop_graph(b);
  for (int v = 0; v < b->nplans; ++v) lbk::batch_plan_free(&b->plans[v]);
  std::vector<lbk::BatchMember> mem(b->kids.size());
  for (size_t i = 0; i < b->kids.size(); ++i)
    if (b->kids[i]->m.chm != b->kids[0]->m.chm)
      return bfail(b, LBPF_EINVAL, "instance %d: a batch holds one flow collision", int(i));
  for (size_t i = 0; i < b->kids.size(); ++i) {
    lbpf* k = b->kids[i];
    mem[i].m = k->m;
    for (int c = 0; c < 2; ++c) {
      mem[i].pops[c] = k->pops[c];
      mem[i].rings[c] = k->phi[c];
    }
    mem[i].err = k->d_err;
    b->gens[i] = k->gen;
  }
  // one plan per (tile order, compiled variant): plan p = order * variants + variant
  const int nvar = lbk::batch_variant_count();
  b->nplans = lbk::kBatchOrders * nvar;
  if (b->nplans > int(sizeof(b->plans) / sizeof(b->plans[0])))
    return bfail(b, LBPF_EINVAL, "%d batch plans exceed the handle's table", b->nplans);
  const lbpf* k0 = b->kids[0];
  for (int p = 0; p < b->nplans; ++p)
    BCK(b, lbk::batch_plan_build(mem.data(), int(mem.size()), k0->m.storage, k0->m.flow,
                                 p % nvar, p / nvar, &b->plans[p]));
  return LBPF_OK;
}

int batch_launch(lbpf_batch* b, int v, cudaStream_t s) {
  BCK(b, lbk::batch_plan_launch(b->plans[v], b->cur, s));
  b->cur ^= 1;
  return LBPF_OK;
}

int batch_build_graph(lbpf_batch* b) {
  if (b->graph) return LBPF_OK;
  if (!b->cap_stream) BCK(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  const int saved = b->cur;
  b->cur = 0;
  cudaGraph_t g = nullptr;
  BCK(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = LBPF_OK;
  for (int i = 0; i < kGraphSteps && rc == LBPF_OK; ++i) rc = batch_launch(b, b->chosen, b->cap_stream);
  cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
  b->cur = saved;
  if (rc != LBPF_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return bfail(b, LBPF_ECUDA, "batch graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess)
    return bfail(b, LBPF_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
  return LBPF_OK;
}

}  // namespace

extern "C" {

lbpf_status lbpf_batch_create(const lbpf_params* p, const lbpf_seed* s, int count, void* stream,
                      lbpf_batch_t** out) {
  if (!p || !s || !out || count < 1 || count > 65535) return LBPF_EINVAL;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (p[i].dim != 2 || p[i].flow != p[0].flow || p[i].storage != p[0].storage ||
        p[i].storage == LBPF_FP64 || p[i].collision != p[0].collision) {
      fprintf(stderr,
              "lbpf_batch_create: instance %d: a batch holds 2D instances with one flow flag, "
              "one flow collision and one storage among FP32, FP16, BF16\n", i);
      return LBPF_EINVAL;
    }
  }
  lbpf_batch* b = new (std::nothrow) lbpf_batch();
  if (!b) return LBPF_ENOMEM;
  b->stream = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < count; ++i) {
    lbpf_t* k = nullptr;
    int rc = lbpf_create(&p[i], stream, &k);
    if (rc == LBPF_OK) {
      b->kids.push_back(k);
      rc = lbpf_init_seed(k, &s[i]);
    }
    if (rc != LBPF_OK) {
      fprintf(stderr, "lbpf_batch_create: instance %d: status %d %s\n", i, rc,
              k ? k->msg : "");
      lbpf_batch_destroy(b);
      return rc;
    }
  }
  b->gens.assign(count, 0);
  int rc = batch_build(b);
  if (rc != LBPF_OK) {
    fprintf(stderr, "lbpf_batch_create: %s\n", b->msg);
    lbpf_batch_destroy(b);
    return rc;
  }
  *out = b;
  return LBPF_OK;
}

lbpf_status lbpf_batch_step(lbpf_batch_t* b, int n) {
  if (!b) return LBPF_EINVAL;
  if (b->status != LBPF_OK) return b->status;
  if (n < 0) return bfail(b, LBPF_EINVAL, "n must be >= 0");
  bool rebuild = false;
  for (size_t i = 0; i < b->kids.size(); ++i) {
    lbpf* k = b->kids[i];
    if (k->status != LBPF_OK) return bfail(b, k->status, "instance %zu: %s", i, k->msg);
    if (!k->initialized) return bfail(b, LBPF_ESTATE, "instance %zu is not initialised", i);
    if (k->gen != b->gens[i]) rebuild = true;
  }
  if (rebuild) {
    int rc = batch_build(b);
    if (rc) return rc;
  }
  b->cur = b->kids[0]->cur;
  for (size_t i = 0; i < b->kids.size(); ++i)
    if (b->kids[i]->cur != b->cur)
      return bfail(b, LBPF_ESTATE, "instances were stepped apart; step them to equal parity");
  int left = n, rc;
  if (b->chosen < 0 && left >= b->nplans * (kTuneWarm + kTuneTimed)) {
    // time every variant on the live batch (they produce identical bits)
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    for (int v = 0; v < b->nplans; ++v) {
      for (int i = 0; i < kTuneWarm; ++i)
        if ((rc = batch_launch(b, v, b->stream))) return rc;
      BCK(b, cudaEventRecord(e0, b->stream));
      for (int i = 0; i < kTuneTimed; ++i)
        if ((rc = batch_launch(b, v, b->stream))) return rc;
      BCK(b, cudaEventRecord(e1, b->stream));
      BCK(b, cudaEventSynchronize(e1));
      float ms = 0.f;
      BCK(b, cudaEventElapsedTime(&ms, e0, e1));
      b->tune_ms[v] = ms / kTuneTimed;
      left -= kTuneWarm + kTuneTimed;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->chosen = 0;
    for (int v = 1; v < b->nplans; ++v)
      if (b->tune_ms[v] < b->tune_ms[b->chosen]) b->chosen = v;
  }
  const int v = b->chosen < 0 ? 0 : b->chosen;
  if (b->chosen >= 0 && left >= kGraphSteps) {
    if (b->cur == 1) {
      if ((rc = batch_launch(b, v, b->stream))) return rc;
      --left;
    }
    if (left >= kGraphSteps) {
      if ((rc = batch_build_graph(b))) return rc;
      while (left >= kGraphSteps) {
        BCK(b, cudaGraphLaunch(b->graph, b->stream));
        left -= kGraphSteps;
      }
    }
  }
  for (; left > 0; --left)
    if ((rc = batch_launch(b, v, b->stream))) return rc;
  for (lbpf* k : b->kids) {
    k->cur = b->cur;
    k->step += n;
  }
  return LBPF_OK;
}

lbpf_status lbpf_batch_diagnostics(lbpf_batch_t* b, lbpf_diag* out) {
  if (!b || !out) return LBPF_EINVAL;
  int worst = LBPF_OK;
  for (size_t i = 0; i < b->kids.size(); ++i) {
    const int rc = lbpf_diagnostics(b->kids[i], &out[i]);
    if (rc != LBPF_OK && worst == LBPF_OK) worst = rc;
  }
  return worst;
}

lbpf_t* lbpf_batch_instance(lbpf_batch_t* b, int i) {
  if (!b || i < 0 || i >= int(b->kids.size())) return nullptr;
  return b->kids[i];
}

lbpf_status lbpf_batch_count(const lbpf_batch_t* b) { return b ? int(b->kids.size()) : 0; }

lbpf_status lbpf_batch_tuning(const lbpf_batch_t* b, int* tile_rows, int* stages, float* ms, int* nvar) {
  if (!b) return LBPF_EINVAL;
  if (nvar) *nvar = b->nplans;
  if (ms)
    for (int v = 0; v < b->nplans; ++v) ms[v] = b->tune_ms[v];
  const int v = b->chosen;
  const int nv = lbk::batch_variant_count();
  if (tile_rows) *tile_rows = v < 0 ? 0 : lbk::batch_variant_rows(v % nv);
  if (stages) *stages = v < 0 ? 0 : lbk::batch_variant_stages(v % nv);
  return v < 0 ? LBPF_ESTATE : LBPF_OK;
}

const char* lbpf_batch_last_error(const lbpf_batch_t* b) { return b ? b->msg : "null handle"; }

void lbpf_batch_destroy(lbpf_batch_t* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (int v = 0; v < b->nplans; ++v) lbk::batch_plan_free(&b->plans[v]);
  for (lbpf* k : b->kids) lbpf_destroy(k);
  delete b;
}

}  // extern "C"
