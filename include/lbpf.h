/*
 * lbpf — coupled lattice-Boltzmann phase-field crystal-growth step on one
 * NVIDIA GB300 (sm_103a).  C ABI of liblbpf.so.
 *
 * The model is the one of Sec. 2 of Tan, Hosseini, Seidel-Morgenstern,
 * Thevenin and Lorenz, "Mandelic acid single-crystal growth: experiments vs
 * numerical simulations":
 *   - phase field phi (solid +1, liquid -1) on the modified LB scheme of
 *     Eq. 19 with source Eq. 20, equilibrium Eq. 21, moment Eq. 22 and
 *     relaxation Eq. 23, anisotropy a_s(n) of Eq. 3 with n = -grad phi/|grad phi|;
 *   - supersaturation U on the advection-diffusion LB of Eqs. 13-18 with the
 *     growth source of Eq. 14;
 *   - flow on the BGK LB of Eqs. 4-12 with Guo forcing (Eq. 5), the solid drag
 *     of Eq. 6 and the velocity mask of Eq. 7.
 * 2D uses D2Q9 for all three lattices; 3D uses D3Q19 for the flow and D3Q7
 * for U and phi.
 *
 * Conventions of every call:
 *   - returns LBPF_OK (0) or a negative lbpf_status; never aborts;
 *   - a NULL or destroyed handle gives LBPF_EINVAL;
 *   - errors are sticky per handle: after a CUDA error or a device-detected
 *     non-finite value every later call returns that status, and
 *     lbpf_last_error() gives a one-line description;
 *   - the library owns all device memory of a handle; host buffers passed in
 *     are owned by the caller and are not retained after the call returns;
 *   - work is issued on the CUDA stream given at creation (NULL = legacy
 *     default stream); calls documented as synchronising wait for that
 *     stream, the others return as soon as the work is queued.
 * Node order of every field and state array: x fastest, then y, then z;
 * no padding.
 */
#ifndef LBPF_H
#define LBPF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbpf lbpf_t;

typedef enum {
  LBPF_OK = 0,
  LBPF_EINVAL = -1,      /* invalid argument, parameter or buffer size */
  LBPF_ECUDA = -2,       /* a CUDA runtime call failed */
  LBPF_ENOMEM = -3,      /* device or host allocation failed */
  LBPF_ESTATE = -4,      /* call out of order (e.g. step before init) */
  LBPF_ENONFINITE = -5,  /* a NaN/Inf appeared in the fields */
  LBPF_ETIMEDOUT = -6    /* a bounded device wait gave up */
} lbpf_status_code;
/* What every status-returning call returns: one of the lbpf_status_code
 * values above (an int, so that the ABI is the same from C, C++ and any
 * foreign-function interface). */
typedef int lbpf_status;

/* Boundary condition per axis. */
enum {
  LBPF_BC_PERIODIC = 0,
  /* x only: inflow ghost at x = -1 in equilibrium with rho = 1,
   * u = (u_inlet, 0, 0), U = u0_inlet, phi = -1; outflow ghost at x = nx that
   * repeats the post-collision state of the last column (zero gradient). */
  LBPF_BC_INLET_OUTLET = 1,
  /* half-way bounce-back for f, g and h (zero flux; no-slip for the flow) */
  LBPF_BC_WALL = 2
};

/* Population storage.  Arithmetic is FP32 except for LBPF_FP64. */
enum {
  LBPF_FP32 = 0,
  LBPF_FP64 = 1,
  LBPF_FP16_SHIFTED = 2, /* binary16 deviation from the lattice weight times a reference moment */
  LBPF_BF16_SHIFTED = 3  /* bfloat16, same shift */
};
/* With 16-bit storage the reference moment of g is per node (2D and 3D):
 * each node keeps its U of an earlier step (FP16, two planes that alternate
 * with the population buffers), and the g pushed to a node is stored as its
 * deviation from w_a times that node's reference.  The rounding of the stored
 * deviations then no longer accumulates into a drift of the growth rate over
 * long runs.  f and h keep one global reference. */

/* Field selection bits of lbpf_read_fields. */
enum {
  LBPF_FIELD_PHI = 1u << 0,      /* phi = sum h (Eq. 22) */
  LBPF_FIELD_U = 1u << 1,        /* U = sum g (Eq. 17) */
  LBPF_FIELD_RHO = 1u << 2,      /* rho = sum f (Eq. 11); 1 without flow */
  LBPF_FIELD_UX = 1u << 3,       /* fluid velocity (Eq. 12 with the Guo half force) */
  LBPF_FIELD_UY = 1u << 4,
  LBPF_FIELD_UZ = 1u << 5,
  LBPF_FIELD_PHI_PREV = 1u << 6, /* phi at the previous time level */
  LBPF_FIELD_STATE = 1u << 8     /* the full restartable state (see below) */
};

/* Model and run parameters.  Lattice units: dx = dt = 1. */
typedef struct {
  int dim;            /* 2 or 3 */
  int nx, ny, nz;     /* grid; nz is ignored (taken as 1) in 2D */
  int bc[3];          /* LBPF_BC_* for x, y, z; INLET_OUTLET only on x */
  int flow;           /* 0: phase field + solute only; 1: coupled flow lattice */
  int storage;        /* LBPF_FP32, LBPF_FP64, LBPF_FP16_SHIFTED, LBPF_BF16_SHIFTED */
  int fold;           /* k of a_s = 1 + eps cos(k (theta - theta0)) (Eq. 3), 1..12;
                         0 = cubic a_s = 1 - 3 eps + 4 eps sum n_i^4 (required in 3D) */
  int aniso_literal;  /* 0: N = |grad phi|^2 a_s d(a_s)/d(grad phi) (Eq. 21 read in
                         its variational form); 1: twice that (the literal factor) */
  double tau_phi0;    /* tau_phi at a_s = 1 (Eq. 23); sets tau0 = W0^2/(cs^2 (tau_phi0 - 1/2)) */
  double tau_u_liquid;/* tau_U in the liquid (Eq. 18); D = cs^2 (tau_u_liquid - 1/2) */
  double tau_f;       /* flow relaxation time (Eq. 10); nu = (tau_f - 1/2)/3 */
  double w0;          /* interface width W0 (Eqs. 1, 6, 21, 23) */
  double lambda;      /* coupling constant (Eq. 20); < 0 selects D tau0 / (0.6267 W0^2) */
  double eps_aniso;   /* anisotropy strength eps (Eq. 3), 0 <= eps < 1 */
  double theta0;      /* anisotropy orientation (radians) */
  double h_drag;      /* drag constant h of Eq. 6 (2.757) */
  double u_inlet;     /* inflow velocity along +x (|u| <= 0.1) */
  double u0_inlet;    /* supersaturation of the inflow */
  double body_force[3]; /* constant body force density (test flows); usually 0 */
  int collision;      /* flow collision: LBPF_COLL_BGK (Eq. 8) or LBPF_COLL_CHM */
  double chm_omega_bulk; /* CHM: rate of the trace of the second-order central
                            moments, in (0, 2); 0 selects 1 */
  double chm_omega_high; /* CHM: rate of the third- and fourth-order central
                            moments, in (0, 2); 0 selects 1 */
} lbpf_params;

/* Flow collision.  LBPF_COLL_CHM: the central Hermite multiple-relaxation-
 * time collision the paper uses for the flow (after Eq. 9; defined in the
 * work it cites), with flow only.  Central Hermite moments of f about the
 * equilibrium velocity u* (in 2D the nine D2Q9 polynomials of X = c_x - u*_x,
 * Y = c_y - u*_y: 1, X, Y, X^2 - cs^2, Y^2 - cs^2, XY, X^2 Y - cs^2 Y,
 * X Y^2 - cs^2 X, X^2 Y^2 - cs^2 (X^2 + Y^2) + cs^4; in 3D the nineteen
 * D3Q19 products H_i(X) H_j(Y) H_k(Z), H_0 = 1, H_1 = X, H_2 = X^2 - cs^2,
 * i, j, k <= 2 with at most two non-zero) relax towards rho and zeros: first
 * order, the mixed and the deviatoric second order at 1/tau_f (the first
 * order with (1 - 1/(2 tau_f)) F, as Eq. 4-5 do), the trace of the second
 * order at chm_omega_bulk, third and fourth order at chm_omega_high.  With
 * every rate 1/tau_f and no force it is BGK with the equilibrium that has
 * the Maxwellian's moments (in 2D the product form).  A batch holds one
 * collision for all its instances. */
enum { LBPF_COLL_BGK = 0, LBPF_COLL_CHM = 1 };

/* Circular (2D) / spherical (3D) seed: phi0 = tanh((radius - r)/(sqrt(2) W0))
 * + noise_amp * xi, xi in [-1, 1) from SplitMix64 of (seed XOR
 * (node_index * 0x9E3779B97F4A7C15)); U = u0; rho = 1;
 * u = (u_inlet, 0, 0) when flow is on; all populations at equilibrium. */
typedef struct {
  double cx, cy, cz;  /* centre in node units */
  double radius;
  double u0;          /* initial supersaturation */
  double noise_amp;
  uint64_t seed;
} lbpf_seed;

/* Convex polygon seed, 2D (the rhombic and hexagonal seeds of Sec. 3.1):
 * the polygon {x : (x - c) . n_i <= dist_i for every facet i}. */
#define LBPF_MAX_FACETS 12
typedef struct {
  double cx, cy;                /* centre in node units */
  int nfacets;                  /* 3 .. LBPF_MAX_FACETS */
  double nx[LBPF_MAX_FACETS];   /* outward unit normal of facet i */
  double ny[LBPF_MAX_FACETS];
  double dist[LBPF_MAX_FACETS]; /* distance of facet i's line from the centre */
  double u0;                    /* initial supersaturation */
  double noise_amp;
  uint64_t seed;
} lbpf_polygon_seed;

/* Shape of a faceted 2D crystal (Sec. 3.1.2, Sec. 3.2), from the phi = 0
 * contour: the crossings of phi = 0 on the grid's x- and y-edges (phi > 0 at
 * one end only; linear interpolation; no edge across a periodic wrap). */
typedef struct {
  int64_t points;                  /* contour points found; 0: every value NaN */
  int nfacets;
  double support[LBPF_MAX_FACETS]; /* h_i = max over the contour of p . n_i (node units) */
  double side_cx[LBPF_MAX_FACETS]; /* centre of side i: midpoint of the segment of */
  double side_cy[LBPF_MAX_FACETS]; /* p . n_i = h_i between sides i - 1 and i + 1 */
  double cx, cy;                   /* crystal centre: least-squares meet of the lines
                                      joining the centres of opposite sides */
  double L[LBPF_MAX_FACETS];       /* normal distance of side i from the centre */
  double L_avg;                    /* mean of L */
  double Q;                        /* quality parameter max L / min L (Sec. 3.2) */
  double width, height;            /* extent of the contour along x and along y */
  double aspect;                   /* width / height (Sec. 3.2) */
} lbpf_facets;

/* FP64 diagnostics of the current state. */
typedef struct {
  int64_t step;
  double solute_total;      /* sum over nodes of U(t) + phi(t-1); conserved without inflow */
  double solute_drift_rel;  /* (solute_total - value at init) / |value at init| */
  double mass_total;        /* sum rho */
  double solid_volume;      /* sum (1 + clamp(phi, -1, 1)) / 2 */
  double r_eq;              /* equivalent radius of solid_volume (circle / sphere) */
  double iface_pos[6];      /* distance of the phi = 0 crossing from the seed-centre
                               node along +x, -x, +y, -y, +z, -z; -1 if none */
  double max_u;             /* max |u| */
  int64_t nonfinite;        /* nodes with a non-finite phi, U or rho */
} lbpf_diag;

/* Fill *p with the defaults: 2D 128 x 128 periodic, no flow, FP32, fold 4,
 * eps 0.05, tau_phi0 = tau_u_liquid = 0.8, tau_f = 0.6, W0 = 2, default
 * lambda, h_drag = 2.757. */
lbpf_status lbpf_params_default(lbpf_params* p);

/* Validate *p, allocate the device state and return a handle in *out.
 * stream: a cudaStream_t (NULL = legacy default stream).  EINVAL cases:
 * tau <= 1/2, W0 <= 0, eps outside [0, 1), fold outside 0..12 (or != 0 in
 * 3D), grid dimension < 4, INLET_OUTLET on y or z, |u_inlet| > 0.1. */
lbpf_status lbpf_create(const lbpf_params* p, void* stream, lbpf_t** out);

/* Initial state from a seed (computed on the device in FP64, stored in the
 * population type); resets the step counter to 0.  Asynchronous. */
lbpf_status lbpf_init_seed(lbpf_t* h, const lbpf_seed* s);

/* Initial state from a convex polygon seed (2D only): phi0 = tanh(-s /
 * (sqrt(2) W0)) with s = max_i [(x - c) . n_i - dist_i], plus the noise of
 * lbpf_init_seed (same generator and amplitude meaning); U = u0, rho = 1, the
 * inlet velocity as there.  Resets the step counter.  EINVAL for 3D, a
 * facet count outside 3..LBPF_MAX_FACETS, a normal whose length differs from
 * 1 by more than 1e-9, or a non-finite value.  Asynchronous. */
lbpf_status lbpf_init_polygon(lbpf_t* h, const lbpf_polygon_seed* s);

/* Initial state from host FP64 fields of nx*ny*nz values each: every
 * population at the equilibrium of (rho, u* = (1 - clamp(phi))/2 u, U, phi);
 * phi(t-1) = phi.  rho, ux, uy, uz may be NULL (1, 0).  Synchronising. */
lbpf_status lbpf_init_fields(lbpf_t* h, const double* phi, const double* U, const double* rho,
                     const double* ux, const double* uy, const double* uz);

/* Advance n >= 0 coupled steps (Eqs. 4-23, pull-equivalent push streaming).
 * Asynchronous; n = 0 is a no-op. */
lbpf_status lbpf_step(lbpf_t* h, int n);

/* Copy fields to host_dst (caller-owned).  Without LBPF_FIELD_STATE: the
 * selected fields one after another in bit order, nx*ny*nz values each, as
 * double if as_fp64 else float; bytes must equal that total.  With
 * LBPF_FIELD_STATE alone: the restartable state of lbpf_state_bytes() bytes.
 * Synchronising. */
lbpf_status lbpf_read_fields(lbpf_t* h, unsigned field_mask, void* host_dst, size_t bytes,
                     int as_fp64);

/* Size of the restartable state: a 128-byte header (magic "LBPFST02", int64
 * step, int32 dim, nx, ny, nz, storage, flow, populations per node, element
 * bytes, then at byte 48 the double U_ref, at byte 56 int32 cx, cy, cz: the
 * node the interface rays of lbpf_diagnostics start from, at byte 72 the
 * double solute total at initialisation that solute_drift_rel is relative
 * to; the rest zero), then the populations
 * direction-major in the storage type (f, then g, then h; directions in the
 * order: D2Q9 (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1);
 * D3Q19 rest, +x, -x, +y, -y, +z, -z, (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0)
 * (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1);
 * D3Q7 the first seven of those), each stored as its deviation
 * d_a = p_a - w_a M_ref with M_ref = 1 for f, U_ref for g and -1 for h; then
 * phi(t-1) + 1 in FP64 for LBPF_FP64 storage and FP32 otherwise; then, for
 * 16-bit storage only, two FP16 planes of nx*ny*nz values: the per-node g
 * reference of the stored populations (their M_ref of g instead of U_ref),
 * and the one the next step encodes against. */
size_t lbpf_state_bytes(const lbpf_t* h);

/* Restore a state written by lbpf_read_fields(LBPF_FIELD_STATE) of a handle
 * with the same grid, flow and storage: the populations, the phi ring, the
 * step count and the diagnostics' references (ray origin, initial solute
 * total), so that a restored run continues and reports exactly as the
 * uninterrupted one.  Synchronising. */
lbpf_status lbpf_write_state(lbpf_t* h, const void* host_src, size_t bytes);

/* FP64 reductions of the current state (deterministic two-pass sums).
 * Synchronising; reports a non-finite state as LBPF_ENONFINITE. */
lbpf_status lbpf_diagnostics(lbpf_t* h, lbpf_diag* out);

/* Crystal shape of the current state along k facet normals (nx[k], ny[k],
 * host arrays read during the call): k even in 4..LBPF_MAX_FACETS, unit
 * normals in counter-clockwise order, normal i + k/2 opposite to normal i.
 * The support values are FP64 maxima over the contour, reduced on the device
 * in a fixed order (reproducible bit for bit); the side centres, the centre
 * and the lengths follow on the host in FP64.  The first call allocates a
 * small device scratch.  2D only (EINVAL otherwise); ESTATE before init.
 * Synchronising. */
lbpf_status lbpf_measure_facets(lbpf_t* h, int k, const double* nx, const double* ny,
                        lbpf_facets* out);

/* The same in two halves.  lbpf_facets_enqueue validates as above and queues
 * the device part on the handle's stream (the state at that point of the
 * stream is measured; the normals are copied); asynchronous.
 * lbpf_facets_collect waits for it and fills *out (synchronising); ESTATE if
 * nothing is queued.  A second enqueue before the collect replaces the
 * first. */
lbpf_status lbpf_facets_enqueue(lbpf_t* h, int k, const double* nx, const double* ny);
lbpf_status lbpf_facets_collect(lbpf_t* h, lbpf_facets* out);

/* Straight-line fit L'(t) = intercept + slope t of a size history of n >= 2
 * points (host arrays), and its coefficient of determination R^2 =
 * 1 - A_res / A_tot (Eqs. 26-28); R^2 is NaN when every L is the same.
 * EINVAL for a null pointer, n < 2, non-finite data or all t equal.  A host
 * computation; needs no handle. */
lbpf_status lbpf_growth_fit(const double* t, const double* L, int n, double* slope, double* intercept,
                    double* r2);

/* Solid nodes (the reactor walls and baffles of Sec. 3.1.2 and 3.2): mask is
 * a host array of nx*ny*nz bytes (x fastest, then y, then z; nz = 1 in 2D),
 * nonzero = solid, read during the call; NULL removes the mask.  A fluid node
 * sends what it would stream into a solid node back into itself reversed
 * (half-way bounce-back, for f, g and h: no flow through, zero flux of U and
 * phi); in the phi gradient a solid neighbour x + c counts as the first fluid
 * node among the single-axis steps x + c_x e_x, x + c_y e_y, x + c_z e_z (those
 * with a non-zero component, in that order) and x itself (zero normal
 * derivative; for a straight row or plane of solid nodes this is exactly the
 * LBPF_BC_WALL boundary).  Solid nodes keep their state (both buffers hold it;
 * the field read-out and the diagnostics include their constant values).
 * Tiles (3D: column chunks) that touch no solid node run at full speed.  With
 * LBPF_BC_INLET_OUTLET the first and last columns (x = 0 and x = nx - 1 of
 * every row) must be fluid.  The mask is configuration, not state:
 * lbpf_write_state keeps it.  The block propagator refuses a handle with solid
 * nodes.  Synchronising. */
lbpf_status lbpf_set_solid(lbpf_t* h, const uint8_t* mask);

/* Rebind the handle to another stream (e.g. the caller's current stream). */
lbpf_status lbpf_set_stream(lbpf_t* h, void* stream);

/* Bytes of device memory the handle owns. */
size_t lbpf_device_bytes(const lbpf_t* h);

/* Human-readable description of the last error of h ("" if none). */
const char* lbpf_last_error(const lbpf_t* h);

/* Release everything the handle owns; NULL is a no-op. */
void lbpf_destroy(lbpf_t* h);

/* ---- batched sweep ------------------------------------------------------------
 * Many independent 2D instances (the parametric sweeps of Sec. 3: supersaturation,
 * seed size, inflow) advanced together by ONE persistent kernel launch per time
 * step: the tiles of all instances are split over the resident CTAs once per
 * plan.  Every instance is an ordinary handle with its own state
 * (lbpf_batch_instance); a batched instance evolves bit for bit like the same
 * instance stepped alone.  Several tile shapes are compiled, each with two tile
 * orders (large instances interleaved, or instance after instance); the first
 * lbpf_batch_step that is long enough (>= 48 steps) times every (order, shape)
 * plan on the live batch and keeps the fastest (lbpf_batch_tuning); every plan
 * produces the same bits.  Steps of 64 are replayed from a CUDA graph. */
typedef struct lbpf_batch lbpf_batch_t;

/* Create `count` instances (1..65535) from p[i] and seed them with s[i]
 * (lbpf_create + lbpf_init_seed each).  All p[i] must be 2D with the same
 * `flow`, the same `collision` and the same storage among LBPF_FP32,
 * LBPF_FP16_SHIFTED, LBPF_BF16_SHIFTED; sizes and every other model
 * parameter may differ.  EINVAL otherwise.  Instances may carry solid nodes
 * (lbpf_set_solid on lbpf_batch_instance; picked up by the next step).  stream: as for lbpf_create, shared by all instances. */
lbpf_status lbpf_batch_create(const lbpf_params* p, const lbpf_seed* s, int count, void* stream,
                      lbpf_batch_t** out);

/* Advance every instance by n >= 0 steps.  Asynchronous, except that the
 * first call of >= 24 steps synchronises once to time the tile shapes.
 * Instances re-initialised or restored since the last call are picked up;
 * instances stepped individually to a different buffer parity give
 * LBPF_ESTATE.  An error of any instance is reported here. */
lbpf_status lbpf_batch_step(lbpf_batch_t* b, int n);

/* lbpf_diagnostics of every instance into out[0..count-1].  Synchronising;
 * returns the first non-OK status (all entries are still filled). */
lbpf_status lbpf_batch_diagnostics(lbpf_batch_t* b, lbpf_diag* out);

/* Borrowed handle of instance i (NULL if out of range); owned by the batch.
 * Use it for lbpf_read_fields, lbpf_diagnostics, lbpf_write_state. */
lbpf_t* lbpf_batch_instance(lbpf_batch_t* b, int i);
lbpf_status lbpf_batch_count(const lbpf_batch_t* b);

/* The tile shape the tuner chose (rows of the 32-wide tile, pipeline stages)
 * and the measured ms per step of each plan (ms[0..*nvar-1], at most 8: plan
 * p is tile order p / 4 (0 large instances interleaved, 1 instance after
 * instance) with compiled shape p % 4); any pointer may be NULL.  LBPF_ESTATE
 * before tuning has run. */
lbpf_status lbpf_batch_tuning(const lbpf_batch_t* b, int* tile_rows, int* stages, float* ms, int* nvar);
const char* lbpf_batch_last_error(const lbpf_batch_t* b);
void lbpf_batch_destroy(lbpf_batch_t* b);

/* ---- learned surrogate --------------------------------------------------------
 * A BF16 U-Net (NHWC activations, FP32 accumulation, FP32 master weights,
 * Adam) trained and run by the library's own tensor-core kernels.  It maps
 * normalised fields (phi, U, ux, uy) to the normalised change of those fields
 * over a fixed block of LB steps.  Architecture per level l (channels
 * C_l = base_ch 2^l): encoder conv3x3 + ReLU twice, 2x2 average pooling;
 * decoder nearest 2x upsampling, conv3x3 + ReLU, concatenation with the
 * encoder output, conv3x3 + ReLU twice; a 1x1 FP32 head.  There is no
 * counterpart in the paper: it is the sweep-exploration accelerator whose
 * fallback and judge is the LB step above. */
typedef struct lbpf_unet lbpf_unet_t;
typedef struct {
  int in_ch, out_ch;  /* 1..16 inputs, 1..4 outputs */
  int base_ch;        /* 32 */
  int levels;         /* 1..6 */
  int batch, height, width; /* width / 2^(levels-1) a multiple of 64 */
  uint64_t seed;      /* weight initialisation (He uniform, SplitMix64) */
} lbpf_unet_cfg;

/* Allocates the network's weights, optimiser state and activations on the
 * current device (owned by the handle until lbpf_unet_destroy) and
 * initialises the weights from cfg->seed.  stream: the CUDA stream its work
 * is queued on (NULL = legacy default).  LBPF_EINVAL for an unsupported
 * configuration (reason on stderr), LBPF_ENOMEM if an allocation fails. */
lbpf_status lbpf_unet_create(const lbpf_unet_cfg* cfg, void* stream, lbpf_unet_t** out);
/* x: device FP32 [batch][height][width][in_ch]; y: device FP32 [..][out_ch];
 * both caller-owned, not overlapping.  Asynchronous on the network's stream. */
lbpf_status lbpf_unet_forward(lbpf_unet_t* n, const float* x, float* y);
/* Loss (mean squared error against device FP32 targets t, same layout as y)
 * and the gradients of every parameter, without updating them; the loss is
 * written to *loss_host (synchronising) if loss_host is not NULL. */
lbpf_status lbpf_unet_grad(lbpf_unet_t* n, const float* x, const float* t, float* loss_host);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) at learning rate lr; the loss
 * of the batch goes to the device float *loss_dev if not NULL.  Asynchronous. */
lbpf_status lbpf_unet_train_step(lbpf_unet_t* n, const float* x, const float* t, float lr,
                         float* loss_dev);
/* The training loop of the block propagator's network, on pairs held on the
 * device: per step, a minibatch of pairs gathered (and mirrored) into the
 * network's own buffers, then one lbpf_unet_train_step at the step's learning
 * rate; every step is queued on the network's stream, with one
 * synchronisation at the end.
 *   X, T: device FP32 [n_pairs][height][width][4], the normalised fields
 *         (phi, U, ux, uy) and their targets (lbpf_surrogate_sample /
 *         lbpf_surrogate_target); height and width those of the network,
 *         which maps 4 inputs to 4 outputs.  Caller-owned, read only.
 *   idx:  host int32 [steps][batch], the pairs of each minibatch, in
 *         [0, n_pairs);
 *   flip: host int32 [steps] or NULL: 0 as stored, 1 mirrored in y (row
 *         height-1-i, uy negated), 2 mirrored in x (column width-1-j, ux
 *         negated) -- the mirror symmetries of a channel with walls in y;
 *   lr:   host float [steps], the learning rate of each step (>= 0, finite);
 *   loss_log: host float [ceil(steps / log_every)] or NULL: the minibatch
 *         loss at steps log_every, 2 log_every, ... and at the last step.
 * The caller draws the minibatches and the schedule: the same draws give the
 * same minibatches and rates as a loop of lbpf_unet_train_step calls (the
 * gradients are reduced with atomic additions, so two runs agree to rounding,
 * not bit for bit).  The first call allocates two minibatch buffers
 * owned by the network.  LBPF_EINVAL for an index, flip or rate out of range
 * or a network that is not 4 -> 4 (nothing queued). */
lbpf_status lbpf_surrogate_train(lbpf_unet_t* net, const float* X, const float* T, int64_t n_pairs,
                         int steps, const int32_t* idx, const int32_t* flip, const float* lr,
                         int log_every, float* loss_log);

/* Number of parameters and their copy to / from host FP32 memory in a fixed
 * order: the first encoder convolution of every level (0..L-1), the second
 * encoder convolution of every level, the upsampling convolution of every
 * level 0..L-2, the first and then the second decoder convolution of every
 * level 0..L-2 -- each as weights [9][Cout][Cin] (taps row-major) then bias
 * [Cout]; then the head weights [out][C0] and bias [out].  The first encoder
 * convolution has Cin = 16 (inputs zero-padded).  which: 0 weights,
 * 1 gradients; set = 1 writes weights.  Synchronising. */
size_t lbpf_unet_param_count(const lbpf_unet_t* n);
lbpf_status lbpf_unet_params(lbpf_unet_t* n, int which, float* host, size_t count, int set);
/* Select the convolution kernels: 1 (default) the tcgen05 / TMEM / TMA
 * kernel wherever the layer's shape allows it, 0 the warp-level mma.sync
 * kernel everywhere.  Takes effect at the next pass. */
lbpf_status lbpf_unet_set_tensor_path(lbpf_unet_t* n, int use_tcgen05);
/* Synchronises the network's stream and returns LBPF_ETIMEDOUT if a
 * tensor-core kernel gave up waiting on one of its barriers since creation
 * (lbpf_unet_grad and lbpf_surrogate_advance check the same). */
lbpf_status lbpf_unet_status(lbpf_unet_t* n);
size_t lbpf_unet_device_bytes(const lbpf_unet_t* n);
const char* lbpf_unet_last_error(const lbpf_unet_t* n);
void lbpf_unet_destroy(lbpf_unet_t* n);

/* ---- learned block propagator -----------------------------------------------
 * Advances a 2D simulation by blocks of steps_per_block LB steps, each either
 * by one application of a trained network (input: the fields (phi, U, ux, uy)
 * normalised as (f - shift) / scale; output: their change over the block
 * divided by res_scale) or, as fallback, by the LB step itself.  The LB is
 * also the judge: on judged blocks it advances the state and the network's
 * prediction from the same start is measured against it.  A prediction is
 * committed (the state becomes the equilibrium of the predicted fields at
 * the current density, with phi(t-1) from the block's mean rate of change)
 * only if
 *   - the predicted solute invariant sum(U + phi(t-1)) (Eq. 13 with its
 *     source -dphi/dt: conserved by the LB in a closed domain) differs from
 *     the value at initialisation by at most drift_tol (relative), and
 *   - its interface error estimate is at most iface_tol lattice units: the
 *     largest difference, over the axis rays of lbpf_diag.iface_pos, between
 *     the predicted interface displacement and the displacement the LB
 *     produced in its most recent block; and, if iface_budget > 0, the
 *     accumulated estimate stays within iface_budget: per ray, the signed
 *     sum of those differences over every block the call has committed (this
 *     one included), never reset, so that a biased network runs into the
 *     bound and the rest of the call falls back to the LB; and, if
 *     iface_rel_tol > 0, the estimate is also at most iface_rel_tol times the
 *     largest displacement of that LB block over the rays, so that a network
 *     that freezes or doubles the growth fails even where the interface moves
 *     far less than iface_tol per block.
 * A judged prediction earns trust if its error against the LB block (the
 * largest difference of the interface positions over the rays) is at most
 * iface_tol and, if iface_rel_tol > 0, at most iface_rel_tol times the LB
 * block's largest displacement.
 * An accepted prediction's remaining solute deficit is spread over the
 * liquid in proportion to (1 - phi)/2 before it is committed, so that the
 * committed state keeps the invariant exactly as the LB does.
 * A block that fails a check is advanced by the LB and the next block is
 * judged; so is every judge_every-th block (0: only those).  Meaningful for
 * closed domains (periodic or wall boundaries); the network must have
 * batch 1, 4 inputs, 4 outputs, height ny and width nx. */
typedef struct {
  int steps_per_block;       /* LB steps one network application stands for (>= 1) */
  int judge_every;           /* judge every judge_every-th block (0: only after a failed check) */
  double drift_tol;          /* relative solute drift bound (e.g. 1e-3) */
  double iface_tol;          /* per-block interface error bound, lattice units (e.g. 1.0) */
  double iface_budget;       /* bound on the accumulated estimate over a call (0: none) */
  double iface_rel_tol;      /* bound relative to the LB's displacement per block (0: none) */
  float shift[4], scale[4];  /* input normalisation of (phi, U, ux, uy); scale != 0 */
  float res_scale[4];        /* output scale of the change of (phi, U, ux, uy) */
} lbpf_surrogate_cfg;

typedef struct {
  int64_t blocks;            /* blocks advanced by the call */
  int64_t surrogate_blocks;  /* advanced by the network */
  int64_t judged_blocks;     /* advanced by the LB while judging a prediction */
  int64_t fallback_blocks;   /* advanced by the LB because a check failed */
  double max_drift;          /* largest predicted relative solute drift (before correction) */
  double max_iface_err;      /* largest judged interface error (lattice units) */
  double max_iface_est;      /* largest per-block interface error estimate committed */
  double iface_acc;          /* accumulated estimate at the end of the call (largest ray) */
  double max_drift_committed; /* largest drift among the blocks the network advanced
                                 (at most drift_tol: a larger one falls back to the LB) */
} lbpf_surrogate_report;

/* The network input of the current state: device FP32 [ny][nx][4]. */
lbpf_status lbpf_surrogate_sample(lbpf_t* h, const lbpf_surrogate_cfg* cfg, float* x);
/* Training target from the inputs x0 (state at t) and x1 (at t + block):
 * t = (x1 - x0) scale / res_scale per channel; device FP32 [npix][4];
 * queued on `stream`. */
lbpf_status lbpf_surrogate_target(const lbpf_surrogate_cfg* cfg, const float* x0, const float* x1,
                          int64_t npix, float* t, void* stream);
/* Advance `blocks` blocks (synchronising once per block); rep may be NULL.
 * The network's kernels run on the simulation's stream during the call.  The
 * first call for a network allocates its propagator scratch (device memory
 * and a small pinned host buffer, owned by the network) and captures the
 * prediction phase as a CUDA graph per state buffer, recaptured when the
 * simulation, its stream or cfg change: do not call it inside a stream
 * capture of your own.  The scratch (its FP64 reduction included) belongs to
 * the network, so propagators with networks of their own run independently,
 * on unordered streams too; calls that share one network must not overlap
 * (from several host threads).  LBPF_ETIMEDOUT if a tensor-core kernel gave
 * up waiting; LBPF_EINVAL for a mismatched network or cfg. */
lbpf_status lbpf_surrogate_advance(lbpf_t* h, lbpf_unet_t* net, const lbpf_surrogate_cfg* cfg,
                           int blocks, lbpf_surrogate_report* rep);

/* ---- allocation-free reduction ------------------------------------------------
 * The paper has no counterpart of this entry point; it serves callers that
 * cannot allocate device memory where they need the conservation sums: code
 * running inside a memory-pool or allocator callback, a host whose own arena
 * owns all of the GPU's memory, or a real-time loop in which a cudaMalloc would
 * stall.  It computes the three FP64 sums of lbpf_diagnostics from fields the
 * caller already holds on the device, and allocates nothing: its only scratch
 * (the per-block partial sums of a deterministic two-pass reduction) is a
 * fixed file-scope device array of LBPF_NOALLOC_MAX_BLOCKS x 3 doubles
 * (96 KiB), which every GPU that loads the library holds until the process
 * exits.
 *
 * phi, phi_prev, U, rho: device arrays of n values each, float (fp64 = 0) or
 * double (fp64 = 1), caller-owned; rho may be NULL (taken as 1).
 * out: device pointer to 3 doubles, caller-owned, written with
 *   out[0] = sum(U + phi_prev)   (lbpf_diag.solute_total),
 *   out[1] = sum(rho)            (lbpf_diag.mass_total),
 *   out[2] = sum((1 + clamp(phi, -1, 1)) / 2)   (lbpf_diag.solid_volume).
 * n above LBPF_NOALLOC_MAX_NODES returns LBPF_EINVAL (the scratch holds one
 * row per block, and a block covers at most 256 x 64 nodes); a NULL input or
 * output, or n < 0, also returns LBPF_EINVAL.  Work is queued on `stream`
 * (NULL = legacy default stream) and the call returns without waiting.
 * The first call on a device looks up the device address of the scratch
 * array (with that device current): make that first call before any stream
 * capture.  The address is kept per device together with the ID of the
 * context it belongs to, and looked up again when that context changes (after
 * a cudaDeviceReset, for instance).  Every call shares the one scratch array;
 * calls that can overlap on the GPU (different streams without ordering) race
 * on it and must be serialised by the caller.  The library's own block
 * propagator does not use it (it reduces into its network's scratch). */
#define LBPF_NOALLOC_MAX_BLOCKS 4096
#define LBPF_NOALLOC_MAX_NODES ((int64_t)LBPF_NOALLOC_MAX_BLOCKS * 256 * 64)
lbpf_status lbpf_field_sums_noalloc(const void* phi, const void* phi_prev, const void* U,
                            const void* rho, int64_t n, int fp64, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBPF_H */
