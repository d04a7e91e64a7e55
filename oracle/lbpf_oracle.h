/*
 * FP64 CPU oracle of the coupled lattice-Boltzmann phase-field crystal-growth
 * step (Tan, Hosseini, Seidel-Morgenstern, Thevenin, Lorenz, "Mandelic acid
 * single-crystal growth: experiments vs numerical simulations", Sec. 2.2,
 * Eqs. 1-23).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the independent checker of the CUDA
 * library.  Only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it; the product path never does.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Everything is plain double-precision loops over nodes and directions in the
 * order the paper states the operators: moments (Eqs. 11, 12, 17, 22), normal
 * and anisotropy (Eq. 3, Eq. 21, Eq. 23), sources (Eq. 14, Eq. 20), forcing
 * (Eqs. 5-7), collisions (Eq. 8, Eq. 15, Eq. 19) and pull streaming.
 *
 * Pins (tests/test_oracle_*.py): Gaussian diffusion, advected Gaussian,
 * Taylor-Green decay, Poiseuille profile, planar tanh interface (isotropic
 * and tilted anisotropic width), uniform-state recurrences of the phase field
 * and of the drag, conservation of sum(U + phi_lag) and of mass, fixed
 * points, k-fold symmetry, translation invariance, anisotropy-flux identity,
 * normal orientation, and the axis-vs-diagonal growth habit.
 */
#ifndef LBPF_ORACLE_H
#define LBPF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PERIODIC = 0, ORC_INLET_OUTLET = 1, ORC_WALL = 2 };

typedef struct {
  int dim;            /* 2 or 3 */
  int nx, ny, nz;     /* nz = 1 in 2D */
  int bc[3];          /* per axis: ORC_PERIODIC, ORC_INLET_OUTLET (x only), ORC_WALL */
  int flow;           /* 0: phase field + solute only; 1: coupled flow lattice */
  int fold;           /* anisotropy fold k in 2D; 0 = cubic form (required in 3D) */
  int aniso_literal;  /* 1: use |grad phi|^2 d(a_s^2)/d(grad phi) literally (x2) */
  double tau_phi0;    /* tau_phi where a_s = 1 (Eq. 23) */
  double tau_u_liquid;/* tau_U in the liquid, phi = -1 (Eq. 18) */
  double tau_f;       /* flow relaxation time (Eq. 10) */
  double w0;          /* interface width W0 */
  double lambda;      /* coupling constant (Eq. 1, Eq. 20) */
  double eps;         /* anisotropy strength (Eq. 3) */
  double theta0;      /* anisotropy orientation */
  double h_drag;      /* drag constant h of Eq. 6 */
  double u_inlet;     /* inlet velocity along +x */
  double u0_inlet;    /* supersaturation of the inflow */
  double body[3];     /* constant body force (test cases only) */
  int collision;      /* flow collision: 0 BGK (Eq. 8), 1 central Hermite MRT */
  double omega_bulk;  /* CHM: rate of the trace of the second-order moments (0: 1) */
  double omega_high;  /* CHM: rate of the third- and fourth-order moments (0: 1) */
} orc_params;

typedef struct orc_sim orc_sim;

/* Derived constants: tau0 from tau_phi0 (Eq. 23 at a_s = 1) and the solute
 * diffusivity in the liquid (Eq. 18 at q = 1).  */
double orc_tau0(const orc_params* p);
/* Coupling constant: p->lambda if >= 0, else the thin-interface value
 * D tau0 / (a2 W0^2) with a2 = 0.6267. */
double orc_lambda(const orc_params* p);

orc_sim* orc_create(const orc_params* p);
void     orc_destroy(orc_sim* s);

/* Circular/spherical tanh seed plus SplitMix64 noise; every population at
 * its equilibrium (ghost-free initial state). */
void orc_init_seed(orc_sim* s, double cx, double cy, double cz, double radius,
                   double u0, double noise_amp, uint64_t seed);
/* Equilibrium populations from given macroscopic fields (length nx*ny*nz,
 * x fastest).  uz may be NULL in 2D. */
/* convex polygon seed (2D): facets with outward unit normals (nx, ny) at
 * distances d from the centre (cx, cy) */
void orc_init_polygon(orc_sim* s, double cx, double cy, int k, const double* nx,
                      const double* ny, const double* d, double u0, double noise_amp,
                      uint64_t seed);
/* Solid nodes (2D and 3D): mask[nodes] (x fastest), nonzero = solid; NULL
 * removes the mask.  Fluid nodes bounce back (half-way) what they send into a
 * solid node, for f, g and h; solid nodes keep their state; in the phi
 * gradient a solid node counts as the first fluid node among the single-axis
 * steps x + c_d e_d of its non-zero components (in the order x, y, z) and x
 * itself.  With an inlet/outlet along x the first and last columns must be
 * fluid.  Returns 0, or -1 (a solid inlet/outlet column). */
int orc_set_solid(orc_sim* s, const unsigned char* mask);
void orc_init_fields(orc_sim* s, const double* phi, const double* U, const double* rho,
                     const double* ux, const double* uy, const double* uz);

/* Advance n steps with nthreads OpenMP threads (1 = serial). */
void orc_step(orc_sim* s, int n, int nthreads);
long long orc_step_count(const orc_sim* s);

/* Macroscopic fields at the current time; any pointer may be NULL. */
void orc_fields(const orc_sim* s, double* phi, double* U, double* rho,
                double* ux, double* uy, double* uz);
/* phi at the previous time level. */
void orc_phi_prev(const orc_sim* s, double* out);
/* Populations, direction-major [q][node]; returns q of that lattice
 * (which: 0 = f, 1 = g, 2 = h).  out may be NULL to query q. */
int orc_pops(const orc_sim* s, int which, double* out);

/* Per-node a_s and grad phi of the current state (NULL allowed). */
void orc_aux(const orc_sim* s, double* a_s, double* gx, double* gy, double* gz);

/* a_s and the anisotropic flux vector N for a given gradient (Eq. 3, Eq. 21). */
void orc_aniso(const orc_params* p, const double grad[3], double* a_s, double n_vec[3]);

/* FP64 diagnostics: [0] sum(U + phi_prev), [1] sum(rho), [2] solid volume
 * sum((1+phihat)/2), [3] r_eq, [4] max|u|, [5] non-finite count,
 * [6..11] interface crossing distance along +x,-x,+y,-y,+z,-z from node
 * (icx, icy, icz). */
void orc_diag(const orc_sim* s, int icx, int icy, int icz, double out[12]);

#ifdef __cplusplus
}
#endif
#endif
