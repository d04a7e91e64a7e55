/*
 * FP64 CPU oracle of the coupled LB phase-field crystal-growth step.
 * TEST INFRASTRUCTURE ONLY: loaded by tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the product path.
 *
 * The method (Sec. 2.2 of the paper):
 *   flow lattice   f : stream-collide with BGK (Eq. 4, Eq. 8), second-order
 *                      Hermite equilibrium (Eq. 9) evaluated at the masked
 *                      velocity u* (Eq. 7), Guo forcing (Eq. 5) with the
 *                      solid drag of Eq. 6, moments Eqs. 11-12, tau_f Eq. 10;
 *   solute lattice g : stream-collide with BGK (Eq. 13, Eq. 15), equilibrium
 *                      Eq. 16, source Eq. 14, moment Eq. 17, tau_U(phi) Eq. 18;
 *   phase lattice  h : the modified scheme of Eq. 19 with source Eq. 20,
 *                      equilibrium Eq. 21, moment Eq. 22 and tau_phi Eq. 23;
 *   anisotropy        : Eq. 3, with n = -grad(phi)/|grad(phi)| (Sec. 2.1).
 *
 * Readings where the paper is silent or ambiguous (each is listed with its
 * reason in the design notes):
 *   - theta = atan2(n_y, n_x); a_s = 1 + eps cos(k (theta - theta0)); the 3D
 *     form is the cubic a_s = 1 - 3 eps + 4 eps sum n_i^4.
 *   - N = |grad phi|^2 a_s d(a_s)/d(grad phi) (half of the literal
 *     |grad phi|^2 d(a_s^2)/d(grad phi), the variational form); aniso_literal
 *     restores the literal factor.
 *   - a_s^2 and tau_phi of Eq. 19 are evaluated at the source node r.
 *   - q(phi) is normalised through tau_U in the liquid:
 *     tau_U = 1/2 + (tau_U,liq - 1/2) (1 - phihat)/2.
 *   - phihat = clamp(phi, -1, 1) inside q, the drag and the velocity mask
 *     only; Q and h^eq use the raw phi.
 *   - d(phi)/dt = phi(t) - phi(t-1) at the source node; 0 at the first step.
 *   - u* (Eq. 7) is used in f^eq, in g^eq and in the Guo term; the drag
 *     force uses the unmasked u.  F = -K u is linear in u, so the Guo
 *     half-force velocity is u = (m + b/2) / (rho + K/2) exactly.
 *   - grad phi = (1/cs^2) sum_a w_a c_a phi(x + c_a) over D2Q9 (2D) or
 *     D3Q19 (3D); |grad phi|^2 <= 1e-12 gives a_s = 1, N = 0.
 *   - D3Q7 for g and h in 3D: w = 1/4, 1/8; cs^2 = 1/4.
 *   - inlet ghost (x = -1): equilibrium at rho = 1, u = u_in e_x,
 *     U = U_inlet, phi = -1, a_s = 1; outlet ghost (x = nx): the post-collision
 *     state of node nx - 1; walls: half-way bounce-back for f, g and h;
 *     gradient ghosts copy the nearest node (zero normal derivative).
 */
#include "lbpf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int q;
  int c[19][3];
  double w[19];
  double cs2;
} lattice;

/* D2Q9: rest, 4 axis links, 4 diagonals (w = 4/9, 1/9, 1/36; cs^2 = 1/3). */
static void make_d2q9(lattice* L) {
  static const int c[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                              {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
  L->q = 9;
  for (int a = 0; a < 9; ++a) {
    L->c[a][0] = c[a][0];
    L->c[a][1] = c[a][1];
    L->c[a][2] = 0;
    int nn = abs(c[a][0]) + abs(c[a][1]);
    L->w[a] = nn == 0 ? 4.0 / 9.0 : (nn == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  L->cs2 = 1.0 / 3.0;
}

/* D3Q19: rest, 6 faces, 12 edges (w = 1/3, 1/18, 1/36; cs^2 = 1/3). */
static void make_d3q19(lattice* L) {
  static const int c[19][3] = {
      {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
      {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
      {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
      {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
  L->q = 19;
  for (int a = 0; a < 19; ++a) {
    int nn = 0;
    for (int d = 0; d < 3; ++d) {
      L->c[a][d] = c[a][d];
      nn += abs(c[a][d]);
    }
    L->w[a] = nn == 0 ? 1.0 / 3.0 : (nn == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  L->cs2 = 1.0 / 3.0;
}

/* D3Q7: rest and 6 faces (w = 1/4, 1/8; cs^2 = 1/4). */
static void make_d3q7(lattice* L) {
  static const int c[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                              {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
  L->q = 7;
  for (int a = 0; a < 7; ++a) {
    for (int d = 0; d < 3; ++d) L->c[a][d] = c[a][d];
    L->w[a] = a == 0 ? 0.25 : 0.125;
  }
  L->cs2 = 0.25;
}

static int opposite(const lattice* L, int a) {
  for (int b = 0; b < L->q; ++b)
    if (L->c[b][0] == -L->c[a][0] && L->c[b][1] == -L->c[a][1] &&
        L->c[b][2] == -L->c[a][2])
      return b;
  return -1;
}

struct orc_sim {
  orc_params p;
  lattice LF, LS, LG; /* flow, scalar (g and h), gradient stencil */
  int n;
  long long step;
  double tau0, lambda;
  double *f, *g, *h, *fn, *gn, *hn, *phi_prev;
  /* per-node quantities of the current time level */
  double *phi, *U, *rho, *u[3], *us[3], *F[3], *phihat, *K, *tauU, *dphidt;
  double *grad[3], *as, *a2, *tauphi, *N[3], *Q;
  unsigned char* solid; /* solid mask (1 = solid node), NULL = none */
  double* fpost;        /* central Hermite MRT: post-collision f of every node [q][n] */
};

static double* zalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

double orc_tau0(const orc_params* p) {
  /* Eq. 23 with a_s = 1: tau_phi0 = W0^2 / (cs^2 tau0) + 1/2. */
  double cs2 = p->dim == 3 ? 0.25 : 1.0 / 3.0;
  return p->w0 * p->w0 / (cs2 * (p->tau_phi0 - 0.5));
}

double orc_lambda(const orc_params* p) {
  if (p->lambda >= 0.0) return p->lambda;
  /* thin-interface default lambda = D tau0 / (a2 W0^2), a2 = 0.6267 */
  double cs2 = p->dim == 3 ? 0.25 : 1.0 / 3.0;
  double dliq = cs2 * (p->tau_u_liquid - 0.5);
  return dliq * orc_tau0(p) / (0.6267 * p->w0 * p->w0);
}

orc_sim* orc_create(const orc_params* p) {
  orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
  s->p = *p;
  if (p->dim == 2) {
    make_d2q9(&s->LF);
    make_d2q9(&s->LS);
    make_d2q9(&s->LG);
    s->p.nz = 1;
  } else {
    make_d3q19(&s->LF);
    make_d3q7(&s->LS);
    make_d3q19(&s->LG);
  }
  s->n = s->p.nx * s->p.ny * s->p.nz;
  s->tau0 = orc_tau0(&s->p);
  s->lambda = orc_lambda(&s->p);
  size_t n = (size_t)s->n;
  s->f = zalloc(n * s->LF.q);
  s->fn = zalloc(n * s->LF.q);
  s->g = zalloc(n * s->LS.q);
  s->gn = zalloc(n * s->LS.q);
  s->h = zalloc(n * s->LS.q);
  s->hn = zalloc(n * s->LS.q);
  s->phi_prev = zalloc(n);
  s->phi = zalloc(n);
  s->U = zalloc(n);
  s->rho = zalloc(n);
  for (int d = 0; d < 3; ++d) {
    s->u[d] = zalloc(n);
    s->us[d] = zalloc(n);
    s->F[d] = zalloc(n);
    s->grad[d] = zalloc(n);
    s->N[d] = zalloc(n);
  }
  s->phihat = zalloc(n);
  s->K = zalloc(n);
  s->tauU = zalloc(n);
  s->dphidt = zalloc(n);
  s->as = zalloc(n);
  s->a2 = zalloc(n);
  s->tauphi = zalloc(n);
  s->Q = zalloc(n);
  if (p->collision == 1) s->fpost = zalloc(n * s->LF.q);
  return s;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  free(s->f); free(s->fn); free(s->g); free(s->gn); free(s->h); free(s->hn);
  free(s->phi_prev); free(s->phi); free(s->U); free(s->rho);
  for (int d = 0; d < 3; ++d) {
    free(s->u[d]); free(s->us[d]); free(s->F[d]); free(s->grad[d]); free(s->N[d]);
  }
  free(s->phihat); free(s->K); free(s->tauU); free(s->dphidt);
  free(s->as); free(s->a2); free(s->tauphi); free(s->Q);
  free(s->solid);
  free(s->fpost);
  free(s);
}

long long orc_step_count(const orc_sim* s) { return s->step; }

int orc_set_solid(orc_sim* s, const unsigned char* mask) {
  if (!mask) {
    free(s->solid);
    s->solid = NULL;
    return 0;
  }
  if (s->p.bc[0] == ORC_INLET_OUTLET) { /* the inlet and outlet columns stay fluid */
    const int nz = s->p.dim == 3 ? s->p.nz : 1;
    for (int r = 0; r < s->p.ny * nz; ++r)
      if (mask[(size_t)r * s->p.nx] || mask[(size_t)r * s->p.nx + s->p.nx - 1]) return -1;
  }
  if (!s->solid) s->solid = (unsigned char*)malloc((size_t)s->n);
  for (int i = 0; i < s->n; ++i) s->solid[i] = mask[i] ? 1 : 0;
  return 0;
}

static double clamp1(double v) { return v < -1.0 ? -1.0 : (v > 1.0 ? 1.0 : v); }

/* ---- anisotropy: Eq. 3 and the flux vector of Eq. 21 ---------------------- */
void orc_aniso(const orc_params* p, const double gr[3], double* a_s, double nv[3]) {
  double g2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
  nv[0] = nv[1] = nv[2] = 0.0;
  if (g2 <= 1e-12 || p->eps == 0.0) {
    *a_s = 1.0;
    return;
  }
  double g = sqrt(g2);
  double n[3] = {-gr[0] / g, -gr[1] / g, -gr[2] / g}; /* normal, solid -> liquid */
  double fac = p->aniso_literal ? 2.0 : 1.0;
  if (p->fold > 0) {
    /* a_s = 1 + eps cos(k (theta - theta0)), theta = atan2(n_y, n_x);
     * d(theta)/d(grad) = (-g_y, g_x) / |grad|^2, so
     * N = |grad|^2 a_s d(a_s)/d(grad) = k eps a_s sin(k(theta-theta0)) (g_y, -g_x). */
    double k = (double)p->fold;
    double th = atan2(n[1], n[0]);
    double as = 1.0 + p->eps * cos(k * (th - p->theta0));
    double sn = sin(k * (th - p->theta0));
    *a_s = as;
    nv[0] = fac * k * p->eps * as * sn * gr[1];
    nv[1] = -fac * k * p->eps * as * sn * gr[0];
  } else {
    /* cubic: a_s = 1 - 3 eps + 4 eps S, S = sum n_i^4;
     * N_i = 16 eps a_s |grad| (n_i S - n_i^3). */
    double S = n[0] * n[0] * n[0] * n[0] + n[1] * n[1] * n[1] * n[1] +
               n[2] * n[2] * n[2] * n[2];
    double as = 1.0 - 3.0 * p->eps + 4.0 * p->eps * S;
    *a_s = as;
    for (int d = 0; d < 3; ++d)
      nv[d] = fac * 16.0 * p->eps * as * g * (n[d] * S - n[d] * n[d] * n[d]);
  }
}

/* ---- index helpers ------------------------------------------------------- */
static int dims(const orc_sim* s, int d) {
  return d == 0 ? s->p.nx : (d == 1 ? s->p.ny : s->p.nz);
}

/* neighbour for the gradient stencil: periodic wrap, otherwise clamp */
static int grad_neighbor(const orc_sim* s, const int x[3], const int c[3]) {
  int y[3];
  for (int d = 0; d < 3; ++d) {
    int n = dims(s, d);
    int v = x[d] + c[d];
    if (s->p.bc[d] == ORC_PERIODIC) {
      v = ((v % n) + n) % n;
    } else {
      v = v < 0 ? 0 : (v >= n ? n - 1 : v);
    }
    y[d] = v;
  }
  return (y[2] * s->p.ny + y[1]) * s->p.nx + y[0];
}

/* Gradient neighbour with solid nodes (walls and obstacles of Sec. 3.1.2):
 * a solid node in the stencil is replaced by the first fluid node among the
 * single-axis steps of c -- x + c_x e_x, x + c_y e_y, x + c_z e_z, those with
 * a non-zero component, in that order -- and x itself (each mapped like any
 * stencil neighbour).  For a straight wall this is the nearest-node copy of
 * the domain walls, a zero normal derivative. */
static int grad_neighbor_masked(const orc_sim* s, const int x[3], const int c[3]) {
  int j = grad_neighbor(s, x, c);
  if (!s->solid || !s->solid[j]) return j;
  for (int d = 0; d < 3; ++d) {
    if (c[d] == 0) continue;
    int cd[3] = {0, 0, 0};
    cd[d] = c[d];
    j = grad_neighbor(s, x, cd);
    if (!s->solid[j]) return j;
  }
  const int c0[3] = {0, 0, 0};
  return grad_neighbor(s, x, c0);
}

enum { SRC_NODE = 0, SRC_INLET = 1, SRC_BOUNCE = 2 };

/* Source of the population arriving at x along c (pull form s = x - c). */
static int stream_source(const orc_sim* s, const int x[3], const int c[3], int* sidx) {
  int y[3];
  int wall = 0, inlet = 0;
  for (int d = 0; d < 3; ++d) {
    int n = dims(s, d);
    int v = x[d] - c[d];
    if (v < 0 || v >= n) {
      if (s->p.bc[d] == ORC_PERIODIC) {
        v = ((v % n) + n) % n;
      } else if (s->p.bc[d] == ORC_WALL) {
        wall = 1;
      } else { /* inlet / outlet along x */
        if (v < 0)
          inlet = 1;
        else
          v = n - 1; /* outlet ghost copies the last node */
      }
    }
    y[d] = v;
  }
  if (wall) {
    *sidx = (x[2] * s->p.ny + x[1]) * s->p.nx + x[0];
    return SRC_BOUNCE;
  }
  if (inlet) {
    *sidx = -1;
    return SRC_INLET;
  }
  *sidx = (y[2] * s->p.ny + y[1]) * s->p.nx + y[0];
  if (s->solid && s->solid[*sidx]) { /* half-way bounce-back at a solid node */
    *sidx = (x[2] * s->p.ny + x[1]) * s->p.nx + x[0];
    return SRC_BOUNCE;
  }
  return SRC_NODE;
}

/* ---- per-node quantities of the current time level ------------------------ */
static void node_moments(orc_sim* s, int i) {
  const orc_params* p = &s->p;
  int n = s->n;
  double phi = 0.0, U = 0.0, rho = 1.0, m[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < s->LS.q; ++a) phi += s->h[(size_t)a * n + i]; /* Eq. 22 */
  for (int a = 0; a < s->LS.q; ++a) U += s->g[(size_t)a * n + i];   /* Eq. 17 */
  if (p->flow) {
    rho = 0.0;
    for (int a = 0; a < s->LF.q; ++a) {
      double fa = s->f[(size_t)a * n + i];
      rho += fa; /* Eq. 11 */
      for (int d = 0; d < 3; ++d) m[d] += s->LF.c[a][d] * fa; /* Eq. 12 */
    }
  }
  double ph = clamp1(phi);
  double K = 0.0;
  if (p->flow) /* Eq. 6: F = -K u, K = h tau_f (1+phi)^2 (1-phi) / (4 W0^2) */
    K = p->h_drag * p->tau_f * (1.0 + ph) * (1.0 + ph) * (1.0 - ph) / (4.0 * p->w0 * p->w0);
  s->phi[i] = phi;
  s->U[i] = U;
  s->rho[i] = rho;
  s->phihat[i] = ph;
  s->K[i] = K;
  for (int d = 0; d < 3; ++d) {
    double u = p->flow ? (m[d] + 0.5 * p->body[d]) / (rho + 0.5 * K) : 0.0;
    s->u[d][i] = u;
    s->F[d][i] = p->flow ? p->body[d] - K * u : 0.0;
    s->us[d][i] = 0.5 * (1.0 - ph) * u; /* Eq. 7 */
  }
  /* Eq. 18 with q normalised by the liquid value */
  s->tauU[i] = 0.5 + (p->tau_u_liquid - 0.5) * 0.5 * (1.0 - ph);
  s->dphidt[i] = phi - s->phi_prev[i];
}

static void node_gradient_terms(orc_sim* s, int i) {
  const orc_params* p = &s->p;
  int x[3] = {i % p->nx, (i / p->nx) % p->ny, i / (p->nx * p->ny)};
  double gr[3] = {0.0, 0.0, 0.0};
  for (int a = 1; a < s->LG.q; ++a) {
    int j = grad_neighbor_masked(s, x, s->LG.c[a]);
    for (int d = 0; d < 3; ++d) gr[d] += s->LG.w[a] * s->LG.c[a][d] * s->phi[j];
  }
  for (int d = 0; d < 3; ++d) gr[d] /= s->LG.cs2;
  double as, nv[3];
  orc_aniso(p, gr, &as, nv);
  for (int d = 0; d < 3; ++d) {
    s->grad[d][i] = gr[d];
    s->N[d][i] = nv[d];
  }
  s->as[i] = as;
  s->a2[i] = as * as;
  s->tauphi[i] = as * as * p->w0 * p->w0 / (s->LS.cs2 * s->tau0) + 0.5; /* Eq. 23 */
  double phi = s->phi[i];
  s->Q[i] = (phi - phi * phi * phi) +
            s->lambda * s->U[i] * (1.0 - phi * phi) * (1.0 - phi * phi); /* Eq. 20 */
}

/* ---- central Hermite multiple-relaxation-time collision of f -------------
 * The collision the paper uses for the flow (Sec. 2.2, after Eq. 9: a central
 * Hermite MRT, defined in the work it cites), in this reading:
 *   1. central Hermite moments of f about the velocity u* of the equilibrium,
 *      k_j = sum_a f_a P_j(c_a - u*), with the nine D2Q9 polynomials
 *      1, X, Y, X^2 - cs2, Y^2 - cs2, XY, X^2 Y - cs2 Y, X Y^2 - cs2 X,
 *      X^2 Y^2 - cs2 (X^2 + Y^2) + cs2^2, or the nineteen D3Q19 ones: the
 *      products H_i(X) H_j(Y) H_k(Z) of the Hermite polynomials H_0 = 1,
 *      H_1 = X, H_2 = X^2 - cs2 with i, j, k <= 2 and at most two of them
 *      non-zero (1; X, Y, Z; three H_2; XY, XZ, YZ; six H_2 H_1; three
 *      H_2 H_2);
 *   2. their equilibrium values: rho, then zeros (the moments of the
 *      Maxwellian about its own velocity; in 2D those of the product-form
 *      equilibrium);
 *   3. relaxation by order: the first-order moments at 1/tau_f (as BGK:
 *      momentum relaxes towards rho u*) with the force, (1 - w/2) F; the
 *      deviatoric second-order moments and the mixed ones (XY, ...) at
 *      1/tau_f (the viscosity, Eq. 10); their trace at omega_bulk (default
 *      1); third and fourth order at omega_high (default 1);
 *   4. back to populations: the solution of the q x q system
 *      sum_a P_j(c_a - u*) f*_a = k*_j. */
static void chm_poly(double X, double Y, double cs2, double P[9]) {
  P[0] = 1.0;
  P[1] = X;
  P[2] = Y;
  P[3] = X * X - cs2;
  P[4] = Y * Y - cs2;
  P[5] = X * Y;
  P[6] = X * X * Y - cs2 * Y;
  P[7] = X * Y * Y - cs2 * X;
  P[8] = X * X * Y * Y - cs2 * (X * X + Y * Y) + cs2 * cs2;
}

static double hermite(int k, double X, double cs2) {
  return k == 0 ? 1.0 : k == 1 ? X : X * X - cs2;
}

/* the D3Q19 polynomials, in the order: 1; X, Y, Z; H2(X), H2(Y), H2(Z); XY,
 * XZ, YZ; H2(X) Y, H2(X) Z, X H2(Y), H2(Y) Z, X H2(Z), Y H2(Z); H2(X) H2(Y),
 * H2(X) H2(Z), H2(Y) H2(Z) */
static void chm_poly3(double X, double Y, double Z, double cs2, double P[19]) {
  static const int e[19][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                               {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1},
                               {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {0, 2, 1}, {1, 0, 2},
                               {0, 1, 2}, {2, 2, 0}, {2, 0, 2}, {0, 2, 2}};
  for (int j = 0; j < 19; ++j)
    P[j] = hermite(e[j][0], X, cs2) * hermite(e[j][1], Y, cs2) * hermite(e[j][2], Z, cs2);
}

/* solve A x = b (n x n, row-major) by Gauss-Jordan elimination with partial
 * pivoting; A and b are overwritten, x = b on return */
static void solve_dense(double* A, double* b, int n) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < n; ++k) {
        double t = A[c * n + k];
        A[c * n + k] = A[piv * n + k];
        A[piv * n + k] = t;
      }
      double t = b[c];
      b[c] = b[piv];
      b[piv] = t;
    }
    double d = A[c * n + c];
    for (int k = 0; k < n; ++k) A[c * n + k] /= d;
    b[c] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double m = A[r * n + c];
      if (m == 0.0) continue;
      for (int k = 0; k < n; ++k) A[r * n + k] -= m * A[c * n + k];
      b[r] -= m * b[c];
    }
  }
}

static void chm_collide(orc_sim* s, int i) {
  const lattice* L = &s->LF;
  const int n = s->n, q = L->q, D = s->p.dim;
  const double cs2 = L->cs2;
  const double wf = 1.0 / s->p.tau_f;
  const double wb = s->p.omega_bulk > 0.0 ? s->p.omega_bulk : 1.0;
  const double wh = s->p.omega_high > 0.0 ? s->p.omega_high : 1.0;
  const double v[3] = {s->us[0][i], s->us[1][i], s->us[2][i]};
  double M[19 * 19], k[19];
  for (int j = 0; j < q; ++j) k[j] = 0.0;
  for (int a = 0; a < q; ++a) {
    double P[19];
    if (D == 2)
      chm_poly(L->c[a][0] - v[0], L->c[a][1] - v[1], cs2, P);
    else
      chm_poly3(L->c[a][0] - v[0], L->c[a][1] - v[1], L->c[a][2] - v[2], cs2, P);
    double fa = s->f[(size_t)a * n + i];
    for (int j = 0; j < q; ++j) {
      M[j * q + a] = P[j];
      k[j] += P[j] * fa;
    }
  }
  /* relaxation; equilibrium values: rho (k[0], conserved), zeros.  Moments
   * 1..D: first order; D+1..2D: the diagonal second order; then the mixed
   * second order (1 in 2D, 3 in 3D); the rest third and fourth order. */
  double ks[19];
  ks[0] = k[0];
  for (int d = 0; d < D; ++d) ks[1 + d] = (1.0 - wf) * k[1 + d] + (1.0 - 0.5 * wf) * s->F[d][i];
  double mean = 0.0;
  for (int d = 0; d < D; ++d) mean += k[1 + D + d];
  mean /= D;
  for (int d = 0; d < D; ++d)
    ks[1 + D + d] = (1.0 - wb) * mean + (1.0 - wf) * (k[1 + D + d] - mean);
  const int nmix = D == 2 ? 1 : 3;
  for (int j = 1 + 2 * D; j < 1 + 2 * D + nmix; ++j) ks[j] = (1.0 - wf) * k[j];
  for (int j = 1 + 2 * D + nmix; j < q; ++j) ks[j] = (1.0 - wh) * k[j];
  solve_dense(M, ks, q);
  for (int a = 0; a < q; ++a) s->fpost[(size_t)a * n + i] = ks[a];
}

/* ---- post-collision values at a node (Eqs. 4-9, 13-16, 19-21) ------------- */
static double f_post(const orc_sim* s, int i, int a) {
  if (s->fpost) return s->fpost[(size_t)a * s->n + i];
  const lattice* L = &s->LF;
  double cs2 = L->cs2, tf = s->p.tau_f;
  double cu = 0.0, cF = 0.0, uF = 0.0, uu = 0.0;
  for (int d = 0; d < 3; ++d) {
    cu += L->c[a][d] * s->us[d][i];
    cF += L->c[a][d] * s->F[d][i];
    uF += s->us[d][i] * s->F[d][i];
    uu += s->us[d][i] * s->us[d][i];
  }
  /* Eq. 9, second-order Hermite expansion */
  double feq = s->rho[i] * L->w[a] *
               (1.0 + cu / cs2 + (cu * cu - cs2 * uu) / (2.0 * cs2 * cs2));
  /* Eq. 5 (Guo) with (u F + F u):(c c - cs^2 I) = 2 (c.u)(c.F) - 2 cs^2 u.F */
  double G = L->w[a] * (1.0 - 0.5 / tf) *
             (cF / cs2 + (cu * cF - cs2 * uF) / (cs2 * cs2));
  double fa = s->f[(size_t)a * s->n + i];
  return fa - (fa - feq) / tf + G; /* Eq. 4, Eq. 8 */
}

static double g_post(const orc_sim* s, int i, int a) {
  const lattice* L = &s->LS;
  double cu = 0.0;
  for (int d = 0; d < 3; ++d) cu += L->c[a][d] * s->us[d][i];
  double geq = L->w[a] * s->U[i] * (1.0 + cu / L->cs2); /* Eq. 16 */
  double ga = s->g[(size_t)a * s->n + i];
  return ga - (ga - geq) / s->tauU[i] - L->w[a] * s->dphidt[i]; /* Eq. 13-15 */
}

static double h_post(const orc_sim* s, int i, int a) {
  const lattice* L = &s->LS;
  double cN = 0.0;
  for (int d = 0; d < 3; ++d) cN += L->c[a][d] * s->N[d][i];
  double heq = L->w[a] * (s->phi[i] - cN * s->p.w0 * s->p.w0 / (L->cs2 * s->tau0)); /* Eq. 21 */
  double ha = s->h[(size_t)a * s->n + i];
  return ha - (ha - heq) / s->tauphi[i] + L->w[a] * s->Q[i] / s->tau0; /* Eq. 19 */
}

/* inlet ghost: equilibrium at rho = 1, u = u_in e_x, U = U_inlet, phi = -1 */
static double f_inlet(const orc_sim* s, int a) {
  const lattice* L = &s->LF;
  double cs2 = L->cs2, u = s->p.u_inlet;
  double cu = L->c[a][0] * u;
  return L->w[a] * (1.0 + cu / cs2 + (cu * cu - cs2 * u * u) / (2.0 * cs2 * cs2));
}
static double g_inlet(const orc_sim* s, int a) {
  const lattice* L = &s->LS;
  double u = s->p.flow ? s->p.u_inlet : 0.0;
  return L->w[a] * s->p.u0_inlet * (1.0 + L->c[a][0] * u / L->cs2);
}
static double h_inlet(const orc_sim* s, int a) { return -s->LS.w[a]; }

static void update_node(orc_sim* s, int i) {
  const orc_params* p = &s->p;
  int n = s->n;
  if (s->solid && s->solid[i]) { /* solid nodes keep their state */
    for (int a = 0; a < s->LF.q && p->flow; ++a) s->fn[(size_t)a * n + i] = s->f[(size_t)a * n + i];
    for (int a = 0; a < s->LS.q; ++a) {
      s->gn[(size_t)a * n + i] = s->g[(size_t)a * n + i];
      s->hn[(size_t)a * n + i] = s->h[(size_t)a * n + i];
    }
    return;
  }
  int x[3] = {i % p->nx, (i / p->nx) % p->ny, i / (p->nx * p->ny)};
  int src;
  if (p->flow) {
    for (int a = 0; a < s->LF.q; ++a) {
      int kind = stream_source(s, x, s->LF.c[a], &src);
      double v;
      if (kind == SRC_NODE) v = f_post(s, src, a);
      else if (kind == SRC_INLET) v = f_inlet(s, a);
      else v = f_post(s, src, opposite(&s->LF, a));
      s->fn[(size_t)a * n + i] = v;
    }
  }
  for (int a = 0; a < s->LS.q; ++a) {
    int kind = stream_source(s, x, s->LS.c[a], &src);
    double gv, hv, a2;
    if (kind == SRC_NODE) {
      gv = g_post(s, src, a);
      hv = h_post(s, src, a);
      a2 = s->a2[src];
    } else if (kind == SRC_INLET) {
      gv = g_inlet(s, a);
      hv = h_inlet(s, a);
      a2 = 1.0;
    } else {
      int b = opposite(&s->LS, a);
      gv = g_post(s, src, b);
      hv = h_post(s, src, b);
      a2 = s->a2[src];
    }
    s->gn[(size_t)a * n + i] = gv;
    /* Eq. 19: a_s^2 h(x, t+1) = h*(r) - (1 - a_s^2) h(x, t), a_s at r */
    s->hn[(size_t)a * n + i] = (hv - (1.0 - a2) * s->h[(size_t)a * n + i]) / a2;
  }
}

static void compute_node_fields(orc_sim* s, int nthreads) {
  int n = s->n;
  (void)nthreads;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int i = 0; i < n; ++i) node_moments(s, i);
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int i = 0; i < n; ++i) node_gradient_terms(s, i);
  if (s->fpost && s->p.flow) {
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int i = 0; i < n; ++i) chm_collide(s, i);
  }
}

void orc_step(orc_sim* s, int nsteps, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  int n = s->n;
  for (int t = 0; t < nsteps; ++t) {
    compute_node_fields(s, nthreads);
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int i = 0; i < n; ++i) update_node(s, i);
    /* phi(t-1) <- phi(t); swap population buffers */
    memcpy(s->phi_prev, s->phi, sizeof(double) * (size_t)n);
    double* t0;
    t0 = s->f; s->f = s->fn; s->fn = t0;
    t0 = s->g; s->g = s->gn; s->gn = t0;
    t0 = s->h; s->h = s->hn; s->hn = t0;
    s->step++;
  }
}

/* ---- initial state ------------------------------------------------------- */
static void set_equilibrium(orc_sim* s, int i, double phi, double U, double rho,
                            const double u[3]) {
  const orc_params* p = &s->p;
  int n = s->n;
  double ph = clamp1(phi);
  double us[3];
  for (int d = 0; d < 3; ++d) us[d] = p->flow ? 0.5 * (1.0 - ph) * u[d] : 0.0;
  if (p->flow) {
    const lattice* L = &s->LF;
    double uu = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
    for (int a = 0; a < L->q; ++a) {
      double cu = L->c[a][0] * us[0] + L->c[a][1] * us[1] + L->c[a][2] * us[2];
      s->f[(size_t)a * n + i] =
          rho * L->w[a] * (1.0 + cu / L->cs2 + (cu * cu - L->cs2 * uu) / (2.0 * L->cs2 * L->cs2));
    }
  }
  const lattice* L = &s->LS;
  for (int a = 0; a < L->q; ++a) {
    double cu = L->c[a][0] * us[0] + L->c[a][1] * us[1] + L->c[a][2] * us[2];
    s->g[(size_t)a * n + i] = L->w[a] * U * (1.0 + cu / L->cs2);
    s->h[(size_t)a * n + i] = L->w[a] * phi; /* N = 0 at t = 0 */
  }
  s->phi_prev[i] = phi;
}

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the finaliser of a
 * Weyl sequence with increment 0x9E3779B97F4A7C15. */
static uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void orc_init_seed(orc_sim* s, double cx, double cy, double cz, double radius,
                   double u0, double noise_amp, uint64_t seed) {
  const orc_params* p = &s->p;
  for (int i = 0; i < s->n; ++i) {
    int x = i % p->nx, y = (i / p->nx) % p->ny, z = i / (p->nx * p->ny);
    double dx = x - cx, dy = y - cy, dz = p->dim == 3 ? z - cz : 0.0;
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    double phi = tanh((radius - r) / (sqrt(2.0) * p->w0));
    uint64_t bits = splitmix64(seed ^ ((uint64_t)i * 0x9E3779B97F4A7C15ull));
    double xi = (double)(bits >> 11) * (1.0 / 4503599627370496.0) - 1.0; /* [-1, 1) */
    phi += noise_amp * xi;
    double u[3] = {p->flow ? p->u_inlet : 0.0, 0.0, 0.0};
    set_equilibrium(s, i, phi, u0, 1.0, u);
  }
  s->step = 0;
}

/* Convex polygon seed, 2D (the rhombic and hexagonal seeds of Sec. 3.1):
 * the polygon is {x : (x - c).n_i <= d_i for every facet i}; the signed
 * distance to it is taken as s(x) = max_i [(x - c).n_i - d_i] (exact inside
 * and beside the sides, an underestimate only outside the corners) and
 * phi0 = tanh(-s / (sqrt(2) W0)), plus the noise of the round seed; U = u0,
 * rho = 1 and the inlet velocity as there. */
void orc_init_polygon(orc_sim* s, double cx, double cy, int k, const double* nx,
                      const double* ny, const double* d, double u0, double noise_amp,
                      uint64_t seed) {
  const orc_params* p = &s->p;
  for (int i = 0; i < s->n; ++i) {
    int x = i % p->nx, y = (i / p->nx) % p->ny;
    double sd = -1e300;
    for (int f = 0; f < k; ++f) {
      double v = (x - cx) * nx[f] + (y - cy) * ny[f] - d[f];
      if (v > sd) sd = v;
    }
    double phi = tanh(-sd / (sqrt(2.0) * p->w0));
    uint64_t bits = splitmix64(seed ^ ((uint64_t)i * 0x9E3779B97F4A7C15ull));
    double xi = (double)(bits >> 11) * (1.0 / 4503599627370496.0) - 1.0; /* [-1, 1) */
    phi += noise_amp * xi;
    double u[3] = {p->flow ? p->u_inlet : 0.0, 0.0, 0.0};
    set_equilibrium(s, i, phi, u0, 1.0, u);
  }
  s->step = 0;
}

void orc_init_fields(orc_sim* s, const double* phi, const double* U, const double* rho,
                     const double* ux, const double* uy, const double* uz) {
  for (int i = 0; i < s->n; ++i) {
    double u[3] = {ux ? ux[i] : 0.0, uy ? uy[i] : 0.0, uz ? uz[i] : 0.0};
    set_equilibrium(s, i, phi[i], U[i], rho ? rho[i] : 1.0, u);
  }
  s->step = 0;
}

/* ---- read-out ------------------------------------------------------------- */
void orc_fields(const orc_sim* s, double* phi, double* U, double* rho, double* ux,
                double* uy, double* uz) {
  orc_sim* m = (orc_sim*)s;
  for (int i = 0; i < s->n; ++i) node_moments(m, i);
  for (int i = 0; i < s->n; ++i) {
    if (phi) phi[i] = s->phi[i];
    if (U) U[i] = s->U[i];
    if (rho) rho[i] = s->rho[i];
    if (ux) ux[i] = s->u[0][i];
    if (uy) uy[i] = s->u[1][i];
    if (uz) uz[i] = s->u[2][i];
  }
}

void orc_phi_prev(const orc_sim* s, double* out) {
  memcpy(out, s->phi_prev, sizeof(double) * (size_t)s->n);
}

int orc_pops(const orc_sim* s, int which, double* out) {
  const double* src = which == 0 ? s->f : (which == 1 ? s->g : s->h);
  int q = which == 0 ? s->LF.q : s->LS.q;
  if (which == 0 && !s->p.flow) return 0;
  if (out) memcpy(out, src, sizeof(double) * (size_t)q * s->n);
  return q;
}

void orc_aux(const orc_sim* s, double* a_s, double* gx, double* gy, double* gz) {
  orc_sim* m = (orc_sim*)s;
  compute_node_fields(m, 1);
  for (int i = 0; i < s->n; ++i) {
    if (a_s) a_s[i] = s->as[i];
    if (gx) gx[i] = s->grad[0][i];
    if (gy) gy[i] = s->grad[1][i];
    if (gz) gz[i] = s->grad[2][i];
  }
}

static double crossing(const orc_sim* s, int ic[3], int axis, int dir) {
  int n = dims(s, axis);
  int x[3] = {ic[0], ic[1], ic[2]};
  int i0 = (x[2] * s->p.ny + x[1]) * s->p.nx + x[0];
  double prev = s->phi[i0];
  if (!(prev >= 0.0)) return -1.0;
  int limit = s->p.bc[axis] == ORC_PERIODIC ? n / 2 : n;
  for (int d = 1; d < limit; ++d) {
    int v = ic[axis] + dir * d;
    if (s->p.bc[axis] == ORC_PERIODIC) v = ((v % n) + n) % n;
    else if (v < 0 || v >= n) break;
    x[axis] = v;
    double cur = s->phi[(x[2] * s->p.ny + x[1]) * s->p.nx + x[0]];
    if (cur < 0.0) return (double)(d - 1) + prev / (prev - cur);
    prev = cur;
  }
  return -1.0;
}

void orc_diag(const orc_sim* s, int icx, int icy, int icz, double out[12]) {
  orc_sim* m = (orc_sim*)s;
  for (int i = 0; i < s->n; ++i) node_moments(m, i);
  double I = 0.0, M = 0.0, A = 0.0, umax = 0.0, bad = 0.0;
  for (int i = 0; i < s->n; ++i) {
    I += s->U[i] + s->phi_prev[i];
    M += s->rho[i];
    A += 0.5 * (1.0 + s->phihat[i]);
    double uu = s->u[0][i] * s->u[0][i] + s->u[1][i] * s->u[1][i] + s->u[2][i] * s->u[2][i];
    if (sqrt(uu) > umax) umax = sqrt(uu);
    if (!isfinite(s->phi[i]) || !isfinite(s->U[i]) || !isfinite(s->rho[i])) bad += 1.0;
  }
  out[0] = I;
  out[1] = M;
  out[2] = A;
  out[3] = s->p.dim == 3 ? cbrt(3.0 * A / (4.0 * M_PI)) : sqrt(A / M_PI);
  out[4] = umax;
  out[5] = bad;
  int ic[3] = {icx, icy, s->p.dim == 3 ? icz : 0};
  out[6] = crossing(s, ic, 0, +1);
  out[7] = crossing(s, ic, 0, -1);
  out[8] = crossing(s, ic, 1, +1);
  out[9] = crossing(s, ic, 1, -1);
  out[10] = s->p.dim == 3 ? crossing(s, ic, 2, +1) : -1.0;
  out[11] = s->p.dim == 3 ? crossing(s, ic, 2, -1) : -1.0;
}
