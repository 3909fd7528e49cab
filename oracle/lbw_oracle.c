/*
 * lbw_oracle.c -- plain FP64 CPU oracle of the curvilinear wave lattice-Boltzmann step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py may load this file's library.  It shares no code, header,
 * table or constant with the CUDA path in paper_1705_01801_gb300/csrc; the two meet only in
 * the seeded inputs (grid sizes, pulses, probe nodes) that the tests hand to both.
 *
 * Method: Velasco, Munoz, Mendoza, "Lattice Boltzmann model for the simulation of the wave
 * equation in curvilinear coordinates" (arXiv:1705.01801).  One time step, per node, in the
 * paper's order (Sec. III "LBM for waves in generalized coordinates", the "Summarizing"
 * paragraph):
 *   1. streaming of the post-collision populations along xi_i (Eq. eq:evolution, delta_t = 1),
 *      pull form, with the boundary rules of Sec. IV.A (periodic, bounce-back with damping D,
 *      free = copy of the normal neighbour) plus anti-bounce-back for Dirichlet P = 0;
 *   2. rho = sqrt(g) P = sum_i f_i (Eq. PressureCurvedSystem);
 *   3. forcing term F^a = -c^2 rho G^a - d_b A^{ab},  A^{ab} = rho (c^2 g^{ab} - cs^2 delta^{ab})
 *      (Eqs. 2ConservationcurvedForce, JCorrectionForce; reading of sign and cs^2 below),
 *      with d_b taken by the lattice-weighted stencil of Eq. DerivativeFromTaylor / App. B,
 *      which for D3Q7 is the central difference (1/2)[A(x+e_b) - A(x-e_b)];
 *   4. sqrt(g) J'^a = sum_i f_i xi_i^a + F^a / 2 (Eq. JCorrectionForce, Eq. JShifted);
 *   5. f_i^eq = w_i [rho + xi_i . (sqrt(g) J') / cs^2], f_0^eq = w_0 rho
 *      (Eq. EquilibriumCurvedSystemHermiteCorrected);
 *   6. BGK relaxation with tau = 1/2 (Sec. II, Eq. SecondOrder; App. A): f* = 2 f^eq - f.
 *
 * Readings where the paper is silent, garbled or inconsistent (each pinned by a test):
 *   R1 sign/cs^2 of the moved term: the recovered momentum law needs lattice stress cs^2 rho
 *      plus force to equal d_b(c^2 rho g^{ab}) + c^2 rho G^a, so the divergence enters with a
 *      minus sign and with cs^2 (not c^2) in the delta term.  Pinned by the flat-space wave
 *      speed test (c != cs).
 *   R2 the Christoffel term carries sqrt(g) (Eq. 2ConservationcurvedForce): -c^2 rho G^a.
 *      Pinned by the annulus Bessel frequencies; the trumpet's assembled metric terms by the
 *      axial modes of Bessel and exponential horns against Webster's horn equation.
 *   R3 D3Q7 weights (the figure is missing): w_0 = 1 - 3 cs^2, w_i = cs^2 / 2, cs^2 a parameter.
 *   R4 neighbour rho for the gradient is taken at the same time level (after streaming).
 *      Pinned by second-order convergence, in flat space and on an annular cylinder mode (a
 *      one-step lag would make the scheme first order).
 *   R5 ghost values for the gradient at a non-periodic face: free -> rho copied; bounce-back
 *      (rigid) -> P mirrored (even); anti-bounce-back (Dirichlet) -> P mirrored with a sign
 *      change (odd); the ghost's metric is evaluated at the ghost position.  Walls are pinned
 *      by the annulus, closed-pipe and horn modes.  The free (copy) face is pinned by the
 *      open-closed pipe of Sec. IV.A: a channel closed by a wall and ended by a free face has
 *      the quarter-wave modes (2n+1) pi c / (2 L_e), L - 1 < L_e <= L (L - 1/2 at c = cs),
 *      in flat space and on a cylinder's q3 face.  The damping D of the bounce-back rule is
 *      pinned by the impedance reflection coefficient (c - beta) / (c + beta),
 *      beta = cs^2 (1 - D) / (1 + D), that the rule implies for the wave equation.
 *   R6 the metric is written in lattice coordinates q: x^a = x0^a + (q^a + 1/2) h^a, so
 *      g_q^{ab} = g^{ab} / (h_a h_b), sqrt(g_q) = h1 h2 h3 sqrt(g), G_q^a = G^a / h_a.
 *   R7 initial state at rest: J'(0) = 0 (Eq. JShifted), so the stored post-collision
 *      populations are f^eq(rho0, +F(rho0)/2).  Pinned by the finite-difference test (the
 *      naive f^eq(rho0, 0) start leaves an O(dt) velocity error: first-order convergence).
 *   R8 harmonic sources (the paper imposes P, or J'_z for the plate, at source nodes): after
 *      each step the source nodes' populations become the equilibrium carrying the imposed
 *      value (apply_sources).  Pinned by the radiated cylindrical wave of a ring source
 *      matching the radial Bessel equation's solutions, and by the plate's plane waves: a
 *      dipole (opposite signs either side, speed c), amplitude C / (cs^2 + c) at c = cs from
 *      the equilibrium of a running wave, uniform across a pipe (the sqrt(g) factor).
 *   Also corrected from the printed formulas (verified symbolically): trumpet
 *   Gamma^theta_{z theta} = lambda / Zc (printed lambda / Zc^2) and torus
 *   Gamma^r_{theta theta} = -(R + r cos phi) cos phi (printed with +); the contracted
 *   symbols G^a = g^{bc} Gamma^a_{bc} used here are G^a = -(1/sqrt g) d_b (sqrt g g^{ab}).
 *
 * Layout: f[i][q3][q1][q2] (q2 fastest).  Velocities: 0 rest, 1 +e1, 2 -e1, 3 +e2, 4 -e2,
 * 5 +e3, 6 -e3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KIND_CARTESIAN 0
#define KIND_POLAR 1
#define KIND_CYLINDRICAL 2
#define KIND_TRUMPET 3
#define KIND_TOROIDAL 4

#define FACE_PERIODIC 0
#define FACE_BOUNCE 1
#define FACE_ANTIBOUNCE 2
#define FACE_FREE 3

#define EQ_CURVILINEAR 0
#define EQ_MOMENT_MATCHING 1
#define EQ_HERMITE 2

typedef struct {
  int kind, profile, eq;
  int n[3];
  int bc[6];
  double h[3], x0[3];
  double c, cs2, damping;
  double gp[4];
  long long nn;
  double *f, *fnew, *fpull, *rho;
  /* probes */
  int nprobe;
  long long *probe_node;
  long long cap, nrec;
  double *series; /* [nprobe][cap] */
  /* harmonic sources (reading R8 below) */
  int nsrc, src_kind;
  long long *src_node;
  double src_amp, src_omega;
  long long t; /* time steps since lbwo_init */
} OGrid;

static const int XI[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                             {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static const int OPP[7] = {0, 2, 1, 4, 3, 6, 5};

/* ---- geometry in physical coordinates (u1, u2, u3) ------------------------------------ */

/* Flare profile s(z) of the horn x = r s(z) cos(theta), y = r s(z) sin(theta).
 * profile 0: Bessel horn s = Zc^{-lambda}, Zc = Zmax - z (Sec. IV.B, Eq. coordinatesTrumpet);
 * profile 1: exponential flare s = (a0 + b e^{alpha z}) / (a0 + b). */
static void flare(const OGrid *g, double z, double *s, double *ds, double *dds) {
  if (g->profile == 0) {
    double Zmax = g->gp[0], lam = g->gp[1];
    double Zc = Zmax - z;
    *s = pow(Zc, -lam);
    *ds = lam * pow(Zc, -lam - 1.0);
    *dds = lam * (lam + 1.0) * pow(Zc, -lam - 2.0);
  } else {
    double a0 = g->gp[0], b = g->gp[1], al = g->gp[2];
    double e = exp(al * z), A = a0 + b;
    *s = (a0 + b * e) / A;
    *ds = b * al * e / A;
    *dds = b * al * al * e / A;
  }
}

/* sqrt(g), contravariant metric g^{ab} and contracted Christoffel symbols G^a in physical
 * coordinates.  Cylinder: Eqs. MetricCylindrical, CylindricalChr.  Trumpet: Eqs.
 * coordinatesTrumpet, MetricTrumpet, ChristoffelTrumpet (general flare s(z)).  Torus: Eqs.
 * CoordinatesTorus, AMetricTorus, AChristoffelTorus. */
static void geom_phys(const OGrid *g, double u1, double u2, double u3, double *sqrtg,
                      double ginv[3][3], double G[3]) {
  (void)u2;
  memset(ginv, 0, 9 * sizeof(double));
  G[0] = G[1] = G[2] = 0.0;
  if (g->kind == KIND_CARTESIAN) {
    *sqrtg = 1.0;
    ginv[0][0] = ginv[1][1] = ginv[2][2] = 1.0;
  } else if (g->kind == KIND_POLAR || g->kind == KIND_CYLINDRICAL) {
    double r = u1;
    *sqrtg = r;
    ginv[0][0] = 1.0;
    ginv[1][1] = 1.0 / (r * r);
    ginv[2][2] = 1.0;
    /* G^r = g^{theta theta} Gamma^r_{theta theta} = (1/r^2)(-r) */
    G[0] = -1.0 / r;
  } else if (g->kind == KIND_TRUMPET) {
    double r = u1, s, ds, dds;
    flare(g, u3, &s, &ds, &dds);
    *sqrtg = r * s * s;
    ginv[0][0] = (1.0 + r * r * ds * ds) / (s * s);
    ginv[0][2] = ginv[2][0] = -r * ds / s;
    ginv[1][1] = 1.0 / (r * r * s * s);
    ginv[2][2] = 1.0;
    G[0] = (r * r * s * dds - 2.0 * r * r * ds * ds - 1.0) / (r * s * s);
  } else { /* torus: u1 = r, u2 = theta (major), u3 = phi (minor) */
    double R = g->gp[0], r = u1, phi = u3;
    double Rr = R + r * cos(phi);
    *sqrtg = r * Rr;
    ginv[0][0] = 1.0;
    ginv[1][1] = 1.0 / (Rr * Rr);
    ginv[2][2] = 1.0 / (r * r);
    G[0] = -(R + 2.0 * r * cos(phi)) / (r * Rr);
    G[2] = sin(phi) / (r * Rr);
  }
}

/* Physical embedding X(u) in R^3 (used only to place Gaussian pulses). */
static void embed(const OGrid *g, double u1, double u2, double u3, double X[3]) {
  if (g->kind == KIND_CARTESIAN) {
    X[0] = u1; X[1] = u2; X[2] = u3;
  } else if (g->kind == KIND_POLAR || g->kind == KIND_CYLINDRICAL) {
    X[0] = u1 * cos(u2); X[1] = u1 * sin(u2); X[2] = u3;
  } else if (g->kind == KIND_TRUMPET) {
    double s, ds, dds;
    flare(g, u3, &s, &ds, &dds);
    X[0] = u1 * s * cos(u2); X[1] = u1 * s * sin(u2); X[2] = u3;
  } else {
    double R = g->gp[0];
    X[0] = (R + u1 * cos(u3)) * cos(u2);
    X[1] = (R + u1 * cos(u3)) * sin(u2);
    X[2] = u1 * sin(u3);
  }
}

/* Geometry in lattice coordinates at integer position q (may be one cell outside: ghost).
 * Reading R6: x^a = x0^a + (q^a + 1/2) h^a. */
static void geom_q(const OGrid *g, int q1, int q2, int q3, double *sqrtg, double ginv[3][3],
                   double G[3]) {
  double u1 = g->x0[0] + (q1 + 0.5) * g->h[0];
  double u2 = g->x0[1] + (q2 + 0.5) * g->h[1];
  double u3 = g->x0[2] + (q3 + 0.5) * g->h[2];
  double sg, gi[3][3], Gp[3];
  geom_phys(g, u1, u2, u3, &sg, gi, Gp);
  *sqrtg = sg * g->h[0] * g->h[1] * g->h[2];
  for (int a = 0; a < 3; a++) {
    for (int b = 0; b < 3; b++) ginv[a][b] = gi[a][b] / (g->h[a] * g->h[b]);
    G[a] = Gp[a] / g->h[a];
  }
}

static long long nid(const OGrid *g, int q1, int q2, int q3) {
  return ((long long)q3 * g->n[0] + q1) * g->n[1] + q2;
}

/* ---- public (ctypes) interface ------------------------------------------------------- */

/* ints: kind, n1, n2, n3, bc[6], profile, equilibrium   (12 values)
 * dbls: h[3], x0[3], c, cs2, damping, gp[4] (13 values) */
void *lbwo_create(const int32_t *ints, const double *dbls) {
  OGrid *g = (OGrid *)calloc(1, sizeof(OGrid));
  g->kind = ints[0];
  for (int a = 0; a < 3; a++) g->n[a] = ints[1 + a];
  for (int k = 0; k < 6; k++) g->bc[k] = ints[4 + k];
  g->profile = ints[10];
  g->eq = ints[11];
  for (int a = 0; a < 3; a++) {
    g->h[a] = dbls[a];
    g->x0[a] = dbls[3 + a];
  }
  g->c = dbls[6];
  g->cs2 = dbls[7];
  g->damping = dbls[8];
  for (int k = 0; k < 4; k++) g->gp[k] = dbls[9 + k];
  g->nn = (long long)g->n[0] * g->n[1] * g->n[2];
  g->f = (double *)calloc(7 * g->nn, sizeof(double));
  g->fnew = (double *)calloc(7 * g->nn, sizeof(double));
  g->fpull = (double *)calloc(7 * g->nn, sizeof(double));
  g->rho = (double *)calloc(g->nn, sizeof(double));
  return g;
}

void lbwo_destroy(void *p) {
  OGrid *g = (OGrid *)p;
  if (!g) return;
  free(g->f); free(g->fnew); free(g->fpull); free(g->rho);
  free(g->probe_node); free(g->series); free(g->src_node);
  free(g);
}

/* Geometry query for tests: out = sqrtg, g^{11}, g^{22}, g^{33}, g^{12}, g^{13}, g^{23},
 * G^1, G^2, G^3, all in physical coordinates. */
void lbwo_geometry(void *p, double u1, double u2, double u3, double *out) {
  OGrid *g = (OGrid *)p;
  double sg, gi[3][3], G[3];
  geom_phys(g, u1, u2, u3, &sg, gi, G);
  out[0] = sg;
  out[1] = gi[0][0]; out[2] = gi[1][1]; out[3] = gi[2][2];
  out[4] = gi[0][1]; out[5] = gi[0][2]; out[6] = gi[1][2];
  out[7] = G[0]; out[8] = G[1]; out[9] = G[2];
}

void lbwo_embed(void *p, double u1, double u2, double u3, double *X) {
  embed((OGrid *)p, u1, u2, u3, X);
}

/* Step 1: pull streaming with the face rules.  Returns f_i at node q after streaming. */
static double pulled(const OGrid *g, int i, const int q[3]) {
  int src[3] = {q[0] - XI[i][0], q[1] - XI[i][1], q[2] - XI[i][2]};
  int out_axis = -1, face = -1;
  for (int a = 0; a < 3; a++) {
    if (src[a] < 0) { out_axis = a; face = 2 * a; }
    if (src[a] >= g->n[a]) { out_axis = a; face = 2 * a + 1; }
  }
  long long x = nid(g, q[0], q[1], q[2]);
  if (out_axis < 0) return g->f[i * g->nn + nid(g, src[0], src[1], src[2])];
  switch (g->bc[face]) {
    case FACE_PERIODIC:
      src[out_axis] = (src[out_axis] + g->n[out_axis]) % g->n[out_axis];
      return g->f[i * g->nn + nid(g, src[0], src[1], src[2])];
    case FACE_BOUNCE: /* Sec. IV.A: f_out = D f_in, halfway bounce-back */
      return g->damping * g->f[OPP[i] * g->nn + x];
    case FACE_ANTIBOUNCE: /* Dirichlet P = 0 at the wall */
      return -g->f[OPP[i] * g->nn + x];
    default: /* FACE_FREE: ghost holds a copy of the boundary node (Sec. IV.A) */
      return g->f[i * g->nn + x];
  }
}

/* rho at the neighbour x + s e_b, with reading R5 at a non-periodic face.  Also returns the
 * lattice position used for the neighbour's metric (ghost position when outside). */
static double rho_neighbour(const OGrid *g, const int q[3], int b, int s, int pos[3]) {
  pos[0] = q[0]; pos[1] = q[1]; pos[2] = q[2];
  pos[b] += s;
  if (pos[b] >= 0 && pos[b] < g->n[b]) return g->rho[nid(g, pos[0], pos[1], pos[2])];
  int face = 2 * b + (s > 0 ? 1 : 0);
  if (g->bc[face] == FACE_PERIODIC) {
    pos[b] = (pos[b] + g->n[b]) % g->n[b];
    return g->rho[nid(g, pos[0], pos[1], pos[2])];
  }
  double rho_x = g->rho[nid(g, q[0], q[1], q[2])];
  if (g->bc[face] == FACE_FREE) return rho_x;
  double sg_x, sg_gh, gi[3][3], G[3];
  geom_q(g, q[0], q[1], q[2], &sg_x, gi, G);
  geom_q(g, pos[0], pos[1], pos[2], &sg_gh, gi, G);
  double sign = (g->bc[face] == FACE_BOUNCE) ? 1.0 : -1.0;
  return sign * (rho_x / sg_x) * sg_gh; /* P mirrored (even or odd), times ghost sqrt(g) */
}

/* Steps 3: F^a = -c^2 rho G^a - sum_b (1/2)[A^{ab}(x + e_b) - A^{ab}(x - e_b)],
 * A^{ab} = rho (c^2 g^{ab} - cs^2 delta^{ab}), with g->rho holding rho at the current time
 * level (reading R4) and G the node's contracted Christoffel symbols in lattice units. */
static void force(const OGrid *g, const int q[3], double rho, const double G[3], double F[3]) {
  const double c2 = g->c * g->c, cs2 = g->cs2;
  double divA[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < 3; b++)
    for (int s = -1; s <= 1; s += 2) {
      int pos[3];
      double rn = rho_neighbour(g, q, b, s, pos);
      double sgn, gin[3][3], Gn[3];
      geom_q(g, pos[0], pos[1], pos[2], &sgn, gin, Gn);
      for (int a = 0; a < 3; a++) {
        double A = rn * (c2 * gin[a][b] - (a == b ? cs2 : 0.0));
        divA[a] += 0.5 * s * A;
      }
    }
  for (int a = 0; a < 3; a++) F[a] = -c2 * rho * G[a] - divA[a];
}

/* The Cartesian schemes that Sec. II compares (flat space, lattice units, no forcing term),
 * with P = sum_i f_i and J = sum_i f_i xi_i (Eq. MacroscopicQuantities):
 *   moment matching (Chopard, Eq. feqMomentMatchingCartesian):
 *     f_0 = P + (c^2 / cs^2) P (w_0 - 1),  f_i = (w_i / cs^2)(c^2 P + xi_i . J);
 *   Hermite (Eq. EquilibriumHermite, discretised from the Gaussian of Eq. continuousfeq):
 *     f_i = w_i [P + xi_i . J / cs^2 + P (c^2 - cs^2)(|xi_i|^2 - 3 cs^2) / (2 cs^4)],
 *     f_0 = P - sum_{i >= 1} f_i (the paper's own rule for the rest population). */
static void cartesian_feq(const OGrid *g, double P, const double J[3], double feq[7]) {
  const double cs2 = g->cs2, c2 = g->c * g->c, w0 = 1.0 - 3.0 * cs2, w1 = 0.5 * cs2;
  if (g->eq == EQ_MOMENT_MATCHING) {
    feq[0] = P + (c2 / cs2) * P * (w0 - 1.0);
    for (int i = 1; i < 7; i++) {
      double xj = XI[i][0] * J[0] + XI[i][1] * J[1] + XI[i][2] * J[2];
      feq[i] = (w1 / cs2) * (c2 * P + xj);
    }
  } else {
    double rest = P;
    for (int i = 1; i < 7; i++) {
      double xj = XI[i][0] * J[0] + XI[i][1] * J[1] + XI[i][2] * J[2];
      double xi2 = (double)(XI[i][0] * XI[i][0] + XI[i][1] * XI[i][1] + XI[i][2] * XI[i][2]);
      feq[i] = w1 * (P + xj / cs2 + P * (c2 - cs2) * (xi2 - 3.0 * cs2) / (2.0 * cs2 * cs2));
      rest -= feq[i];
    }
    feq[0] = rest;
  }
}

static void record_probes(OGrid *g) {
  if (g->nprobe <= 0 || g->nrec >= g->cap) return;
  for (int k = 0; k < g->nprobe; k++) {
    long long x = g->probe_node[k];
    int q2 = (int)(x % g->n[1]);
    int q1 = (int)((x / g->n[1]) % g->n[0]);
    int q3 = (int)(x / ((long long)g->n[1] * g->n[0]));
    double sg, gi[3][3], G[3];
    geom_q(g, q1, q2, q3, &sg, gi, G);
    g->series[(long long)k * g->cap + g->nrec] = g->rho[x] / sg; /* P = rho / sqrt(g) */
  }
  g->nrec++;
}

/* Reading R8 (harmonic sources, Sec. IV: the ring, plate and point sources that impose
 * P = C sin(omega t), or J'_z = C sin(omega t) for the plate, at their nodes): at the end of
 * time step t (t = 1, 2, ... since lbwo_init) the post-collision populations of every source
 * node are replaced by an equilibrium carrying the imposed value.
 *   kind 0 (P source):   f*_i = f_i^eq(rho_s, j' = 0),  rho_s = sqrt(g) C sin(omega t);
 *   kind 1 (J'_z source): f*_i = f_i^eq(rho, j' = (0, 0, sqrt(g) C sin(omega t))), rho = sum f*_i
 *                         of the node (kept); the component is along q3. */
static void apply_sources(OGrid *g, double *f) {
  const double cs2 = g->cs2, w0 = 1.0 - 3.0 * cs2, w1 = 0.5 * cs2;
  const double v = g->src_amp * sin(g->src_omega * (double)g->t);
  for (int k = 0; k < g->nsrc; k++) {
    long long x = g->src_node[k];
    int q2 = (int)(x % g->n[1]);
    int q1 = (int)((x / g->n[1]) % g->n[0]);
    int q3 = (int)(x / ((long long)g->n[1] * g->n[0]));
    double sg, gi[3][3], G[3];
    geom_q(g, q1, q2, q3, &sg, gi, G);
    double rho, j3;
    if (g->src_kind == 0) {
      rho = sg * v;
      j3 = 0.0;
    } else {
      rho = 0.0;
      for (int i = 0; i < 7; i++) rho += f[i * g->nn + x];
      j3 = sg * v;
    }
    if (g->eq != EQ_CURVILINEAR) { /* the scheme's own equilibrium carries the imposed value */
      const double J[3] = {0.0, 0.0, j3};
      double feq[7];
      cartesian_feq(g, rho, J, feq);
      for (int i = 0; i < 7; i++) f[i * g->nn + x] = feq[i];
      continue;
    }
    for (int i = 0; i < 7; i++)
      f[i * g->nn + x] = (i == 0) ? w0 * rho : w1 * (rho + XI[i][2] * j3 / cs2);
  }
}

static void one_step(OGrid *g) {
  const double cs2 = g->cs2;
  const double w0 = 1.0 - 3.0 * cs2, w1 = 0.5 * cs2;
  /* 1 + 2: stream, then rho = sum_i f_i at every node */
#pragma omp parallel for schedule(static)
  for (int q3 = 0; q3 < g->n[2]; q3++)
    for (int q1 = 0; q1 < g->n[0]; q1++)
      for (int q2 = 0; q2 < g->n[1]; q2++) {
        int q[3] = {q1, q2, q3};
        long long x = nid(g, q1, q2, q3);
        double r = 0.0;
        for (int i = 0; i < 7; i++) {
          double fi = pulled(g, i, q);
          g->fpull[i * g->nn + x] = fi;
          r += fi;
        }
        g->rho[x] = r;
      }
  record_probes(g);
  /* 3..6: force, shifted momentum, equilibrium, relaxation */
#pragma omp parallel for schedule(static)
  for (int q3 = 0; q3 < g->n[2]; q3++)
    for (int q1 = 0; q1 < g->n[0]; q1++)
      for (int q2 = 0; q2 < g->n[1]; q2++) {
        int q[3] = {q1, q2, q3};
        long long x = nid(g, q1, q2, q3);
        double f[7];
        for (int i = 0; i < 7; i++) f[i] = g->fpull[i * g->nn + x];
        double rho = g->rho[x];
        double m[3] = {f[1] - f[2], f[3] - f[4], f[5] - f[6]};
        if (g->eq != EQ_CURVILINEAR) { /* Sec. II schemes: P = rho, J = m, no forcing term */
          double feq[7];
          cartesian_feq(g, rho, m, feq);
          for (int i = 0; i < 7; i++) g->fnew[i * g->nn + x] = 2.0 * feq[i] - f[i];
          continue;
        }
        double sg, gi[3][3], G[3];
        geom_q(g, q1, q2, q3, &sg, gi, G);
        double F[3];
        force(g, q, rho, G, F);
        double jp[3];
        for (int a = 0; a < 3; a++) jp[a] = m[a] + 0.5 * F[a];
        for (int i = 0; i < 7; i++) {
          double xj = XI[i][0] * jp[0] + XI[i][1] * jp[1] + XI[i][2] * jp[2];
          double feq = (i == 0) ? w0 * rho : w1 * (rho + xj / cs2);
          g->fnew[i * g->nn + x] = 2.0 * feq - f[i];
        }
      }
  g->t++;
  apply_sources(g, g->fnew);
  double *t = g->f;
  g->f = g->fnew;
  g->fnew = t;
}

/* Reading R7: the run starts at rest, J'(0) = 0 in the sense of Eq. JShifted
 * (J' = J + F/2).  The pre-collision populations at t = 0 are then f^eq(rho0, m = -F/2) and
 * the relaxation (tau = 1/2) turns them into f*_i = 2 f_i^eq(rho0, J' = 0) - f_i =
 * f_i^eq(rho0, +F(rho0)/2), which is the state stored here; F(rho0) is the forcing term of
 * the initial field.  rho0 = sqrt(g) P0, P0 a sum of Gaussians in the embedding distance.
 * pulses: n x {X, Y, Z, sigma, amp}. */
void lbwo_init(void *p, const double *pulses, int npulse) {
  OGrid *g = (OGrid *)p;
  double w0 = 1.0 - 3.0 * g->cs2, w1 = 0.5 * g->cs2;
  for (int q3 = 0; q3 < g->n[2]; q3++)
    for (int q1 = 0; q1 < g->n[0]; q1++)
      for (int q2 = 0; q2 < g->n[1]; q2++) {
        double u1 = g->x0[0] + (q1 + 0.5) * g->h[0];
        double u2 = g->x0[1] + (q2 + 0.5) * g->h[1];
        double u3 = g->x0[2] + (q3 + 0.5) * g->h[2];
        double X[3];
        embed(g, u1, u2, u3, X);
        double P0 = 0.0;
        for (int k = 0; k < npulse; k++) {
          const double *pk = pulses + 5 * k;
          double d2 = (X[0] - pk[0]) * (X[0] - pk[0]) + (X[1] - pk[1]) * (X[1] - pk[1]) +
                      (X[2] - pk[2]) * (X[2] - pk[2]);
          P0 += pk[4] * exp(-d2 / (2.0 * pk[3] * pk[3]));
        }
        double sg, gi[3][3], G[3];
        geom_q(g, q1, q2, q3, &sg, gi, G);
        g->rho[nid(g, q1, q2, q3)] = sg * P0;
      }
  for (int q3 = 0; q3 < g->n[2]; q3++)
    for (int q1 = 0; q1 < g->n[0]; q1++)
      for (int q2 = 0; q2 < g->n[1]; q2++) {
        int q[3] = {q1, q2, q3};
        long long x = nid(g, q1, q2, q3);
        double sg, gi[3][3], G[3], F[3];
        double rho0 = g->rho[x];
        if (g->eq != EQ_CURVILINEAR) { /* at rest: J = 0, no forcing term */
          const double J0[3] = {0.0, 0.0, 0.0};
          double feq[7];
          cartesian_feq(g, rho0, J0, feq);
          for (int i = 0; i < 7; i++) g->f[i * g->nn + x] = feq[i];
          continue;
        }
        geom_q(g, q1, q2, q3, &sg, gi, G);
        force(g, q, rho0, G, F);
        for (int i = 0; i < 7; i++) {
          double xj = 0.5 * (XI[i][0] * F[0] + XI[i][1] * F[1] + XI[i][2] * F[2]);
          g->f[i * g->nn + x] = (i == 0) ? w0 * rho0 : w1 * (rho0 + xj / g->cs2);
        }
      }
  g->nrec = 0;
  g->t = 0;
}

/* Harmonic sources at n lattice nodes (q1, q2, q3); kind 0 = P source, 1 = J'_z source
 * (reading R8).  n = 0 removes them. */
void lbwo_set_sources(void *p, const int32_t *q, int n, int kind, double amp, double omega) {
  OGrid *g = (OGrid *)p;
  free(g->src_node);
  g->nsrc = n;
  g->src_kind = kind;
  g->src_amp = amp;
  g->src_omega = omega;
  g->src_node = (long long *)malloc((n > 0 ? n : 1) * sizeof(long long));
  for (int k = 0; k < n; k++) g->src_node[k] = nid(g, q[3 * k], q[3 * k + 1], q[3 * k + 2]);
}

void lbwo_step(void *p, long long nsteps) {
  OGrid *g = (OGrid *)p;
  for (long long s = 0; s < nsteps; s++) one_step(g);
}

/* Probe nodes as lattice triples (q1, q2, q3); the series restarts. */
void lbwo_set_probes(void *p, const int32_t *q, int n, long long cap) {
  OGrid *g = (OGrid *)p;
  free(g->probe_node);
  free(g->series);
  g->nprobe = n;
  g->cap = cap;
  g->nrec = 0;
  g->probe_node = (long long *)malloc((n > 0 ? n : 1) * sizeof(long long));
  g->series = (double *)calloc((size_t)(n > 0 ? n : 1) * (cap > 0 ? cap : 1), sizeof(double));
  for (int k = 0; k < n; k++) g->probe_node[k] = nid(g, q[3 * k], q[3 * k + 1], q[3 * k + 2]);
}

long long lbwo_read_probes(void *p, double *out) {
  OGrid *g = (OGrid *)p;
  memcpy(out, g->series, sizeof(double) * (size_t)g->nprobe * g->cap);
  return g->nrec;
}

void lbwo_get_f(void *p, double *out) {
  OGrid *g = (OGrid *)p;
  memcpy(out, g->f, sizeof(double) * 7 * g->nn);
}

void lbwo_set_f(void *p, const double *in) {
  OGrid *g = (OGrid *)p;
  memcpy(g->f, in, sizeof(double) * 7 * g->nn);
}

/* P = rho / sqrt(g) of the current state (rho = sum of post-collision populations, which
 * the relaxation leaves unchanged). */
void lbwo_get_P(void *p, double *out) {
  OGrid *g = (OGrid *)p;
  for (int q3 = 0; q3 < g->n[2]; q3++)
    for (int q1 = 0; q1 < g->n[0]; q1++)
      for (int q2 = 0; q2 < g->n[1]; q2++) {
        long long x = nid(g, q1, q2, q3);
        double r = 0.0;
        for (int i = 0; i < 7; i++) r += g->f[i * g->nn + x];
        double sg, gi[3][3], G[3];
        geom_q(g, q1, q2, q3, &sg, gi, G);
        out[x] = r / sg;
      }
}
