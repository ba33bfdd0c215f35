/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the colour-gradient (CG) and Shan-Chen (SC)
 * lattice Boltzmann steps of arXiv 2110.05197.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the benchmark's CPU
 * baseline leg, never by the product library.  Shares no code with the CUDA path.
 *
 * Each step is written as the paper states it, in the paper's order, one plain loop per
 * stage over all nodes (no blocking, no fusion):
 *   CG (Sec. 2.2, Eqs. threeops..tensorG; repulsion Sec. 2.3, Eqs. repForce..normal2):
 *     1 densities rho_R, rho_B (Eq. density) and colour field rho^N
 *     2 gradients of rho^N, rho_R, rho_B
 *     3 repulsion force (when Pi != 0) + body force
 *     4 per node: velocity (Eq. totalMomentum2, shifted by F/2rho as in Eq. guoforce),
 *       interface viscosity (Eq. interpVisc) and omega_eff (Eq. effRelax), BGK towards the
 *       enhanced equilibrium (Eq. BGK, equiliCG, phi, tensorG), Guo source on the total,
 *       perturbation (Eq. perturbationOp), recolouring (Eqs. recoloringOpR/B, cosphi)
 *     5 streaming (Eq. streaming) with periodic wrap and halfway bounce-back on solid nodes
 *   SC multiphase (Sec. 2.1): rho (Eq. densitySC), psi (Eq. pseudopotential), force
 *     (Eq. interactionforceMP), shifted velocity (Eq. guoforce2), BGK + source (Eqs.
 *     collisSC, equiliSC, source), streaming (Eq. streamingSC).
 *   SC two-component: cross force of Eq. doublebeltrepulsionforce2 between the two
 *     species, common velocity, per-species BGK + source.
 *   SC multicomponent with multirange potentials (Eq. benziforces): per species the
 *     attractive belt-1 force (Eq. doublebeltattractiveforce), the repulsive belt-1 + belt-2
 *     force with the weights p of Eq. pweights (Eq. doublebeltrepulsionforce) and the
 *     cross force of Eq. doublebeltrepulsionforce2; then as the two-component model.
 *
 * Readings where the paper is silent, garbled or ambiguous (stated once here):
 *   - Perturbation: applied as A/2 |grad rho^N| [w_i (c_i.grad rho^N)^2/|grad rho^N|^2 - B_i]
 *     per colour, i.e. A |grad rho^N| [..] on the total (the printed "|rho^N| -" form
 *     breaks mass conservation).
 *   - phi_i^k (Eq. phi) is used in the BGK equilibrium too (with phi=0 the BGK step would
 *     not conserve mass); f^eq|_{u=0} in the recolouring is sum_k rho_k phi_i^k.
 *   - Both colours relax with the local omega_eff; nu_k = (tau_k - 1/2)/3.
 *   - Gradients: isotropic finite difference grad phi = 3 sum_i w_i phi(x+c_i) c_i, summed
 *     as opposite-pair differences.
 *   - Forces enter CG through Guo forcing with tau = 1/omega_eff, on the total population.
 *   - Walls: halfway bounce-back; a solid neighbour's scalar is replaced by the centre's.
 *   - psi_rep defaults to (1-|rho^N|)^chi (maximal at rho^N = 0, decaying away from it);
 *     H(0) = 0; direction 0 is skipped; a node or neighbour with |grad rho^N| <= eps adds 0.
 *   - Repulsion sign: the printed sum of Eq. repForce points, at the two nodes flanking a
 *     rho^N extremum, toward the extremum (for either orientation of the normals, the
 *     terms are quadratic in them), which squeezes the film between two interfaces and
 *     drains it; the text calls the force outward (repulsive), so F_rep is minus that sum.
 *   - Two-component SC: common barycentric velocity, each species relaxes with its own tau.
 *   - D2Q9 constants (the paper prints D3Q19 only) are chosen to satisfy the same moment
 *     identities as the D3Q19 set.
 *   - Multirange SC: belt 1 of the attractive and cross forces is the lattice's own 18
 *     neighbours with the weights w_i (D3Q19 has no (1,1,1) vectors, whose w would be 0);
 *     the repulsive force runs over all 92 non-zero vectors with |c|^2 <= 8 (belts 1 and 2)
 *     with p; Psi_s = rho_0 (1 - exp(-rho_s / rho_0)) as Eq. pseudopotential, per species.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int d, q;
  int c[19][3];
  double w[19], B[19], psi[19], xi[19];
  int grp[19]; /* 0 rest, 1 axis, 2 diagonal */
  int opp[19];
} lattice_t;

static void lattice_fill(int lattice, lattice_t* L) {
  memset(L, 0, sizeof *L);
  if (lattice == ORC_D3Q19) {
    /* Eq. speeds and Eq. weights; B_i, psi_i, xi_i as listed after Eqs. perturbationOp
     * and phi (0-based: rest, axis 1-6, diagonal 7-18). */
    static const int c3[19][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                  {0, 0, 1},   {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                  {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    L->d = 3;
    L->q = 19;
    memcpy(L->c, c3, sizeof c3);
    for (int i = 0; i < 19; i++) {
      int g = (i == 0) ? 0 : (i <= 6 ? 1 : 2);
      L->grp[i] = g;
      L->w[i] = (g == 0) ? 1.0 / 3.0 : (g == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
      L->B[i] = (g == 0) ? -2.0 / 9.0 : (g == 1 ? 1.0 / 54.0 : 1.0 / 27.0);
      L->psi[i] = (g == 0) ? -5.0 / 2.0 : (g == 1 ? -1.0 / 6.0 : 1.0 / 24.0);
      L->xi[i] = (g == 0) ? 0.0 : (g == 1 ? 1.0 / 4.0 : 1.0 / 8.0);
    }
  } else {
    static const int c2[9][3] = {{0, 0, 0}, {1, 0, 0},  {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
    L->d = 2;
    L->q = 9;
    memcpy(L->c, c2, sizeof c2);
    for (int i = 0; i < 9; i++) {
      int g = (i == 0) ? 0 : (i <= 4 ? 1 : 2);
      L->grp[i] = g;
      L->w[i] = (g == 0) ? 4.0 / 9.0 : (g == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
      L->B[i] = (g == 0) ? -4.0 / 27.0 : (g == 1 ? 2.0 / 27.0 : 5.0 / 108.0);
      L->psi[i] = (g == 0) ? -8.0 / 3.0 : (g == 1 ? -1.0 / 6.0 : 1.0 / 12.0);
      L->xi[i] = (g == 0) ? 0.0 : (g == 1 ? 1.0 / 2.0 : 1.0 / 8.0);
    }
  }
  for (int i = 0; i < L->q; i++) {
    for (int j = 0; j < L->q; j++) {
      if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
        L->opp[i] = j;
    }
  }
}

/* Eq. phi (D3Q19); the D2Q9 analogue has c_s^2 = 3(1-alpha)/5. */
static void phi_fill(int lattice, double alpha, double* phi) {
  lattice_t L;
  lattice_fill(lattice, &L);
  for (int i = 0; i < L.q; i++) {
    if (lattice == ORC_D3Q19)
      phi[i] = (L.grp[i] == 0) ? alpha : (L.grp[i] == 1 ? (1.0 - alpha) / 12.0 : (1.0 - alpha) / 24.0);
    else
      phi[i] = (L.grp[i] == 0) ? alpha : (L.grp[i] == 1 ? (1.0 - alpha) / 5.0 : (1.0 - alpha) / 20.0);
  }
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double cdot(const lattice_t* L, int i, const double* v) {
  return L->c[i][0] * v[0] + L->c[i][1] * v[1] + L->c[i][2] * v[2];
}
static double cnorm(const lattice_t* L, int i) {
  return sqrt((double)(L->c[i][0] * L->c[i][0] + L->c[i][1] * L->c[i][1] + L->c[i][2] * L->c[i][2]));
}

/* ------------------------------------------------------------------------------------ */
/* per-node building blocks                                                              */
/* ------------------------------------------------------------------------------------ */

/* Eq. equiliCG with Eq. tensorG: nubar [psi_i (u.grad rho_k) + xi_i (G_k : c_i c_i)]
 *   + rho_k (phi_i^k + w_i [3 c.u + 9/2 (c.u)^2 - 3/2 u.u]).  enhanced == 0 drops the
 * nubar[...] part (the standard CG equilibrium). */
static void cg_feq(const lattice_t* L, const double* phi, double rho_k, const double* u,
                   const double* grad_k, double nubar, int enhanced, double* feq) {
  double Gt[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) Gt[a][b] = u[a] * grad_k[b] + u[b] * grad_k[a];
  double ugrad = dot3(u, grad_k);
  double uu = dot3(u, u);
  for (int i = 0; i < L->q; i++) {
    double GCC = 0.0;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) GCC += Gt[a][b] * L->c[i][a] * L->c[i][b];
    double cu = cdot(L, i, u);
    double enh = enhanced ? nubar * (L->psi[i] * ugrad + L->xi[i] * GCC) : 0.0;
    feq[i] = enh + rho_k * (phi[i] + L->w[i] * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
  }
}

/* Eq. equiliSC with c = 1. */
static void sc_feq(const lattice_t* L, double rho, const double* u, double* feq) {
  double uu = dot3(u, u);
  for (int i = 0; i < L->q; i++) {
    double cu = cdot(L, i, u);
    feq[i] = rho * L->w[i] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
  }
}

/* Eq. source with c_s^2 = 1/3 and 1/tau = omega. */
static void guo_source(const lattice_t* L, const double* u, const double* F, double omega, double* S) {
  double cs2 = 1.0 / 3.0;
  for (int i = 0; i < L->q; i++) {
    double cmu[3] = {L->c[i][0] - u[0], L->c[i][1] - u[1], L->c[i][2] - u[2]};
    double cu = cdot(L, i, u);
    double cF = cdot(L, i, F);
    S[i] = L->w[i] * (1.0 - 0.5 * omega) * (dot3(cmu, F) / cs2 + cu * cF / (cs2 * cs2));
  }
}

/* Eq. perturbationOp (reading: A/2 |grad rho^N| [..] per colour, so A |grad rho^N| [..]
 * on the total population). */
static void perturbation(const lattice_t* L, const double* g, double A, double eps, double* d) {
  double gg = dot3(g, g);
  double gn = sqrt(gg);
  for (int i = 0; i < L->q; i++) {
    if (!(gn > eps)) {
      d[i] = 0.0;
      continue;
    }
    double cg = cdot(L, i, g);
    d[i] = 2.0 * (A / 2.0) * gn * (L->w[i] * cg * cg / gg - L->B[i]);
  }
}

/* Eqs. recoloringOpR/B with Eq. cosphi; f^eq|_{u=0} = sum_k rho_k phi_i^k. */
static void recolor(const lattice_t* L, const double* fstar, double rr, double rb, const double* phiR,
                    const double* phiB, const double* g, double beta, double eps, double* fr, double* fb) {
  double rho = rr + rb;
  double gn = sqrt(dot3(g, g));
  for (int i = 0; i < L->q; i++) {
    double cosphi = 0.0;
    if (i != 0 && gn > eps) cosphi = cdot(L, i, g) / (cnorm(L, i) * gn);
    double feq0 = rr * phiR[i] + rb * phiB[i];
    fr[i] = rr / rho * fstar[i] + beta * (rr * rb / (rho * rho)) * cosphi * feq0;
    fb[i] = rb / rho * fstar[i] - beta * (rr * rb / (rho * rho)) * cosphi * feq0;
  }
}

/* ------------------------------------------------------------------------------------ */
/* simulation state                                                                     */
/* ------------------------------------------------------------------------------------ */

struct orc_sim {
  orc_params p;
  lattice_t L;
  size_t n;
  int ncomp;
  double alpha_r, alpha_b;
  double phiR[19], phiB[19];
  double *f, *fpost;
  uint8_t* solid;
  double *rho_r, *rho_b, *color, *gN, *gR, *gB, *F, *psi, *psi2;  /* gN: 2nd species force for SC */
};

static int g_threads = 0;
void orc_set_threads(int n) {
  g_threads = n;
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#endif
}
int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static size_t node_of(const orc_sim* s, long x, long y, long z) {
  long nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  x = ((x % nx) + nx) % nx;
  y = ((y % ny) + ny) % ny;
  z = ((z % nz) + nz) % nz;
  return (size_t)(x + nx * (y + ny * z));
}
static void coords(const orc_sim* s, size_t n, long* x, long* y, long* z) {
  *x = (long)(n % (size_t)s->p.nx);
  *y = (long)((n / (size_t)s->p.nx) % (size_t)s->p.ny);
  *z = (long)(n / ((size_t)s->p.nx * (size_t)s->p.ny));
}
static size_t neighbour(const orc_sim* s, size_t n, int i) {
  long x, y, z;
  coords(s, n, &x, &y, &z);
  return node_of(s, x + s->L.c[i][0], y + s->L.c[i][1], z + s->L.c[i][2]);
}
static double* fp(const orc_sim* s, double* base, int k, int i) { return base + ((size_t)k * s->L.q + i) * s->n; }

orc_sim* orc_create(const orc_params* p) {
  if (!p || p->nx <= 0 || p->ny <= 0 || p->nz <= 0) return NULL;
  if (p->lattice != ORC_D2Q9 && p->lattice != ORC_D3Q19) return NULL;
  if (p->lattice == ORC_D2Q9 && p->nz != 1) return NULL;
  if (p->model == ORC_SC_MR && p->lattice != ORC_D3Q19) return NULL;
  orc_sim* s = (orc_sim*)calloc(1, sizeof *s);
  s->p = *p;
  lattice_fill(p->lattice, &s->L);
  s->n = (size_t)p->nx * p->ny * p->nz;
  s->ncomp = (p->model == ORC_SC_MP) ? 1 : 2;
  /* Eq. gamma: rho_R0/rho_B0 = (1-alpha_B)/(1-alpha_R). */
  s->alpha_b = p->alpha_b;
  s->alpha_r = 1.0 - (1.0 - p->alpha_b) * p->rho_b0 / p->rho_r0;
  phi_fill(p->lattice, s->alpha_r, s->phiR);
  phi_fill(p->lattice, s->alpha_b, s->phiB);
  size_t nf = (size_t)s->ncomp * s->L.q * s->n;
  s->f = (double*)calloc(nf, sizeof(double));
  s->fpost = (double*)calloc(nf, sizeof(double));
  s->solid = (uint8_t*)calloc(s->n, 1);
  s->rho_r = (double*)calloc(s->n, sizeof(double));
  s->rho_b = (double*)calloc(s->n, sizeof(double));
  s->color = (double*)calloc(s->n, sizeof(double));
  s->psi = (double*)calloc(s->n, sizeof(double));
  s->psi2 = (double*)calloc(s->n, sizeof(double));
  s->gN = (double*)calloc(3 * s->n, sizeof(double));
  s->gR = (double*)calloc(3 * s->n, sizeof(double));
  s->gB = (double*)calloc(3 * s->n, sizeof(double));
  s->F = (double*)calloc(3 * s->n, sizeof(double));
  return s;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  free(s->f);
  free(s->fpost);
  free(s->solid);
  free(s->rho_r);
  free(s->rho_b);
  free(s->color);
  free(s->psi);
  free(s->psi2);
  free(s->gN);
  free(s->gR);
  free(s->gB);
  free(s->F);
  free(s);
}

/* grad phi(x) = 3 sum_i w_i phi(x + c_i) c_i, summed over opposite pairs as
 * 3 w_i (phi(x + c_i) - phi(x - c_i)) c_i so that a field constant along a lattice direction
 * gives an exactly zero component (the Heaviside factor of Eq. repForce is then decided on
 * exact zeros, not rounding residues); a solid neighbour contributes phi(x). */
static void gradient(const orc_sim* s, const double* phi, size_t n, double* g) {
  g[0] = g[1] = g[2] = 0.0;
  for (int i = 1; i < s->L.q; i++) {
    int j = s->L.opp[i];
    if (j < i) continue;
    size_t mp = neighbour(s, n, i), mm = neighbour(s, n, j);
    double vp = s->solid[mp] ? phi[n] : phi[mp];
    double vm = s->solid[mm] ? phi[n] : phi[mm];
    for (int a = 0; a < 3; a++) g[a] += 3.0 * s->L.w[i] * (vp - vm) * s->L.c[i][a];
  }
}

/* Stage 1 (CG and SC): per-colour densities, Eq. density / densitySC. */
static void stage_densities(orc_sim* s) {
  const int Q = s->L.q;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < (long)s->n; n++) {
    double r = 0.0, b = 0.0;
    for (int i = 0; i < Q; i++) r += fp(s, s->f, 0, i)[n];
    if (s->ncomp == 2)
      for (int i = 0; i < Q; i++) b += fp(s, s->f, 1, i)[n];
    s->rho_r[n] = r;
    s->rho_b[n] = b;
  }
}

/* Colour field rho^N (text after Eq. perturbationOp). */
static void stage_color(orc_sim* s) {
#pragma omp parallel for schedule(static)
  for (long n = 0; n < (long)s->n; n++) {
    double r = s->rho_r[n], b = s->rho_b[n];
    if (s->p.color_norm) {
      r = r / s->p.rho_r0;
      b = b / s->p.rho_b0;
    }
    s->color[n] = (r - b) / (r + b);
  }
}

static void stage_cg_gradients(orc_sim* s) {
#pragma omp parallel for schedule(static)
  for (long n = 0; n < (long)s->n; n++) {
    gradient(s, s->color, (size_t)n, s->gN + 3 * n);
    gradient(s, s->rho_r, (size_t)n, s->gR + 3 * n);
    gradient(s, s->rho_b, (size_t)n, s->gB + 3 * n);
  }
}

/* Eq. repForce with Eqs. potential, normal1, normal2 (reading: see file header). */
static void repulsion_at(const orc_sim* s, size_t n, double* Fr) {
  Fr[0] = Fr[1] = Fr[2] = 0.0;
  const double* g = s->gN + 3 * n;
  double gn = sqrt(dot3(g, g));
  if (!(gn > s->p.grad_eps)) return;
  double nrm[3] = {g[0] / gn, g[1] / gn, g[2] / gn};
  double a = fabs(s->color[n]);
  double base = (s->p.rep_psi_kind == 1) ? (1.0 + a) : (1.0 - a);
  double psi_rep = pow(base, s->p.rep_chi);
  double acc[3] = {0.0, 0.0, 0.0};
  for (int i = 1; i < s->L.q; i++) {
    size_t m = neighbour(s, n, i);
    if (s->solid[m]) continue;
    const double* g2 = s->gN + 3 * m;
    double gn2 = sqrt(dot3(g2, g2));
    if (!(gn2 > s->p.grad_eps)) continue;
    double n2[3] = {g2[0] / gn2, g2[1] / gn2, g2[2] / gn2};
    double nc = cdot(&s->L, i, nrm);
    double n2c = cdot(&s->L, i, n2);
    double H = (-(nc * n2c) > 0.0) ? 1.0 : 0.0;
    double cl = cnorm(&s->L, i);
    for (int d = 0; d < 3; d++) acc[d] += H * (nc * nrm[d] / cl + n2c * n2[d] / cl);
  }
  /* outward: the sum points from the film's edge nodes toward the rho^N extremum between
     two interfaces; the force is the repulsive (outward) one of Sec. 2.3, its negative */
  for (int d = 0; d < 3; d++) Fr[d] = -s->p.rep_pi * psi_rep * acc[d];
}

static void stage_cg_force(orc_sim* s) {
#pragma omp parallel for schedule(static)
  for (long n = 0; n < (long)s->n; n++) {
    double Fr[3] = {0.0, 0.0, 0.0};
    if (s->p.rep_pi != 0.0 && !s->solid[n]) repulsion_at(s, (size_t)n, Fr);
    for (int d = 0; d < 3; d++) s->F[3 * n + d] = s->p.body_force[d] + Fr[d];
  }
}

/* Eq. interpVisc, Eq. effRelax with nu_k = (tau_k - 1/2)/3. */
static void interface_viscosity(const orc_sim* s, double rr, double rb, double* nubar, double* omega) {
  double rho = rr + rb;
  double nu_r = (s->p.tau_r - 0.5) / 3.0, nu_b = (s->p.tau_b - 0.5) / 3.0;
  double inv = (rr / rho) / nu_r + (rb / rho) / nu_b;
  *nubar = 1.0 / inv;
  *omega = 2.0 / (6.0 * (*nubar) + 1.0);
}

static void momentum_at(const orc_sim* s, size_t n, double* j) {
  j[0] = j[1] = j[2] = 0.0;
  for (int k = 0; k < s->ncomp; k++)
    for (int i = 0; i < s->L.q; i++) {
      double v = fp(s, s->f, k, i)[n];
      for (int a = 0; a < 3; a++) j[a] += v * s->L.c[i][a];
    }
}

/* Stage 4 (CG): Eqs. BGK, perturbation, recoloring for one node. */
static void cg_collide_node(orc_sim* s, size_t n) {
  const lattice_t* L = &s->L;
  const int Q = L->q;
  double rr = s->rho_r[n], rb = s->rho_b[n], rho = rr + rb;
  const double* F = s->F + 3 * n;
  double j[3], u[3];
  momentum_at(s, n, j);
  for (int a = 0; a < 3; a++) u[a] = (j[a] + 0.5 * F[a]) / rho;
  double nubar, omega;
  interface_viscosity(s, rr, rb, &nubar, &omega);
  double feqR[19], feqB[19], fstar[19], S[19], dP[19], fr[19], fb[19];
  cg_feq(L, s->phiR, rr, u, s->gR + 3 * n, nubar, s->p.enhanced_eq, feqR);
  cg_feq(L, s->phiB, rb, u, s->gB + 3 * n, nubar, s->p.enhanced_eq, feqB);
  for (int i = 0; i < Q; i++) {
    double fRi = fp(s, s->f, 0, i)[n], fBi = fp(s, s->f, 1, i)[n];
    double fRs = fRi - omega * (fRi - feqR[i]);
    double fBs = fBi - omega * (fBi - feqB[i]);
    fstar[i] = fRs + fBs;
  }
  guo_source(L, u, F, omega, S);
  for (int i = 0; i < Q; i++) fstar[i] += S[i];
  perturbation(L, s->gN + 3 * n, s->p.A, s->p.grad_eps, dP);
  for (int i = 0; i < Q; i++) fstar[i] += dP[i];
  recolor(L, fstar, rr, rb, s->phiR, s->phiB, s->gN + 3 * n, s->p.beta, s->p.grad_eps, fr, fb);
  for (int i = 0; i < Q; i++) {
    fp(s, s->fpost, 0, i)[n] = fr[i];
    fp(s, s->fpost, 1, i)[n] = fb[i];
  }
}

/* Stage 5: Eq. streaming; halfway bounce-back returns a population aimed at a solid node
 * to its source node in the opposite direction. */
static void stage_stream(orc_sim* s) {
  const int Q = s->L.q;
  size_t nf = (size_t)s->ncomp * Q * s->n;
  memset(s->f, 0, nf * sizeof(double));
  for (int k = 0; k < s->ncomp; k++)
    for (int i = 0; i < Q; i++) {
      const double* src = fp(s, s->fpost, k, i);
#pragma omp parallel for schedule(static)
      for (long n = 0; n < (long)s->n; n++) {
        if (s->solid[n]) continue;
        size_t m = neighbour(s, (size_t)n, i);
        if (s->solid[m])
          fp(s, s->f, k, s->L.opp[i])[n] = src[n];
        else
          fp(s, s->f, k, i)[m] = src[n];
      }
    }
}

/* Eq. pseudopotential. */
static double sc_psi(double rho, double rho0) { return rho0 * (1.0 - exp(-rho / rho0)); }

/* Belts 1 and 2 (Eq. pweights): every integer vector with |c|^2 <= 8, ordered by |c|^2
 * (rest first), and its weight p, which depends only on |c|^2. */
static int mr_table(int c[93][3], double p[93]) {
  int m = 0;
  for (int r2 = 0; r2 <= 8; r2++) {
    double w;
    switch (r2) {
      case 0: w = 0.0; break;
      case 1: w = 4.0 / 135.0; break;
      case 2: w = 1.0 / 63.0; break;
      case 3: w = 2.0 / 315.0; break;
      case 4: w = 5.0 / 1512.0; break;
      case 5: w = 1.0 / 945.0; break;
      case 6: w = 1.0 / 1890.0; break;
      case 8: w = 1.0 / 15120.0; break;
      default: continue; /* no integer vector has |c|^2 = 7 */
    }
    for (int x = -2; x <= 2; x++)
      for (int y = -2; y <= 2; y++)
        for (int z = -2; z <= 2; z++)
          if (x * x + y * y + z * z == r2) {
            c[m][0] = x;
            c[m][1] = y;
            c[m][2] = z;
            p[m] = w;
            m++;
          }
  }
  return m;
}

int orc_mr_vectors(int* c, double* p) {
  int cc[93][3];
  double pp[93];
  int m = mr_table(cc, pp);
  for (int j = 0; j < m; j++) {
    for (int a = 0; a < 3; a++) c[3 * j + a] = cc[j][a];
    p[j] = pp[j];
  }
  return m;
}

/* SC forces for every node into s->F (Eq. interactionforceMP, or the cross force of
 * Eq. doublebeltrepulsionforce2 for the two-component model: species 0 -> F, species 1 ->
 * the second half of gN, reused as scratch). */
static void stage_sc_force(orc_sim* s) {
  const lattice_t* L = &s->L;
  if (s->p.model == ORC_SC_MP) {
#pragma omp parallel for schedule(static)
    for (long n = 0; n < (long)s->n; n++) s->psi[n] = sc_psi(s->rho_r[n], s->p.rho0_psi);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < (long)s->n; n++) {
      double acc[3] = {0.0, 0.0, 0.0};
      for (int i = 1; i < L->q; i++) {
        size_t m = neighbour(s, (size_t)n, i);
        double v = s->solid[m] ? s->psi[n] : s->psi[m];
        for (int a = 0; a < 3; a++) acc[a] += L->w[i] * v * L->c[i][a];
      }
      for (int a = 0; a < 3; a++) s->F[3 * n + a] = -s->p.G * s->psi[n] * acc[a] + s->p.body_force[a];
    }
  } else if (s->p.model == ORC_SC_MR) {
    /* Eq. benziforces per species s: F^a_s + F^r_s + F^X_s (+ its share of the body force) */
    const double g = s->p.G / (s->p.rho0_psi * s->p.rho0_psi);
    int c[93][3];
    double pw[93];
    const int nv = mr_table(c, pw);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < (long)s->n; n++) {
      s->psi[n] = sc_psi(s->rho_r[n], s->p.rho0_psi);
      s->psi2[n] = sc_psi(s->rho_b[n], s->p.rho0_psi);
    }
#pragma omp parallel for schedule(static)
    for (long n = 0; n < (long)s->n; n++) {
      long x, y, z;
      coords(s, (size_t)n, &x, &y, &z);
      const double* psis[2] = {s->psi, s->psi2};
      const double* rhos[2] = {s->rho_r, s->rho_b};
      const double rho = s->rho_r[n] + s->rho_b[n];
      for (int sp = 0; sp < 2; sp++) {
        const double* ps = psis[sp];
        const double* other = rhos[1 - sp];
        double att[3] = {0.0, 0.0, 0.0}, rep[3] = {0.0, 0.0, 0.0}, crs[3] = {0.0, 0.0, 0.0};
        /* belt 1 with the lattice weights: Eq. doublebeltattractiveforce and the cross
           force of Eq. doublebeltrepulsionforce2 */
        for (int i = 1; i < L->q; i++) {
          size_t m = neighbour(s, (size_t)n, i);
          double vp = s->solid[m] ? ps[n] : ps[m];
          double vo = s->solid[m] ? other[n] : other[m];
          for (int a = 0; a < 3; a++) {
            att[a] += L->w[i] * vp * L->c[i][a];
            crs[a] += L->w[i] * vo * L->c[i][a];
          }
        }
        /* belts 1 + 2 with the weights p: Eq. doublebeltrepulsionforce */
        for (int j = 1; j < nv; j++) {
          size_t m = node_of(s, x + c[j][0], y + c[j][1], z + c[j][2]);
          double vp = s->solid[m] ? ps[n] : ps[m];
          for (int a = 0; a < 3; a++) rep[a] += pw[j] * vp * c[j][a];
        }
        double* out = sp == 0 ? s->F + 3 * n : s->gN + 3 * n;
        for (int a = 0; a < 3; a++)
          out[a] = -s->p.Ga[sp] * ps[n] * att[a] - s->p.Gr[sp] * ps[n] * rep[a] - g * rhos[sp][n] * crs[a] +
                   s->p.body_force[a] * rhos[sp][n] / rho;
      }
    }
  } else {
    double g = s->p.G / (s->p.rho0_psi * s->p.rho0_psi);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < (long)s->n; n++) {
      double a1[3] = {0.0, 0.0, 0.0}, a2[3] = {0.0, 0.0, 0.0};
      for (int i = 1; i < L->q; i++) {
        size_t m = neighbour(s, (size_t)n, i);
        double v2 = s->solid[m] ? s->rho_b[n] : s->rho_b[m];
        double v1 = s->solid[m] ? s->rho_r[n] : s->rho_r[m];
        for (int a = 0; a < 3; a++) {
          a1[a] += L->w[i] * v2 * L->c[i][a];
          a2[a] += L->w[i] * v1 * L->c[i][a];
        }
      }
      double rr = s->rho_r[n], rb = s->rho_b[n], rho = rr + rb;
      for (int a = 0; a < 3; a++) {
        s->F[3 * n + a] = -g * rr * a1[a] + s->p.body_force[a] * rr / rho;
        s->gN[3 * n + a] = -g * rb * a2[a] + s->p.body_force[a] * rb / rho;
      }
    }
  }
}

static void sc_collide_node(orc_sim* s, size_t n) {
  const lattice_t* L = &s->L;
  const int Q = L->q;
  double feq[19], S[19];
  if (s->p.model == ORC_SC_MP) {
    double rho = s->rho_r[n];
    const double* F = s->F + 3 * n;
    double j[3], u[3];
    momentum_at(s, n, j);
    for (int a = 0; a < 3; a++) u[a] = (j[a] + 0.5 * F[a]) / rho; /* Eq. guoforce2 */
    sc_feq(L, rho, u, feq);
    guo_source(L, u, F, 1.0 / s->p.tau_r, S);
    for (int i = 0; i < Q; i++) {
      double fi = fp(s, s->f, 0, i)[n];
      fp(s, s->fpost, 0, i)[n] = fi - (fi - feq[i]) / s->p.tau_r + S[i]; /* Eq. collisSC */
    }
  } else {
    double rr = s->rho_r[n], rb = s->rho_b[n], rho = rr + rb;
    const double* F1 = s->F + 3 * n;
    const double* F2 = s->gN + 3 * n;
    double j[3], u[3];
    momentum_at(s, n, j);
    for (int a = 0; a < 3; a++) u[a] = (j[a] + 0.5 * (F1[a] + F2[a])) / rho;
    const double taus[2] = {s->p.tau_r, s->p.tau_b};
    const double rhos[2] = {rr, rb};
    for (int k = 0; k < 2; k++) {
      sc_feq(L, rhos[k], u, feq);
      guo_source(L, u, k == 0 ? F1 : F2, 1.0 / taus[k], S);
      for (int i = 0; i < Q; i++) {
        double fi = fp(s, s->f, k, i)[n];
        fp(s, s->fpost, k, i)[n] = fi - (fi - feq[i]) / taus[k] + S[i];
      }
    }
  }
}

int orc_init(orc_sim* s, const double* rho_r, const double* rho_b, const double* u,
             const uint8_t* solid, const double* pops) {
  if (!s) return 1;
  const int Q = s->L.q;
  if (solid)
    memcpy(s->solid, solid, s->n);
  else
    memset(s->solid, 0, s->n);
  size_t nf = (size_t)s->ncomp * Q * s->n;
  if (pops) {
    memcpy(s->f, pops, nf * sizeof(double));
    return 0;
  }
  memset(s->f, 0, nf * sizeof(double));
  for (size_t n = 0; n < s->n; n++) {
    s->rho_r[n] = rho_r[n];
    s->rho_b[n] = (s->ncomp == 2 && rho_b) ? rho_b[n] : 0.0;
  }
  if (s->p.model == ORC_CG) {
    stage_color(s);
    stage_cg_gradients(s);
  }
  for (size_t n = 0; n < s->n; n++) {
    if (s->solid[n]) continue;
    double un[3] = {0.0, 0.0, 0.0};
    if (u)
      for (int a = 0; a < 3; a++) un[a] = u[(size_t)a * s->n + n];
    double feq[19];
    if (s->p.model == ORC_CG) {
      double nubar, omega;
      interface_viscosity(s, s->rho_r[n], s->rho_b[n], &nubar, &omega);
      cg_feq(&s->L, s->phiR, s->rho_r[n], un, s->gR + 3 * n, nubar, s->p.enhanced_eq, feq);
      for (int i = 0; i < Q; i++) fp(s, s->f, 0, i)[n] = feq[i];
      cg_feq(&s->L, s->phiB, s->rho_b[n], un, s->gB + 3 * n, nubar, s->p.enhanced_eq, feq);
      for (int i = 0; i < Q; i++) fp(s, s->f, 1, i)[n] = feq[i];
    } else {
      for (int k = 0; k < s->ncomp; k++) {
        sc_feq(&s->L, k == 0 ? s->rho_r[n] : s->rho_b[n], un, feq);
        for (int i = 0; i < Q; i++) fp(s, s->f, k, i)[n] = feq[i];
      }
    }
  }
  return 0;
}

/* Recompute every per-node field the current populations imply (densities, colour,
 * gradients, forces).  Used both by the step and by the moment output. */
static void stage_fields(orc_sim* s) {
  stage_densities(s);
  if (s->p.model == ORC_CG) {
    stage_color(s);
    stage_cg_gradients(s);
    stage_cg_force(s);
  } else {
    stage_sc_force(s);
  }
}

int orc_step(orc_sim* s, int nsteps) {
  if (!s || nsteps < 0) return 1;
  for (int t = 0; t < nsteps; t++) {
    stage_fields(s);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < (long)s->n; n++) {
      if (s->solid[n]) continue;
      if (s->p.model == ORC_CG)
        cg_collide_node(s, (size_t)n);
      else
        sc_collide_node(s, (size_t)n);
    }
    stage_stream(s);
  }
  return 0;
}

void orc_get_pops(const orc_sim* s, double* out) {
  memcpy(out, s->f, (size_t)s->ncomp * s->L.q * s->n * sizeof(double));
}

int orc_force(orc_sim* s, double* F) {
  if (!s) return 1;
  stage_fields(s);
  for (size_t n = 0; n < s->n; n++)
    for (int a = 0; a < 3; a++) F[(size_t)a * s->n + n] = s->F[3 * n + a];
  return 0;
}

int orc_moments(orc_sim* s, double* rho_r, double* rho_b, double* u, double* totals) {
  if (!s) return 1;
  stage_fields(s);
  double t[ORC_NTOTALS] = {0};
  t[8] = INFINITY;
  t[9] = INFINITY;
  for (size_t n = 0; n < s->n; n++) {
    double j[3], un[3];
    momentum_at(s, n, j);
    double rr = s->rho_r[n], rb = s->rho_b[n], rho = rr + rb;
    double Ft[3];
    for (int a = 0; a < 3; a++) Ft[a] = s->F[3 * n + a];
    if (s->p.model == ORC_SC_2C || s->p.model == ORC_SC_MR)
      for (int a = 0; a < 3; a++) Ft[a] += s->gN[3 * n + a];
    for (int a = 0; a < 3; a++) un[a] = s->solid[n] ? 0.0 : (j[a] + 0.5 * Ft[a]) / rho;
    if (rho_r) rho_r[n] = rr;
    if (rho_b) rho_b[n] = rb;
    if (u)
      for (int a = 0; a < 3; a++) u[(size_t)a * s->n + n] = un[a];
    if (s->solid[n]) continue;
    int bad = 0;
    for (int k = 0; k < s->ncomp; k++)
      for (int i = 0; i < s->L.q; i++)
        if (!isfinite(fp(s, s->f, k, i)[n])) bad = 1;
    t[0] += rr;
    t[1] += rb;
    t[2] += j[0];
    t[3] += j[1];
    t[4] += j[2];
    double uu = dot3(un, un);
    t[5] += 0.5 * rho * uu;
    if (sqrt(uu) > t[6]) t[6] = sqrt(uu);
    t[7] += bad;
    if (rr < t[8]) t[8] = rr;
    if (rb < t[9]) t[9] = rb;
  }
  if (totals) memcpy(totals, t, sizeof t);
  return 0;
}

/* ---- exported building blocks ---- */

int orc_lattice_tables(int lattice, int* q, int* c, double* w, double* B, double* psi, double* xi) {
  lattice_t L;
  lattice_fill(lattice, &L);
  if (q) *q = L.q;
  for (int i = 0; i < L.q; i++) {
    if (c)
      for (int a = 0; a < 3; a++) c[3 * i + a] = L.c[i][a];
    if (w) w[i] = L.w[i];
    if (B) B[i] = L.B[i];
    if (psi) psi[i] = L.psi[i];
    if (xi) xi[i] = L.xi[i];
  }
  return L.d;
}

void orc_phi(int lattice, double alpha, double* phi) { phi_fill(lattice, alpha, phi); }

void orc_cg_equilibrium(int lattice, double rho_k, double alpha_k, const double* u, const double* grad_k,
                        double nubar, int enhanced, double* feq) {
  lattice_t L;
  lattice_fill(lattice, &L);
  double phi[19];
  phi_fill(lattice, alpha_k, phi);
  cg_feq(&L, phi, rho_k, u, grad_k, nubar, enhanced, feq);
}

void orc_sc_equilibrium(int lattice, double rho, const double* u, double* feq) {
  lattice_t L;
  lattice_fill(lattice, &L);
  sc_feq(&L, rho, u, feq);
}

void orc_guo_source(int lattice, const double* u, const double* F, double omega, double* S) {
  lattice_t L;
  lattice_fill(lattice, &L);
  guo_source(&L, u, F, omega, S);
}

void orc_perturbation(int lattice, const double* grad_n, double A, double eps, double* d) {
  lattice_t L;
  lattice_fill(lattice, &L);
  perturbation(&L, grad_n, A, eps, d);
}

void orc_recolor(int lattice, const double* fstar, double rho_r, double rho_b, double alpha_r,
                 double alpha_b, const double* grad_n, double beta, double eps, double* fr, double* fb) {
  lattice_t L;
  lattice_fill(lattice, &L);
  double phiR[19], phiB[19];
  phi_fill(lattice, alpha_r, phiR);
  phi_fill(lattice, alpha_b, phiB);
  recolor(&L, fstar, rho_r, rho_b, phiR, phiB, grad_n, beta, eps, fr, fb);
}
