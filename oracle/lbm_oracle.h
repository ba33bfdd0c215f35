/*
 * lbm_oracle.h -- plain FP64 CPU oracle for the two-component lattice Boltzmann step
 * of Datadien, Di Staso, Wijshoff & Toschi, "A quantitative comparison of physical
 * accuracy and numerical stability of lattice Boltzmann color gradient and
 * pseudopotential multicomponent models for microfluidic applications" (arXiv 2110.05197).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously-correct reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the product library never links or calls it.
 *
 * It shares no code, header, table or helper with the CUDA path.  It follows the paper's
 * equations in the paper's order, one plain loop per step, in double precision, compiled
 * with floating-point contraction off.
 *
 * Layout: populations f[k][i][node], node = x + nx*(y + ny*z), x fastest.
 * Direction order (the paper lists only the groups, Eq. speeds):
 *   D3Q19: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),
 *          (1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1).
 *   D2Q9:  0 rest; 1..4 = +x,-x,+y,-y; 5..8 = (1,1),(-1,-1),(1,-1),(-1,1).
 * For every i >= 1 the opposite direction of odd i is i+1.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_D2Q9 = 0, ORC_D3Q19 = 1 };
enum { ORC_CG = 0, ORC_SC_MP = 1, ORC_SC_2C = 2, ORC_SC_MR = 3 };
enum { ORC_NTOTALS = 10 };

typedef struct {
  int32_t lattice;       /* ORC_D2Q9 or ORC_D3Q19 */
  int32_t model;         /* ORC_CG, ORC_SC_MP (one population set), ORC_SC_2C (two sets) */
  int32_t nx, ny, nz;    /* nz = 1 for D2Q9 */
  double rho_r0, rho_b0; /* CG bulk densities: gamma = rho_r0/rho_b0 (Eq. gamma) */
  double alpha_b;        /* CG rest parameter of the blue fluid (0.2 in the paper) */
  double tau_r, tau_b;   /* relaxation times; SC multiphase uses tau_r */
  double A, beta;        /* CG perturbation amplitude (Eq. sigmaA) and recolouring beta */
  int32_t enhanced_eq;   /* 1: enhanced equilibrium (Eq. equiliCG), 0: plain second-order part */
  int32_t color_norm;    /* 0: rho^N = (rR-rB)/(rR+rB); 1: densities scaled by rho_k0 first */
  double rep_pi, rep_chi;/* CG repulsion force: Pi (0 disables) and chi (Eq. repForce, potential) */
  int32_t rep_psi_kind;  /* 0: psi_rep = (1-|rho^N|)^chi, 1: (1+|rho^N|)^chi as printed */
  double grad_eps;       /* |grad rho^N| at or below this: no perturbation, cos(phi)=0, no normal */
  double G, rho0_psi;    /* SC coupling and reference density (Eqs. interactionforceMP, pseudopotential,
                            doublebeltrepulsionforce2) */
  double body_force[3];  /* constant body-force density, applied with Guo forcing */
  double Ga[2], Gr[2];   /* ORC_SC_MR (D3Q19 only): attractive and repulsive self-couplings of
                            each species (Eqs. doublebeltattractiveforce,
                            doublebeltrepulsionforce); G is the cross coupling G_AB */
} orc_params;

typedef struct orc_sim orc_sim;

/* Thread count for the per-node loops (OpenMP); <=0 keeps the runtime default. */
void orc_set_threads(int n);
int orc_get_threads(void);

orc_sim* orc_create(const orc_params* p);
void orc_destroy(orc_sim* s);
/* rho_r, rho_b: [N]; u: [3][N] or NULL; solid: [N] or NULL; pops: [K][Q][N] or NULL.
 * With pops == NULL the populations start at the equilibrium of (rho_k, u, grad rho_k). */
int orc_init(orc_sim* s, const double* rho_r, const double* rho_b, const double* u,
             const uint8_t* solid, const double* pops);
int orc_step(orc_sim* s, int nsteps);
void orc_get_pops(const orc_sim* s, double* out);
/* Any output may be NULL.  u is the force-shifted velocity.  totals[ORC_NTOTALS]:
 * mass_r, mass_b, mom_x, mom_y, mom_z (bare momentum sum_k sum_i f c_i), E_kin (1/2 rho |u|^2),
 * max|u|, nonfinite node count, min rho_r, min rho_b -- all over fluid nodes. */
int orc_moments(orc_sim* s, double* rho_r, double* rho_b, double* u, double* totals);
/* Force density the current state feels (SC force or CG repulsion + body force): [3][N]. */
int orc_force(orc_sim* s, double* F);

/* ---- per-node building blocks, exported for the identity tests ---- */
/* The 93 vectors of belts 1 and 2 (every integer vector with |c|^2 <= 8, rest first) and
 * their forcing weights p (Eq. pweights): c[93][3], p[93].  Returns 93. */
int orc_mr_vectors(int* c, double* p);
int orc_lattice_tables(int lattice, int* q, int* c, double* w, double* B, double* psi,
                       double* xi);
void orc_phi(int lattice, double alpha, double* phi);
void orc_cg_equilibrium(int lattice, double rho_k, double alpha_k, const double* u,
                        const double* grad_k, double nubar, int enhanced, double* feq);
void orc_sc_equilibrium(int lattice, double rho, const double* u, double* feq);
void orc_guo_source(int lattice, const double* u, const double* F, double omega, double* S);
void orc_perturbation(int lattice, const double* grad_n, double A, double eps, double* dOmega);
void orc_recolor(int lattice, const double* fstar, double rho_r, double rho_b, double alpha_r,
                 double alpha_b, const double* grad_n, double beta, double eps, double* fr,
                 double* fb);

#ifdef __cplusplus
}
#endif
#endif
