/*
 * lbm_oracle.h -- plain, slow FP64 CPU oracle of the lattice Boltzmann
 * no-slip path in Peng, Ayala & Wang, "A comparative study of immersed
 * boundary method and interpolated bounce-back scheme for no-slip boundary
 * treatment in the lattice Boltzmann method" (arXiv 1906.05445).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header or table with the CUDA library; the two agree only on the
 * documented interface formats (direction order, [Q][z][y][x] layout and the
 * integer values of the scheme/lattice selectors).
 *
 * Everything is FP64, lattice units (dx = dt = h = 1, c_s^2 = 1/3, rho0 = 1).
 * The state kept by a simulation is the PRE-collision distribution f(x, t).
 * One step follows the paper's evolution equation in its own order:
 * geometry -> (IBM force, Sec. 2.1) -> collision (Eq. 1 / Eq. 3) ->
 * streaming with interpolated bounce-back on cut links (Sec. 2.2) ->
 * momentum exchange (Eq. 17) -> prescribed motion of the solids.
 *
 * Parity status of every function is listed where it is defined.  The
 * refilling of uncovered nodes is a reading (the paper gives no formula); it
 * is pinned by the co-moving uniform flow, an exact fixed point that a
 * refill at the wrong velocity or density, or none, breaks.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* lattice selectors */
#define ORA_D2Q9 0
#define ORA_D3Q19 1
/* collision selectors */
#define ORA_BGK 0
#define ORA_MRT 1
/* solid kinds */
#define ORA_SPHERE 0     /* circle on a 2D lattice */
#define ORA_CYLINDER_Z 1 /* infinite cylinder along z */
/* no-slip schemes */
#define ORA_NONE 0
#define ORA_BB 1            /* simple bounce-back, Eq. 10 */
#define ORA_BOUZIDI_LIN 2   /* linear analogue of Eq. 11 */
#define ORA_BOUZIDI_QUAD 3  /* Eq. 11 */
#define ORA_YU_LIN 4        /* linear analogue of Eqs. 12-14 */
#define ORA_YU_QUAD 5       /* Eqs. 12-14 (combined: Eq. 15, corrected) */
#define ORA_IBM 6           /* direct-forcing IBM, Sec. 2.1 (Eqs. 4-9) */
#define ORA_ZHAO_YONG 7     /* single-node bounce-back, Eq. 16 */

typedef struct ora_sim ora_sim;

/* ---- single-node building blocks (exposed for the pin tests) ---- */
int ora_q(int lattice);
/* e: [Q][3] ints, w: [Q] */
void ora_lattice(int lattice, int *e, double *w);
/* rows of the moment basis, M: [Q][Q] row-major */
void ora_mrt_matrix(int lattice, double *M);
/* default relaxation rates for tau (moment order of ora_mrt_matrix) */
void ora_mrt_default_rates(int lattice, double tau, double *s);
/* incompressible equilibrium, feq[Q] */
void ora_equilibrium(int lattice, double rho, const double u[3], double *feq);
/* one collision (Eq. 1 or Eq. 3 with Guo forcing); rates may be NULL (BGK
 * ignores them, MRT then uses the defaults) */
void ora_collide(int lattice, int collision, double tau, const double *rates,
                 const double *f, const double F[3], double *fout);
/* coefficients c[0..5] of the interpolated bounce-back rule; returns the
 * scheme actually used after the fallback for missing neighbours */
int ora_ibb_coeffs(int scheme, double q, int have_ff, int have_fff, double c[6]);
/* Peskin's 4-point kernel, Eq. 6 */
double ora_phi(double r);
/* delta-function kernels compared in Sec. 3.1 (selector ORA_DELTA_*) */
#define ORA_DELTA_PESKIN4 0  /* Eq. 6 */
#define ORA_DELTA_ROMA3 1    /* Roma, Peskin & Berger 3-point */
#define ORA_DELTA_LINEAR2 2  /* 2-point linear */
#define ORA_DELTA_COSINE4 3  /* 4-point cosine (Appendix B) */
double ora_phi_kernel(int kernel, double r);

/* ---- simulation ---- */
ora_sim *ora_create(int lattice, int nx, int ny, int nz, double tau,
                    int collision, const double *rates /* Q or NULL */,
                    const double g[3], int force_all);
void ora_destroy(ora_sim *s);
/* returns the solid id or -1 */
int ora_add_solid(ora_sim *s, int kind, const double c[3], double R,
                  const double U[3], const double Om[3], int fluid_inside);
/* the IBM kernel (ORA_DELTA_*, default Peskin's 4-point) */
void ora_set_ibm_kernel(ora_sim *s, int kernel);
void ora_set_scheme(ora_sim *s, int scheme, int ibm_iters, double retraction,
                    double marker_density);
void ora_init_equilibrium(ora_sim *s, double rho, const double u[3]);
/* f: [Q][N] pre-collision distributions (full f, not deviations) */
void ora_set_f(ora_sim *s, const double *f);
void ora_get_f(const ora_sim *s, double *f);
void ora_step(ora_sim *s, int nsteps);
/* fields at the current time; entries at solid nodes are 0 */
void ora_density(ora_sim *s, double *rho /*[N]*/);
void ora_velocity(ora_sim *s, double *u /*[d][N]*/);
void ora_strain_rate(ora_sim *s, double *S /*[d(d+1)/2][N]*/);
/* 1 at nodes not simulated (solid nodes under bounce-back), else 0 */
void ora_solid_mask(ora_sim *s, unsigned char *m /*[N]*/);
/* force and torque on solid `id` from the most recent step (bounce-back:
 * momentum exchange of the last streaming; IBM: marker force at the current
 * time) */
void ora_force_torque(ora_sim *s, int id, double F[3], double T[3]);
int ora_num_markers(const ora_sim *s, int id);
/* L2 residual between the velocity now and a snapshot taken by
 * ora_snapshot_velocity */
void ora_snapshot_velocity(ora_sim *s);
double ora_residual(ora_sim *s);
long ora_steps_done(const ora_sim *s);
void ora_solid_centre(const ora_sim *s, int id, double c[3]);
/* number of cut links last handled by each scheme (fallback statistics):
 * counts[0..7] indexed by scheme selector */
void ora_link_stats(const ora_sim *s, long counts[8]);
/* free motion (Sec. 3.2): density ratio rho_p / rho_f (<= 0: prescribed
 * motion) and gravity; the solid's velocities then follow Eq. 20
 * (bounce-back) or Eq. 23 (IBM) every step */
void ora_set_solid_dynamics(ora_sim *s, int id, double rho_ratio, const double g[3]);
/* Domain faces x-, x+, y-, y+, z-, z+ (Sec. 3.4): periodic pairs, plane walls
 * moving with u_face[3k..3k+2] (velocity inlet or no-slip wall), stress-free
 * (specular) faces, and at most one convective outflow face.  Returns 0, or
 * -1 for an unpaired periodic face, a z face on a 2D lattice or a second
 * outflow face.  Solids must keep clear of non-periodic faces. */
#define ORA_FACE_PERIODIC 0
#define ORA_FACE_VELOCITY 1
#define ORA_FACE_FREE_SLIP 2
#define ORA_FACE_CONVECTIVE 3
int ora_set_domain(ora_sim *s, const int face[6], const double *u_face);
/* epsilon = 2 nu s_ij s_ij from the strain rate of ora_strain_rate [N] */
void ora_dissipation(ora_sim *s, double *eps);
/* sigma = -c_s^2 rho I + 2 rho0 nu S (Sec. 3.1), order of ora_strain_rate */
void ora_stress(ora_sim *s, double *sig /*[d(d+1)/2][N]*/);
/* Inertia of the fluid inside a free solid under IBM (Sec. 3.2): the
 * rigid-body form of Feng & Michaelides (Eq. 23, default), Kempe et al.'s
 * volume integrals with level-set cell fractions (Eqs. 24-26), or Uhlmann's
 * reduced inertia (Eq. 22). */
#define ORA_INERTIA_FENG 0
#define ORA_INERTIA_KEMPE 1
#define ORA_INERTIA_UHLMANN 2 /* Eq. 22 (needs rho_p > rho_f) */
void ora_set_ibm_inertia(ora_sim *s, int inertia);
/* Eq. 25 at node (x, y, z) for solid id, and Eq. 24 for solid id at the
 * current time (momentum, then angular momentum about the centre). */
double ora_cell_fraction(ora_sim *s, int id, long x, long y, long z);
void ora_internal_fluid(ora_sim *s, int id, double I[6]);
void ora_solid_velocity(const ora_sim *s, int id, double U[3], double Om[3]);

/* ---- immersed-boundary primitives on a bare periodic grid (pin tests) ----
 * u: [d][N] Eulerian field, X: [3][n] marker positions.
 * interp: U[d][n] = sum_x u(x) delta_h(x - X) h^d        (Eq. 5)
 * spread: f[d][N] += sum_X F(X) delta_h(x - X) dV(X)      (Eq. 8)       */
void ora_ibm_interp(int d, int nx, int ny, int nz, const double *u,
                    int n, const double *X, double *U);
void ora_ibm_spread(int d, int nx, int ny, int nz, double *f, int n,
                    const double *X, const double *F, const double *dV);
/* the same with another kernel */
void ora_ibm_interp_k(int kernel, int d, int nx, int ny, int nz, const double *u,
                      int n, const double *X, double *U);
void ora_ibm_spread_k(int kernel, int d, int nx, int ny, int nz, double *f, int n,
                      const double *X, const double *F, const double *dV);

#ifdef __cplusplus
}
#endif
#endif
