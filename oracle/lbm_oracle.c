/*
 * lbm_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Written from Peng, Ayala & Wang (arXiv 1906.05445).  Each routine names the
 * passage it follows.  No blocking, fusion or reordering beyond what the
 * equations state: the collision runs node by node over whole arrays, then
 * the streaming runs node by node, exactly as Eq. 1 / Eq. 3 read.
 *
 * Readings of passages where the paper is silent (all listed in the design
 * notes of the repository):
 *  - equilibrium: incompressible form w_i[rho + rho0(3e.u + 4.5(e.u)^2 -
 *    1.5u^2)] with u = (j + F dt/2)/rho0 (the paper uses rho0 in Eqs. 10-17);
 *  - MRT basis: Lallemand-Luo (D2Q9) and d'Humieres et al. (D3Q19)
 *    polynomial rows, m_eq = M f_eq, forcing Psi = (I - S/2) M Fbar, i.e.
 *    Guo's term in moment space (the inverse design cited in Sec. 2.1);
 *  - linear Bouzidi / Yu rules: two-point versions of the constructions that
 *    give Eq. 11 and Eqs. 12-14; Eq. 15 is composed from Eqs. 12-14 (its
 *    printed second coefficient does not sum to one);
 *  - missing interpolation neighbours: quadratic -> linear -> Eq. 10;
 *  - refilling: equilibrium at the mean density of neighbours that were
 *    fluid before and after the move, at the local wall velocity (the paper
 *    gives no formula); pinned by the co-moving uniform flow, which it must
 *    keep exact at any uniform density.
 *  - IBM markers: golden-angle (Fibonacci) points on the sphere of radius
 *    R - R_d (R + R_d for an enclosing wall), about `density` markers per
 *    unit area, dV = area * h / N.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define MAXQ 19
#define MAXS 8
#define RHO0 1.0
#define CS2 (1.0 / 3.0)

/* ------------------------------------------------------------------ */
/* Lattices: direction order is an interface format shared (as a format,
 * not as code) with the CUDA library.                                  */
static const int E9[9][3] = {{0, 0, 0},  {1, 0, 0},   {0, 1, 0},
                             {-1, 0, 0}, {0, -1, 0},  {1, 1, 0},
                             {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const double W9[9] = {4.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const int E19[19][3] = {
    {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
    {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

int ora_q(int lattice) { return lattice == ORA_D2Q9 ? 9 : 19; }

void ora_lattice(int lattice, int *e, double *w) {
  int Q = ora_q(lattice);
  for (int i = 0; i < Q; i++) {
    for (int a = 0; a < 3; a++)
      e[3 * i + a] = lattice == ORA_D2Q9 ? E9[i][a] : E19[i][a];
    if (lattice == ORA_D2Q9)
      w[i] = W9[i];
    else
      w[i] = i == 0 ? 1.0 / 3 : (i <= 6 ? 1.0 / 18 : 1.0 / 36);
  }
}

/* Moment basis rows as polynomials of the lattice velocity (Eq. 3 leaves M
 * to the textbooks; these are the standard Gram-Schmidt rows). */
static double mrt_row(int lattice, int k, int ex, int ey, int ez) {
  double e2 = ex * ex + ey * ey + ez * ez;
  if (lattice == ORA_D2Q9) {
    switch (k) {
    case 0: return 1;
    case 1: return -4 + 3 * e2;
    case 2: return 4 - 10.5 * e2 + 4.5 * e2 * e2;
    case 3: return ex;
    case 4: return (-5 + 3 * e2) * ex;
    case 5: return ey;
    case 6: return (-5 + 3 * e2) * ey;
    case 7: return ex * ex - ey * ey;
    default: return ex * ey;
    }
  }
  switch (k) {
  case 0: return 1;
  case 1: return 19 * e2 - 30;
  case 2: return (21 * e2 * e2 - 53 * e2 + 24) / 2;
  case 3: return ex;
  case 4: return (5 * e2 - 9) * ex;
  case 5: return ey;
  case 6: return (5 * e2 - 9) * ey;
  case 7: return ez;
  case 8: return (5 * e2 - 9) * ez;
  case 9: return 3 * ex * ex - e2;
  case 10: return (3 * e2 - 5) * (3 * ex * ex - e2);
  case 11: return ey * ey - ez * ez;
  case 12: return (3 * e2 - 5) * (ey * ey - ez * ez);
  case 13: return ex * ey;
  case 14: return ey * ez;
  case 15: return ex * ez;
  case 16: return (ey * ey - ez * ez) * ex;
  case 17: return (ez * ez - ex * ex) * ey;
  default: return (ex * ex - ey * ey) * ez;
  }
}

void ora_mrt_matrix(int lattice, double *M) {
  int Q = ora_q(lattice), e[MAXQ * 3];
  double w[MAXQ];
  ora_lattice(lattice, e, w);
  for (int k = 0; k < Q; k++)
    for (int i = 0; i < Q; i++)
      M[k * Q + i] = mrt_row(lattice, k, e[3 * i], e[3 * i + 1], e[3 * i + 2]);
}

/* kind of each moment: 'c' conserved, 'b' energy (bulk), 'e' energy square,
 * 'q' energy flux, 'v' stress (shear viscosity), 'p' pi ghost, 'm' m ghost */
static char moment_kind(int lattice, int k) {
  static const char k9[] = "cbecqcqvv";
  static const char k19[] = "cbecqcqcqvpvpvvvmmm";
  return lattice == ORA_D2Q9 ? k9[k] : k19[k];
}

void ora_mrt_default_rates(int lattice, double tau, double *s) {
  int Q = ora_q(lattice);
  double snu = 1.0 / tau;
  /* energy-flux rate from the "magic" product (1/s_nu - 1/2)(1/s_q - 1/2)
   * = 3/16 */
  double sq = 1.0 / (0.5 + (3.0 / 16.0) / (tau - 0.5));
  for (int k = 0; k < Q; k++)
    s[k] = moment_kind(lattice, k) == 'q' ? sq : snu;
}

/* Incompressible equilibrium (reading: the paper's rho0 in Eqs. 10-17). */
void ora_equilibrium(int lattice, double rho, const double u[3], double *feq) {
  int Q = ora_q(lattice), e[MAXQ * 3];
  double w[MAXQ];
  ora_lattice(lattice, e, w);
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q; i++) {
    double eu = e[3 * i] * u[0] + e[3 * i + 1] * u[1] + e[3 * i + 2] * u[2];
    feq[i] = w[i] * (rho + RHO0 * (3 * eu + 4.5 * eu * eu - 1.5 * uu));
  }
}

/* Plain Gauss-Jordan inverse with partial pivoting (n <= 19). */
static void invert(int n, const double *A, double *Ainv) {
  double a[MAXQ][2 * MAXQ];
  for (int r = 0; r < n; r++)
    for (int c = 0; c < 2 * n; c++)
      a[r][c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int c = 0; c < n; c++) {
    int p = c;
    for (int r = c + 1; r < n; r++)
      if (fabs(a[r][c]) > fabs(a[p][c])) p = r;
    if (p != c)
      for (int k = 0; k < 2 * n; k++) {
        double t = a[c][k];
        a[c][k] = a[p][k];
        a[p][k] = t;
      }
    double d = a[c][c];
    for (int k = 0; k < 2 * n; k++) a[c][k] /= d;
    for (int r = 0; r < n; r++)
      if (r != c) {
        double m = a[r][c];
        for (int k = 0; k < 2 * n; k++) a[r][k] -= m * a[c][k];
      }
  }
  for (int r = 0; r < n; r++)
    for (int c = 0; c < n; c++) Ainv[r * n + c] = a[r][c + n];
}

/* Constants of one collision operator (lattice tables, M, M^-1, S), built
 * once so that the per-node loop below only does the arithmetic. */
typedef struct {
  int lattice, Q, collision;
  double tau;
  int e[MAXQ][3];
  double w[MAXQ], M[MAXQ * MAXQ], Minv[MAXQ * MAXQ], s[MAXQ];
} coll_t;

static void coll_init(coll_t *c, int lattice, int collision, double tau,
                      const double *rates) {
  int e[MAXQ * 3];
  c->lattice = lattice;
  c->Q = ora_q(lattice);
  c->collision = collision;
  c->tau = tau;
  ora_lattice(lattice, e, c->w);
  for (int i = 0; i < c->Q; i++)
    for (int a = 0; a < 3; a++) c->e[i][a] = e[3 * i + a];
  ora_mrt_matrix(lattice, c->M);
  invert(c->Q, c->M, c->Minv);
  ora_mrt_default_rates(lattice, tau, c->s);
  if (rates)
    for (int k = 0; k < c->Q; k++)
      if (rates[k] != 0) c->s[k] = rates[k];
}

/* One collision, Eq. 1 (BGK) or Eq. 3 (MRT), with Guo's forcing term
 * (Sec. 2.1): Fbar_i = w_i[(e_i - u)/cs2 + (e_i.u) e_i/cs2^2].F,
 * BGK: f* = f - (f - feq)/tau + (1 - 1/(2 tau)) Fbar,
 * MRT: m* = m - S(m - meq) + (I - S/2) M Fbar,  f* = M^-1 m*. */
static void collide_with(const coll_t *c, const double *f, const double F[3],
                         double *fout) {
  int Q = c->Q;
  double rho = 0, j[3] = {0, 0, 0};
  for (int i = 0; i < Q; i++) {
    rho += f[i];
    for (int a = 0; a < 3; a++) j[a] += f[i] * c->e[i][a];
  }
  double u[3];
  for (int a = 0; a < 3; a++) u[a] = (j[a] + 0.5 * F[a]) / RHO0;
  double feq[MAXQ], Fbar[MAXQ];
  ora_equilibrium(c->lattice, rho, u, feq);
  for (int i = 0; i < Q; i++) {
    double eu = 0, emuF = 0, eF = 0;
    for (int a = 0; a < 3; a++) {
      eu += c->e[i][a] * u[a];
      emuF += (c->e[i][a] - u[a]) * F[a];
      eF += c->e[i][a] * F[a];
    }
    Fbar[i] = c->w[i] * (emuF / CS2 + eu * eF / (CS2 * CS2));
  }
  if (c->collision == ORA_BGK) {
    double tau = c->tau;
    for (int i = 0; i < Q; i++)
      fout[i] = f[i] - (f[i] - feq[i]) / tau + (1 - 0.5 / tau) * Fbar[i];
    return;
  }
  double m[MAXQ], meq[MAXQ], mF[MAXQ], ms[MAXQ];
  for (int k = 0; k < Q; k++) {
    m[k] = meq[k] = mF[k] = 0;
    for (int i = 0; i < Q; i++) {
      m[k] += c->M[k * Q + i] * f[i];
      meq[k] += c->M[k * Q + i] * feq[i];
      mF[k] += c->M[k * Q + i] * Fbar[i];
    }
    ms[k] = m[k] - c->s[k] * (m[k] - meq[k]) + (1 - 0.5 * c->s[k]) * mF[k];
  }
  for (int i = 0; i < Q; i++) {
    fout[i] = 0;
    for (int k = 0; k < Q; k++) fout[i] += c->Minv[i * Q + k] * ms[k];
  }
}

void ora_collide(int lattice, int collision, double tau, const double *rates,
                 const double *f, const double F[3], double *fout) {
  coll_t c;
  coll_init(&c, lattice, collision, tau, rates);
  collide_with(&c, f, F, fout);
}

/* Interpolated bounce-back coefficients (Sec. 2.2).  The rule is
 *   f_i(x_f,t+1) = c0 f*_ib(x_f) + c1 f*_ib(x_ff) + c2 f*_ib(x_fff)
 *                + c3 f_i(x_ff,t+1) + c4 f_i(x_fff,t+1)
 *                + c5 * 2 rho0 w_i (e_i.u_w)/cs2,
 * with f_i(x_ff,t+1) = f*_i(x_f) and f_i(x_fff,t+1) = f*_i(x_ff).
 * Eq. 10 (simple), Eq. 11 (Bouzidi quadratic, both branches), Eqs. 12-14
 * composed (Yu quadratic); the linear rules are the two-point versions of the
 * same constructions (named in Sec. 3.3, not printed). */
int ora_ibb_coeffs(int scheme, double q, int have_ff, int have_fff,
                   double c[6]) {
  for (int k = 0; k < 6; k++) c[k] = 0;
  int s = scheme;
  if ((s == ORA_BOUZIDI_QUAD || s == ORA_YU_QUAD) && !(have_ff && have_fff))
    s = s == ORA_BOUZIDI_QUAD ? ORA_BOUZIDI_LIN : ORA_YU_LIN;
  if ((s == ORA_BOUZIDI_LIN || s == ORA_YU_LIN) && !have_ff) s = ORA_BB;
  switch (s) {
  case ORA_BOUZIDI_QUAD:
    if (q < 0.5) {
      c[0] = q * (2 * q + 1);
      c[1] = (1 + 2 * q) * (1 - 2 * q);
      c[2] = -q * (1 - 2 * q);
      c[5] = 1;
    } else {
      c[0] = 1 / (q * (2 * q + 1));
      c[5] = c[0];
      c[3] = (2 * q - 1) / q;
      c[4] = -(2 * q - 1) / (2 * q + 1);
    }
    break;
  case ORA_BOUZIDI_LIN:
    if (q < 0.5) {
      c[0] = 2 * q;
      c[1] = 1 - 2 * q;
      c[5] = 1;
    } else {
      c[0] = 1 / (2 * q);
      c[5] = c[0];
      c[3] = (2 * q - 1) / (2 * q);
    }
    break;
  case ORA_YU_QUAD: {
    /* Eq. 12: value arriving at the wall, Lagrange weights at 1-q from
     * nodes 0, 1, 2; Eq. 13: bounce; Eq. 14: weights at 0 from -q, 1, 2. */
    double a0 = q * (q + 1) / 2, a1 = (1 + q) * (1 - q), a2 = -q * (1 - q) / 2;
    double bw = 2 / ((1 + q) * (2 + q)), b1 = 2 * q / (1 + q),
           b2 = -q / (2 + q);
    c[0] = bw * a0;
    c[1] = bw * a1;
    c[2] = bw * a2;
    c[3] = b1;
    c[4] = b2;
    c[5] = bw;
    break;
  }
  case ORA_YU_LIN: {
    double a0 = q, a1 = 1 - q;            /* weights at 1-q from 0, 1 */
    double bw = 1 / (1 + q), b1 = q / (1 + q); /* weights at 0 from -q, 1 */
    c[0] = bw * a0;
    c[1] = bw * a1;
    c[3] = b1;
    c[5] = bw;
    break;
  }
  default: /* Eq. 10 */
    s = ORA_BB;
    c[0] = 1;
    c[5] = 1;
  }
  return s;
}

/* Peskin's 4-point regularised delta function, Eq. 6. */
double ora_phi(double r) {
  double a = fabs(r);
  if (a >= 2) return 0;
  if (a >= 1) return (5 - 2 * a - sqrt(-7 + 12 * a - 4 * r * r)) / 8;
  return (3 - 2 * a + sqrt(1 + 4 * a - 4 * r * r)) / 8;
}

/* The one-dimensional kernels compared in Sec. 3.1 (and the cosine kernel
 * named in Appendix B):
 *  - Peskin's 4-point kernel, Eq. 6;
 *  - Roma, Peskin & Berger's 3-point kernel: (1 + sqrt(1 - 3 r^2)) / 3 for
 *    |r| <= 1/2, (5 - 3|r| - sqrt(1 - 3 (1 - |r|)^2)) / 6 for
 *    1/2 <= |r| <= 3/2, 0 beyond;
 *  - the 2-point linear kernel 1 - |r| for |r| <= 1;
 *  - the 4-point cosine kernel (1 + cos(pi r / 2)) / 4 for |r| <= 2.
 * Every support lies inside the 4-point window from floor(X) - 1. */
double ora_phi_kernel(int kernel, double r) {
  double a = fabs(r);
  switch (kernel) {
  case ORA_DELTA_ROMA3:
    if (a >= 1.5) return 0;
    if (a <= 0.5) return (1 + sqrt(1 - 3 * r * r)) / 3;
    return (5 - 3 * a - sqrt(1 - 3 * (1 - a) * (1 - a))) / 6;
  case ORA_DELTA_LINEAR2:
    return a >= 1 ? 0 : 1 - a;
  case ORA_DELTA_COSINE4:
    return a >= 2 ? 0 : (1 + cos(3.14159265358979323846 * r / 2)) / 4;
  default:
    return ora_phi(r);
  }
}

/* ------------------------------------------------------------------ */
typedef struct {
  int kind, fluid_inside;
  double c[3], c0[3], R, U[3], Om[3];
  /* IBM markers: unit directions, control volumes */
  int nm;
  double *dir; /* [3][nm] */
  double *dV;  /* [nm] */
  double *Fm;  /* [3][nm] marker force density */
  double F[3], T[3];
  /* free motion (Eq. 20 under bounce-back, Eq. 23 under IBM): density ratio
   * rho_p / rho_f, gravity, and the velocities of the previous step */
  int free_;
  double rho_p, g[3], Up[3], Omp[3];
  /* Kempe's treatment (Eq. 24): the fluid momentum and angular momentum
   * inside the solid at the previous step, once one has been taken */
  int have_Ip;
  double Ip[6], In[6];
} solid_t;

struct ora_sim {
  int lattice, Q, d, nx, ny, nz, collision, force_all;
  long N;
  double tau, rates[MAXQ], g[3];
  int e[MAXQ][3], opp[MAXQ];
  double w[MAXQ];
  double *f, *fpost;           /* [Q][N] */
  int *inside, *inside_prev;   /* solid id + 1, 0 for fluid */
  int have_prev;
  double *fibm;                /* [3][N] */
  double *usnap;               /* [3][N] */
  int nsol;
  solid_t sol[MAXS];
  int scheme, ibm_iters, ibm_kernel, ibm_inertia;
  double retraction, density;
  long steps;
  long link_counts[8];
  coll_t coll;
  /* domain faces x-, x+, y-, y+, z-, z+ (ORA_FACE_*), the velocity of each
   * velocity face, and the pre-collision populations of the previous time
   * level (outflow faces) */
  int face[6], open;
  double u_face[6][3];
  double *fprev;
};

static long wrapi(long v, long n) {
  v %= n;
  return v < 0 ? v + n : v;
}
static long node(const ora_sim *s, long x, long y, long z) {
  return wrapi(x, s->nx) + s->nx * (wrapi(y, s->ny) + s->ny * wrapi(z, s->nz));
}
static void coords(const ora_sim *s, long n, long *x, long *y, long *z) {
  *x = n % s->nx;
  *y = (n / s->nx) % s->ny;
  *z = n / ((long)s->nx * s->ny);
}
/* nearest periodic image of a separation along an axis of length L */
static double mimage(double d, double L) { return d - L * round(d / L); }

static int is_ibb(int scheme) {
  return (scheme >= ORA_BB && scheme <= ORA_YU_QUAD) || scheme == ORA_ZHAO_YONG;
}

ora_sim *ora_create(int lattice, int nx, int ny, int nz, double tau,
                    int collision, const double *rates, const double g[3],
                    int force_all) {
  ora_sim *s = (ora_sim *)calloc(1, sizeof(ora_sim));
  s->lattice = lattice;
  s->Q = ora_q(lattice);
  s->d = lattice == ORA_D2Q9 ? 2 : 3;
  s->nx = nx;
  s->ny = ny;
  s->nz = lattice == ORA_D2Q9 ? 1 : nz;
  s->N = (long)s->nx * s->ny * s->nz;
  s->tau = tau;
  s->collision = collision;
  s->force_all = force_all;
  for (int k = 0; k < MAXQ; k++) s->rates[k] = 0;
  if (rates)
    for (int k = 0; k < s->Q; k++) s->rates[k] = rates[k];
  for (int a = 0; a < 3; a++) s->g[a] = g ? g[a] : 0;
  if (s->d == 2) s->g[2] = 0;
  int e[MAXQ * 3];
  ora_lattice(lattice, e, s->w);
  for (int i = 0; i < s->Q; i++)
    for (int a = 0; a < 3; a++) s->e[i][a] = e[3 * i + a];
  for (int i = 0; i < s->Q; i++)
    for (int j = 0; j < s->Q; j++)
      if (s->e[j][0] == -s->e[i][0] && s->e[j][1] == -s->e[i][1] &&
          s->e[j][2] == -s->e[i][2])
        s->opp[i] = j;
  s->f = (double *)calloc((size_t)s->Q * s->N, sizeof(double));
  s->fpost = (double *)calloc((size_t)s->Q * s->N, sizeof(double));
  s->inside = (int *)calloc((size_t)s->N, sizeof(int));
  s->inside_prev = (int *)calloc((size_t)s->N, sizeof(int));
  s->fibm = (double *)calloc((size_t)3 * s->N, sizeof(double));
  s->usnap = (double *)calloc((size_t)3 * s->N, sizeof(double));
  s->scheme = ORA_NONE;
  s->ibm_iters = 1;
  s->ibm_kernel = ORA_DELTA_PESKIN4;
  s->density = 1;
  coll_init(&s->coll, lattice, collision, tau, rates);
  double u0[3] = {0, 0, 0};
  ora_init_equilibrium(s, 1.0, u0);
  return s;
}

void ora_destroy(ora_sim *s) {
  if (!s) return;
  for (int k = 0; k < s->nsol; k++) {
    free(s->sol[k].dir);
    free(s->sol[k].dV);
    free(s->sol[k].Fm);
  }
  free(s->f);
  free(s->fpost);
  free(s->inside);
  free(s->inside_prev);
  free(s->fibm);
  free(s->usnap);
  free(s->fprev);
  free(s);
}

/* separation of node n from the centre of solid k, nearest image */
static void rel(const ora_sim *s, const solid_t *b, double x, double y,
                double z, double r[3]) {
  r[0] = mimage(x - b->c[0], s->nx);
  r[1] = mimage(y - b->c[1], s->ny);
  r[2] = s->d == 2 ? 0 : mimage(z - b->c[2], s->nz);
  if (b->kind == ORA_CYLINDER_Z) r[2] = 0;
}

/* inside the solid region (node exactly on the surface counts as solid) */
static int in_solid(const ora_sim *s, const solid_t *b, long n) {
  long x, y, z;
  coords(s, n, &x, &y, &z);
  double r[3];
  rel(s, b, (double)x, (double)y, (double)z, r);
  double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  return b->fluid_inside ? r2 >= b->R * b->R : r2 <= b->R * b->R;
}

static void compute_inside(ora_sim *s, int *ins) {
  for (long n = 0; n < s->N; n++) {
    ins[n] = 0;
    if (s->scheme == ORA_NONE) continue;
    for (int k = 0; k < s->nsol; k++)
      if (in_solid(s, &s->sol[k], n)) {
        ins[n] = k + 1;
        break;
      }
  }
}

static void build_markers(ora_sim *s, solid_t *b) {
  free(b->dir);
  free(b->dV);
  free(b->Fm);
  b->dir = b->dV = b->Fm = NULL;
  b->nm = 0;
  if (s->scheme != ORA_IBM) return;
  double RL = b->fluid_inside ? b->R + s->retraction : b->R - s->retraction;
  const double pi = 3.14159265358979323846;
  if (s->d == 3 && b->kind == ORA_SPHERE) {
    double area = 4 * pi * RL * RL;
    int n = (int)round(s->density * area);
    if (n < 1) n = 1;
    b->nm = n;
    b->dir = (double *)calloc(3 * (size_t)n, sizeof(double));
    b->dV = (double *)calloc((size_t)n, sizeof(double));
    double ga = pi * (3 - sqrt(5.0));
    for (int k = 0; k < n; k++) {
      double zz = 1 - (2.0 * k + 1) / n;
      double rr = sqrt(1 - zz * zz);
      b->dir[k] = rr * cos(ga * k);
      b->dir[n + k] = rr * sin(ga * k);
      b->dir[2 * n + k] = zz;
      b->dV[k] = area / n;
    }
  } else {
    /* circle on a 2D lattice, or one ring of markers per z-plane for a
     * cylinder along z on a 3D lattice */
    double circ = 2 * pi * RL;
    int per = (int)round(s->density * circ);
    if (per < 1) per = 1;
    int rings = s->d == 3 ? s->nz : 1;
    int n = per * rings;
    b->nm = n;
    b->dir = (double *)calloc(3 * (size_t)n, sizeof(double));
    b->dV = (double *)calloc((size_t)n, sizeof(double));
    for (int r = 0; r < rings; r++)
      for (int k = 0; k < per; k++) {
        int m = r * per + k;
        double th = 2 * pi * k / per;
        b->dir[m] = cos(th);
        b->dir[n + m] = sin(th);
        b->dir[2 * n + m] = r; /* plane index, not a direction */
        b->dV[m] = circ / per;
      }
  }
  b->Fm = (double *)calloc(3 * (size_t)b->nm, sizeof(double));
}

static void marker_pos(const ora_sim *s, const solid_t *b, int m,
                       double X[3]) {
  double RL = b->fluid_inside ? b->R + s->retraction : b->R - s->retraction;
  int n = b->nm;
  X[0] = b->c[0] + RL * b->dir[m];
  X[1] = b->c[1] + RL * b->dir[n + m];
  if (s->d == 2)
    X[2] = 0;
  else if (b->kind == ORA_CYLINDER_Z)
    X[2] = b->dir[2 * n + m];
  else
    X[2] = b->c[2] + RL * b->dir[2 * n + m];
}

int ora_add_solid(ora_sim *s, int kind, const double c[3], double R,
                  const double U[3], const double Om[3], int fluid_inside) {
  if (s->nsol >= MAXS) return -1;
  solid_t *b = &s->sol[s->nsol];
  memset(b, 0, sizeof(*b));
  b->kind = kind;
  b->fluid_inside = fluid_inside;
  b->R = R;
  for (int a = 0; a < 3; a++) {
    b->c[a] = b->c0[a] = c[a];
    b->U[a] = U ? U[a] : 0;
    b->Om[a] = Om ? Om[a] : 0;
  }
  if (s->d == 2) {
    b->c[2] = b->c0[2] = 0;
    b->U[2] = 0;
    b->Om[0] = b->Om[1] = 0;
  }
  s->nsol++;
  build_markers(s, b);
  compute_inside(s, s->inside);
  s->have_prev = 0;
  return s->nsol - 1;
}

void ora_set_scheme(ora_sim *s, int scheme, int ibm_iters, double retraction,
                    double marker_density) {
  s->scheme = scheme;
  s->ibm_iters = ibm_iters < 1 ? 1 : ibm_iters;
  s->retraction = retraction;
  s->density = marker_density > 0 ? marker_density : 1;
  for (int k = 0; k < s->nsol; k++) build_markers(s, &s->sol[k]);
  compute_inside(s, s->inside);
  s->have_prev = 0;
}

void ora_set_ibm_inertia(ora_sim *s, int inertia) {
  s->ibm_inertia = (inertia == ORA_INERTIA_KEMPE || inertia == ORA_INERTIA_UHLMANN)
                       ? inertia : ORA_INERTIA_FENG;
  for (int k = 0; k < s->nsol; k++) s->sol[k].have_Ip = 0;
}

void ora_set_ibm_kernel(ora_sim *s, int kernel) {
  s->ibm_kernel = (kernel >= ORA_DELTA_PESKIN4 && kernel <= ORA_DELTA_COSINE4) ? kernel
                                                                               : ORA_DELTA_PESKIN4;
}

static int simulated(const ora_sim *s, long n) {
  return !(is_ibb(s->scheme) && s->inside[n]);
}

void ora_init_equilibrium(ora_sim *s, double rho, const double u[3]) {
  double feq[MAXQ], uu[3] = {u[0], u[1], s->d == 2 ? 0 : u[2]};
  ora_equilibrium(s->lattice, rho, uu, feq);
  for (int i = 0; i < s->Q; i++)
    for (long n = 0; n < s->N; n++) s->f[(long)i * s->N + n] = feq[i];
}

void ora_set_f(ora_sim *s, const double *f) {
  memcpy(s->f, f, sizeof(double) * (size_t)s->Q * s->N);
}
void ora_get_f(const ora_sim *s, double *f) {
  memcpy(f, s->f, sizeof(double) * (size_t)s->Q * s->N);
}

/* external force at a node: g on nodes outside every solid (reading of the
 * "fluid region only" variant of Sec. 3.3), or everywhere if force_all */
static void gext(const ora_sim *s, long n, double F[3]) {
  int on = s->force_all || s->inside[n] == 0;
  for (int a = 0; a < 3; a++) F[a] = on ? s->g[a] : 0;
}

static void wall_velocity(const solid_t *b, const double r[3], double uw[3]) {
  /* U + Omega x r */
  uw[0] = b->U[0] + b->Om[1] * r[2] - b->Om[2] * r[1];
  uw[1] = b->U[1] + b->Om[2] * r[0] - b->Om[0] * r[2];
  uw[2] = b->U[2] + b->Om[0] * r[1] - b->Om[1] * r[0];
}

/* ---- immersed boundary (Sec. 2.1, Eqs. 4-9) ---- */
static double delta_w(int kernel, int d, const double r[3]) {
  double v = ora_phi_kernel(kernel, r[0]) * ora_phi_kernel(kernel, r[1]);
  return d == 3 ? v * ora_phi_kernel(kernel, r[2]) : v;
}

void ora_ibm_interp_k(int kernel, int d, int nx, int ny, int nz, const double *u, int n,
                      const double *X, double *U) {
  long N = (long)nx * ny * (d == 3 ? nz : 1);
  for (int m = 0; m < n; m++) {
    double Xm[3] = {X[m], X[n + m], d == 3 ? X[2 * n + m] : 0};
    long b[3];
    for (int a = 0; a < 3; a++) b[a] = (long)floor(Xm[a]) - 1;
    for (int a = 0; a < d; a++) U[a * n + m] = 0;
    int kz_n = d == 3 ? 4 : 1;
    for (int kz = 0; kz < kz_n; kz++)
      for (int ky = 0; ky < 4; ky++)
        for (int kx = 0; kx < 4; kx++) {
          double r[3] = {b[0] + kx - Xm[0], b[1] + ky - Xm[1],
                         d == 3 ? b[2] + kz - Xm[2] : 0};
          double wgt = delta_w(kernel, d, r);
          long nn = wrapi(b[0] + kx, nx) +
                    nx * (wrapi(b[1] + ky, ny) +
                          ny * (d == 3 ? wrapi(b[2] + kz, nz) : 0));
          for (int a = 0; a < d; a++) U[a * n + m] += u[a * N + nn] * wgt;
        }
  }
}

void ora_ibm_spread_k(int kernel, int d, int nx, int ny, int nz, double *f, int n,
                      const double *X, const double *F, const double *dV) {
  long N = (long)nx * ny * (d == 3 ? nz : 1);
  for (int m = 0; m < n; m++) {
    double Xm[3] = {X[m], X[n + m], d == 3 ? X[2 * n + m] : 0};
    long b[3];
    for (int a = 0; a < 3; a++) b[a] = (long)floor(Xm[a]) - 1;
    int kz_n = d == 3 ? 4 : 1;
    for (int kz = 0; kz < kz_n; kz++)
      for (int ky = 0; ky < 4; ky++)
        for (int kx = 0; kx < 4; kx++) {
          double r[3] = {b[0] + kx - Xm[0], b[1] + ky - Xm[1],
                         d == 3 ? b[2] + kz - Xm[2] : 0};
          double wgt = delta_w(kernel, d, r);
          long nn = wrapi(b[0] + kx, nx) +
                    nx * (wrapi(b[1] + ky, ny) +
                          ny * (d == 3 ? wrapi(b[2] + kz, nz) : 0));
          for (int a = 0; a < d; a++) f[a * N + nn] += F[a * n + m] * wgt * dV[m];
        }
  }
}

void ora_ibm_interp(int d, int nx, int ny, int nz, const double *u, int n,
                    const double *X, double *U) {
  ora_ibm_interp_k(ORA_DELTA_PESKIN4, d, nx, ny, nz, u, n, X, U);
}

void ora_ibm_spread(int d, int nx, int ny, int nz, double *f, int n,
                    const double *X, const double *F, const double *dV) {
  ora_ibm_spread_k(ORA_DELTA_PESKIN4, d, nx, ny, nz, f, n, X, F, dV);
}

/* The IB-LBM variant examined in Sec. 2.1: before the collision of step t,
 * interpolate the unforced velocity (external half force only, no IBM half
 * force) to the markers, F = rho0 (U^d - U~)/dt (Eq. 7), spread it (Eq. 8);
 * extra iterations re-interpolate u~ + f dt/rho0 and add the correction
 * (Eq. 9 applied to the spread force).  Force and torque on the solid are
 * minus the sum of marker forces times dV (Eq. 45 / Sec. 3.1). */
static void ibm_forces(ora_sim *s) {
  long N = s->N;
  int d = s->d;
  for (long k = 0; k < 3 * N; k++) s->fibm[k] = 0;
  if (s->scheme != ORA_IBM || s->nsol == 0) return;
  double *ut = (double *)calloc((size_t)3 * N, sizeof(double));
  double *uc = (double *)calloc((size_t)3 * N, sizeof(double));
  double *X[MAXS], *Ud[MAXS], *Ui[MAXS];
  for (long n = 0; n < N; n++) {
    double j[3] = {0, 0, 0}, G[3];
    for (int i = 0; i < s->Q; i++)
      for (int a = 0; a < 3; a++) j[a] += s->f[(long)i * N + n] * s->e[i][a];
    gext(s, n, G);
    for (int a = 0; a < d; a++) ut[a * N + n] = (j[a] + 0.5 * G[a]) / RHO0;
  }
  for (int k = 0; k < s->nsol; k++) {
    solid_t *b = &s->sol[k];
    int nm = b->nm;
    X[k] = (double *)calloc(3 * (size_t)nm, sizeof(double));
    Ud[k] = (double *)calloc(3 * (size_t)nm, sizeof(double));
    Ui[k] = (double *)calloc(3 * (size_t)nm, sizeof(double));
    for (int m = 0; m < nm; m++) {
      double Xm[3], r[3], uw[3];
      marker_pos(s, b, m, Xm);
      for (int a = 0; a < 3; a++) {
        X[k][a * nm + m] = Xm[a];
        r[a] = Xm[a] - b->c[a];
      }
      if (b->kind == ORA_CYLINDER_Z || d == 2) r[2] = 0;
      wall_velocity(b, r, uw);
      for (int a = 0; a < 3; a++) Ud[k][a * nm + m] = uw[a];
    }
    for (int a = 0; a < 3 * nm; a++) b->Fm[a] = 0;
  }
  for (int it = 0; it < s->ibm_iters; it++) {
    /* velocity seen by the markers: u~ + f dt / rho0 (f = 0 at it = 0) */
    for (int a = 0; a < d; a++)
      for (long n = 0; n < N; n++)
        uc[a * N + n] = ut[a * N + n] + s->fibm[a * N + n] / RHO0;
    for (int k = 0; k < s->nsol; k++) {
      solid_t *b = &s->sol[k];
      int nm = b->nm;
      ora_ibm_interp_k(s->ibm_kernel, d, s->nx, s->ny, s->nz, uc, nm, X[k], Ui[k]);
      for (int a = 0; a < d; a++)
        for (int m = 0; m < nm; m++)
          b->Fm[a * nm + m] += RHO0 * (Ud[k][a * nm + m] - Ui[k][a * nm + m]);
    }
    /* Eulerian force = spread of the accumulated marker forces (Eq. 8) */
    for (long q = 0; q < 3 * N; q++) s->fibm[q] = 0;
    for (int k = 0; k < s->nsol; k++)
      ora_ibm_spread_k(s->ibm_kernel, d, s->nx, s->ny, s->nz, s->fibm, s->sol[k].nm, X[k],
                       s->sol[k].Fm, s->sol[k].dV);
  }
  for (int k = 0; k < s->nsol; k++) {
    solid_t *b = &s->sol[k];
    int nm = b->nm;
    for (int a = 0; a < 3; a++) b->F[a] = b->T[a] = 0;
    for (int m = 0; m < nm; m++) {
      double Fm[3] = {b->Fm[m], b->Fm[nm + m], d == 3 ? b->Fm[2 * nm + m] : 0};
      double r[3] = {X[k][m] - b->c[0], X[k][nm + m] - b->c[1],
                     d == 3 ? X[k][2 * nm + m] - b->c[2] : 0};
      if (b->kind == ORA_CYLINDER_Z) r[2] = 0;
      for (int a = 0; a < 3; a++) b->F[a] -= Fm[a] * b->dV[m];
      b->T[0] -= (r[1] * Fm[2] - r[2] * Fm[1]) * b->dV[m];
      b->T[1] -= (r[2] * Fm[0] - r[0] * Fm[2]) * b->dV[m];
      b->T[2] -= (r[0] * Fm[1] - r[1] * Fm[0]) * b->dV[m];
    }
    free(X[k]);
    free(Ud[k]);
    free(Ui[k]);
  }
  free(ut);
  free(uc);
}

/* Geometry at the current solid positions; nodes uncovered since the last
 * call are refilled (bounce-back schemes only, Sec. 3.2 mentions refilling,
 * formula is a reading, pinned by the co-moving uniform flow). */
static void update_geometry(ora_sim *s) {
  memcpy(s->inside_prev, s->inside, sizeof(int) * (size_t)s->N);
  compute_inside(s, s->inside);
  if (!s->have_prev || !is_ibb(s->scheme)) {
    s->have_prev = 1;
    return;
  }
  long N = s->N;
  for (long n = 0; n < N; n++) {
    if (!(s->inside_prev[n] && !s->inside[n])) continue;
    long x, y, z;
    coords(s, n, &x, &y, &z);
    double rs = 0;
    int cnt = 0;
    for (int i = 1; i < s->Q; i++) {
      long nb = node(s, x + s->e[i][0], y + s->e[i][1], z + s->e[i][2]);
      if (s->inside[nb] || s->inside_prev[nb]) continue;
      double r = 0;
      for (int k = 0; k < s->Q; k++) r += s->f[(long)k * N + nb];
      rs += r;
      cnt++;
    }
    double rho = cnt ? rs / cnt : RHO0;
    solid_t *b = &s->sol[s->inside_prev[n] - 1];
    double r[3], uw[3], feq[MAXQ];
    rel(s, b, (double)x, (double)y, (double)z, r);
    wall_velocity(b, r, uw);
    if (s->d == 2) uw[2] = 0;
    ora_equilibrium(s->lattice, rho, uw, feq);
    for (int i = 0; i < s->Q; i++) s->f[(long)i * N + n] = feq[i];
  }
}

/* Wall fraction q = |x_f - x_w| / |x_f - x_b| along the link from x_f
 * towards x_b = x_f - e_i (Fig. 1 / Sec. 2.2). */
static double link_q(const ora_sim *s, const solid_t *b, long nf, int i) {
  long x, y, z;
  coords(s, nf, &x, &y, &z);
  double r[3];
  rel(s, b, (double)x, (double)y, (double)z, r);
  double dvec[3] = {-(double)s->e[i][0], -(double)s->e[i][1],
                    -(double)s->e[i][2]};
  if (b->kind == ORA_CYLINDER_Z || s->d == 2) dvec[2] = 0;
  double A = 0, B = 0, C = -b->R * b->R;
  for (int a = 0; a < 3; a++) {
    A += dvec[a] * dvec[a];
    B += 2 * r[a] * dvec[a];
    C += r[a] * r[a];
  }
  if (A == 0) return 0.5;
  double D = B * B - 4 * A * C;
  if (D < 0) D = 0;
  double q = b->fluid_inside ? (-B + sqrt(D)) / (2 * A) : (-B - sqrt(D)) / (2 * A);
  if (q > 1) q = 1;
  if (q < 1e-12) q = 1e-12;
  return q;
}

/* Volume and moment of inertia (about the centre, the z axis for cylinders)
 * per unit solid density: a sphere 4/3 pi R^3 and 2/5 R^2 of its mass, a
 * cylinder pi R^2 times its length (1 in 2D, nz along z in 3D) and 1/2 R^2. */
static void solid_volume(const ora_sim *s, const solid_t *b, double *V, double *Ir2) {
  const double pi = 3.14159265358979323846;
  if (s->d == 2 || b->kind == ORA_CYLINDER_Z) {
    *V = pi * b->R * b->R * (s->d == 2 ? 1.0 : (double)s->nz);
    *Ir2 = 0.5 * b->R * b->R;
  } else {
    *V = 4.0 / 3.0 * pi * b->R * b->R * b->R;
    *Ir2 = 0.4 * b->R * b->R;
  }
}

static void node_velocity(const ora_sim *s, long n, double u[3], double F[3]);
static void current_forces(ora_sim *s);

/* Fraction of the cell around node (x, y, z) inside solid b (Eq. 25):
 * sum over the cell's corners (x +- 1/2, ...; 8 in 3D, 4 in 2D) of
 * -phi H(-phi) over the sum of |phi|, with the signed distance function of
 * Eq. 26 for a sphere (a = b = c = R) or a circle / z-cylinder (the z term
 * dropped). */
static double cell_fraction(const ora_sim *s, const solid_t *b, long x, long y, long z) {
  const int flat = s->d == 2 || b->kind == ORA_CYLINDER_Z;
  double num = 0, den = 0;
  for (int c = 0; c < (s->d == 2 ? 4 : 8); c++) {
    double r[3];
    rel(s, b, x + ((c & 1) ? 0.5 : -0.5), y + ((c & 2) ? 0.5 : -0.5),
        z + ((c & 4) ? 0.5 : -0.5), r);
    if (flat) r[2] = 0;
    const double phi = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) / b->R - 1;
    if (phi < 0) num += -phi;
    den += fabs(phi);
  }
  return den > 0 ? num / den : 0;
}

/* Eq. 24: the fluid momentum and angular momentum inside solid b,
 * sum over nodes of u alpha and r x u alpha (h = 1), u the velocity at the
 * current time (with this step's forces) and r the node's separation from
 * the centre. */
static void internal_fluid(const ora_sim *s, const solid_t *b, double I[6]) {
  for (int k = 0; k < 6; k++) I[k] = 0;
  for (long n = 0; n < s->N; n++) {
    long x, y, z;
    coords(s, n, &x, &y, &z);
    const double al = cell_fraction(s, b, x, y, z);
    if (al == 0) continue;
    double u[3], F[3], r[3];
    node_velocity(s, n, u, F);
    if (s->d == 2) u[2] = 0;
    rel(s, b, (double)x, (double)y, (double)z, r);
    if (s->d == 2 || b->kind == ORA_CYLINDER_Z) r[2] = 0;
    for (int a = 0; a < 3; a++) I[a] += al * u[a];
    I[3] += al * (r[1] * u[2] - r[2] * u[1]);
    I[4] += al * (r[2] * u[0] - r[0] * u[2]);
    I[5] += al * (r[0] * u[1] - r[1] * u[0]);
  }
}

double ora_cell_fraction(ora_sim *s, int id, long x, long y, long z) {
  return cell_fraction(s, &s->sol[id], x, y, z);
}

void ora_internal_fluid(ora_sim *s, int id, double I[6]) {
  current_forces(s);
  internal_fluid(s, &s->sol[id], I);
}

/* New velocities of a free solid from this step's hydrodynamic force and
 * torque (dt = 1, rho_f = rho0):
 *  - bounce-back (Eq. 20): rho_p V dv = F + (rho_p - rho_f) V g, I dw = T;
 *  - IBM (Eq. 23): rho_p V dv = rho_f V (v - v_prev) + F + (rho_p - rho_f) V g,
 *    I dw = I (rho_f / rho_p)(w - w_prev) + T.
 * Cylinders turn about z only. */
static void free_motion(const ora_sim *s, const solid_t *b, const double Inow[6], double Un[3],
                        double On[3]) {
  double V, Ir2;
  solid_volume(s, b, &V, &Ir2);
  const double m = b->rho_p * RHO0 * V, I = m * Ir2;
  const int ibm = s->scheme == ORA_IBM;
  for (int a = 0; a < 3; a++) {
    double dv = b->F[a] + (b->rho_p - 1.0) * RHO0 * V * b->g[a];
    double dw = b->T[a];
    if (ibm && s->ibm_inertia == ORA_INERTIA_UHLMANN) {
      /* Eq. 22: the inside fluid moves rigidly with the solid and its inertia
       * is taken off the solid's: (rho_p - rho_f) V dv = F + (rho_p - rho_f) V g,
       * I (1 - rho_f / rho_p) dw = T */
      Un[a] = b->U[a] + dv / ((b->rho_p - 1.0) * RHO0 * V);
      On[a] = b->Om[a] + dw / (I * (1.0 - 1.0 / b->rho_p));
      continue;
    }
    if (ibm && s->ibm_inertia == ORA_INERTIA_KEMPE) {
      /* Eq. 21 with Eq. 24: rho_f times the change of the inside fluid's
       * momentum (angular momentum) over the last step */
      dv += RHO0 * (Inow[a] - b->Ip[a]);
      dw += RHO0 * (Inow[3 + a] - b->Ip[3 + a]);
    } else if (ibm) {
      dv += RHO0 * V * (b->U[a] - b->Up[a]);
      dw += I / b->rho_p * (b->Om[a] - b->Omp[a]);
    }
    Un[a] = b->U[a] + dv / m;
    On[a] = b->Om[a] + dw / I;
  }
  if (s->d == 2) Un[2] = 0;
  if (s->d == 2 || b->kind == ORA_CYLINDER_Z) On[0] = On[1] = 0;
}

/* ---- domain faces (Sec. 3.4: uniform flow past a sphere) ----
 * A non-periodic face lies half a spacing outside the outermost nodes.  A
 * pull from (x, y, z) along e_i that leaves the domain crosses one face, or
 * two at an edge; bit 2a marks the low face of axis a, bit 2a + 1 the high
 * one. */
static int crossed(const ora_sim *s, long x, long y, long z, int i) {
  const long src[3] = {x - s->e[i][0], y - s->e[i][1], z - s->e[i][2]};
  const long len[3] = {s->nx, s->ny, s->nz};
  int m = 0;
  for (int a = 0; a < s->d; a++) {
    if (src[a] < 0 && s->face[2 * a] != ORA_FACE_PERIODIC) m |= 1 << (2 * a);
    if (src[a] >= len[a] && s->face[2 * a + 1] != ORA_FACE_PERIODIC) m |= 1 << (2 * a + 1);
  }
  return m;
}

/* whether x - k e_i lies beyond a non-periodic face (k < 0: downstream) */
static int crossed_at(const ora_sim *s, long x, long y, long z, int i, int k) {
  if (!s->open) return 0;
  const long p[3] = {x - k * s->e[i][0], y - k * s->e[i][1], z - k * s->e[i][2]};
  const long len[3] = {s->nx, s->ny, s->nz};
  for (int a = 0; a < s->d; a++) {
    if (p[a] < 0 && s->face[2 * a] != ORA_FACE_PERIODIC) return 1;
    if (p[a] >= len[a] && s->face[2 * a + 1] != ORA_FACE_PERIODIC) return 1;
  }
  return 0;
}

static int crosses_type(const ora_sim *s, int m, int type) {
  for (int k = 0; k < 6; k++)
    if (((m >> k) & 1) && s->face[k] == type) return k;
  return -1;
}

static void domain_abort(const char *what) {
  fprintf(stderr, "oracle: %s\n", what);
  abort();
}

/* f_i(x, t+1) when the pull along e_i leaves through velocity or free-slip
 * faces only:
 *  - a velocity face is a plane wall moving with its velocity u_f: the
 *    population bounces back at the node, f_i = f*_ib + 2 rho0 w_i e_i.u_f
 *    / cs^2 (the moving-wall term of the bounce-back rules, q = 1/2);
 *  - free-slip faces reflect specularly: the value is f*_r at the node that
 *    keeps x's coordinates on the crossed axes and x - e_i's on the others,
 *    r being e_i with its crossed components reversed (no normal velocity
 *    and no shear stress at the face: the stress-free condition). */
static double wall_pull(const ora_sim *s, long x, long y, long z, int i, int m) {
  const long N = s->N;
  const int vf = crosses_type(s, m, ORA_FACE_VELOCITY);
  if (vf >= 0) {
    const double *u = s->u_face[vf];
    const double eu = s->e[i][0] * u[0] + s->e[i][1] * u[1] + s->e[i][2] * u[2];
    return s->fpost[(long)s->opp[i] * N + node(s, x, y, z)] + 2 * RHO0 * s->w[i] * eu / CS2;
  }
  int r[3] = {s->e[i][0], s->e[i][1], s->e[i][2]};
  long src[3] = {x - s->e[i][0], y - s->e[i][1], z - s->e[i][2]};
  const long at[3] = {x, y, z};
  for (int a = 0; a < 3; a++)
    if ((m >> (2 * a)) & 3) {
      r[a] = -r[a];
      src[a] = at[a];
    }
  int j = -1;
  for (int k = 0; k < s->Q; k++)
    if (s->e[k][0] == r[0] && s->e[k][1] == r[1] && s->e[k][2] == r[2]) j = k;
  const long n = node(s, src[0], src[1], src[2]);
  if (j < 0 || !simulated(s, n)) domain_abort("solid too close to a free-slip face");
  return s->fpost[(long)j * N + n];
}

/* f_i(x, t+1) of plain streaming, or through velocity / free-slip faces. */
static double side_pull(const ora_sim *s, long x, long y, long z, int i) {
  const int m = crossed(s, x, y, z, i);
  if (m == 0) {
    const long n = node(s, x - s->e[i][0], y - s->e[i][1], z - s->e[i][2]);
    if (!simulated(s, n)) domain_abort("solid too close to an outflow face");
    return s->fpost[(long)i * s->N + n];
  }
  if (crosses_type(s, m, ORA_FACE_CONVECTIVE) >= 0) domain_abort("two outflow faces meet");
  return wall_pull(s, x, y, z, i, m);
}

/* f_i(x, t+1) at a node whose pull along e_i leaves the domain (m != 0).
 * A velocity face decides first, then an outflow face, then free slip.  At
 * an outflow face with outward normal n the convective condition
 * d(rho0 u)/dt + U_o d(rho0 u)/dn = 0 is imposed on each unknown population,
 * upwind in space and implicit in the neighbour:
 *   f_i(x, t+1) = [f_i(x, t) + U_o f_i(x - n, t+1)] / (1 + U_o),
 * U_o = max(0, u(x, t).n), the outward velocity at the node at time t. */
static double face_value(const ora_sim *s, long n, long x, long y, long z, int i, int m) {
  if (crosses_type(s, m, ORA_FACE_VELOCITY) >= 0) return wall_pull(s, x, y, z, i, m);
  const int cf = crosses_type(s, m, ORA_FACE_CONVECTIVE);
  if (cf < 0) return wall_pull(s, x, y, z, i, m);
  const int a = cf / 2;
  const int sg = (cf & 1) ? 1 : -1;
  long in[3] = {x, y, z};
  in[a] -= sg;
  const double vin = side_pull(s, in[0], in[1], in[2], i);
  double j = 0, F[3];
  for (int k = 0; k < s->Q; k++) j += s->fprev[(long)k * s->N + n] * s->e[k][a];
  gext(s, n, F);
  F[a] += s->fibm[a * s->N + n];
  double U = sg * (j + 0.5 * F[a]) / RHO0;
  if (U < 0) U = 0;
  return (s->fprev[(long)i * s->N + n] + U * vin) / (1 + U);
}

int ora_set_domain(ora_sim *s, const int face[6], const double *u_face) {
  for (int k = 0; k < 6; k++) {
    const int t = face ? face[k] : ORA_FACE_PERIODIC;
    if (t < ORA_FACE_PERIODIC || t > ORA_FACE_CONVECTIVE) return -1;
    if (k >= 2 * s->d && t != ORA_FACE_PERIODIC) return -1;
  }
  int conv = 0;
  for (int a = 0; a < 3; a++) {
    const int lo = face ? face[2 * a] : 0, hi = face ? face[2 * a + 1] : 0;
    if ((lo == ORA_FACE_PERIODIC) != (hi == ORA_FACE_PERIODIC)) return -1;
    conv += (lo == ORA_FACE_CONVECTIVE) + (hi == ORA_FACE_CONVECTIVE);
  }
  if (conv > 1) return -1;
  s->open = 0;
  for (int k = 0; k < 6; k++) {
    s->face[k] = face ? face[k] : ORA_FACE_PERIODIC;
    s->open |= s->face[k] != ORA_FACE_PERIODIC;
    for (int a = 0; a < 3; a++) s->u_face[k][a] = u_face ? u_face[3 * k + a] : 0;
    if (s->d == 2) s->u_face[k][2] = 0;
  }
  if (conv && !s->fprev) s->fprev = (double *)calloc((size_t)s->Q * s->N, sizeof(double));
  return 0;
}

/* Collision at every simulated node, then streaming (pull of post-collision
 * values) with the interpolated bounce-back rule on links whose upstream
 * node is solid, accumulating the momentum exchange of Eq. 17. */
static void one_step(ora_sim *s) {
  long N = s->N;
  int Q = s->Q;
  update_geometry(s);
  ibm_forces(s);
  if (s->scheme == ORA_IBM && s->ibm_inertia == ORA_INERTIA_KEMPE)
    for (int k = 0; k < s->nsol; k++)
      if (s->sol[k].free_) internal_fluid(s, &s->sol[k], s->sol[k].In);
  /* collision */
  for (long n = 0; n < N; n++) {
    if (!simulated(s, n)) continue;
    double fl[MAXQ], fo[MAXQ], F[3];
    for (int i = 0; i < Q; i++) fl[i] = s->f[(long)i * N + n];
    gext(s, n, F);
    for (int a = 0; a < 3; a++) F[a] += s->fibm[a * N + n];
    collide_with(&s->coll, fl, F, fo);
    for (int i = 0; i < Q; i++) s->fpost[(long)i * N + n] = fo[i];
  }
  if (is_ibb(s->scheme))
    for (int k = 0; k < s->nsol; k++)
      for (int a = 0; a < 3; a++) s->sol[k].F[a] = s->sol[k].T[a] = 0;
  /* streaming (outflow faces read the pre-collision populations of time t) */
  if (s->fprev) memcpy(s->fprev, s->f, sizeof(double) * (size_t)Q * N);
  for (long n = 0; n < N; n++) {
    if (!simulated(s, n)) continue;
    long x, y, z;
    coords(s, n, &x, &y, &z);
    /* this node's pre-collision values f(t), before streaming replaces them
     * (Eq. 16 uses the one travelling towards the wall) */
    double fpre[MAXQ];
    for (int i = 0; i < Q; i++) fpre[i] = s->f[(long)i * N + n];
    for (int i = 0; i < Q; i++) {
      const int m = s->open ? crossed(s, x, y, z, i) : 0;
      if (m) {
        s->f[(long)i * N + n] = face_value(s, n, x, y, z, i, m);
        continue;
      }
      long src = node(s, x - s->e[i][0], y - s->e[i][1], z - s->e[i][2]);
      if (simulated(s, src)) {
        s->f[(long)i * N + n] = s->fpost[(long)i * N + src];
        continue;
      }
      /* cut link: x_b = src is solid */
      int ib = s->opp[i];
      solid_t *b = &s->sol[s->inside[src] - 1];
      long nff = node(s, x + s->e[i][0], y + s->e[i][1], z + s->e[i][2]);
      long nfff =
          node(s, x + 2 * s->e[i][0], y + 2 * s->e[i][1], z + 2 * s->e[i][2]);
      /* a stencil node beyond a non-periodic face does not exist */
      int hff = !crossed_at(s, x, y, z, i, -1) && simulated(s, nff);
      int hfff = hff && !crossed_at(s, x, y, z, i, -2) && simulated(s, nfff);
      double q = link_q(s, b, n, i), c[6];
      int used = s->scheme == ORA_ZHAO_YONG ? ORA_ZHAO_YONG
                                            : ora_ibb_coeffs(s->scheme, q, hff, hfff, c);
      s->link_counts[used]++;
      double r[3], xw[3], uw[3];
      rel(s, b, (double)x, (double)y, (double)z, r);
      for (int a = 0; a < 3; a++) xw[a] = r[a] - q * s->e[i][a];
      if (b->kind == ORA_CYLINDER_Z || s->d == 2) xw[2] = 0;
      wall_velocity(b, xw, uw);
      if (s->d == 2) uw[2] = 0;
      double eu = s->e[i][0] * uw[0] + s->e[i][1] * uw[1] + s->e[i][2] * uw[2];
      double fin;
      if (s->scheme == ORA_ZHAO_YONG) {
        /* Eq. 16 as printed: the post-collision value leaving the wall at
         * x_f, the pre-collision value arriving at x_f towards the wall, and
         * the moving-wall term, weighted 2q, 1 and 2 over 1 + 2q */
        fin = (2 * q * s->fpost[(long)i * N + n] + fpre[ib] + 2 * RHO0 * s->w[i] * eu / CS2) /
              (1 + 2 * q);
      } else {
        fin = c[0] * s->fpost[(long)ib * N + n] +
              (c[1] != 0 ? c[1] * s->fpost[(long)ib * N + nff] : 0) +
              (c[2] != 0 ? c[2] * s->fpost[(long)ib * N + nfff] : 0) +
              (c[3] != 0 ? c[3] * s->fpost[(long)i * N + n] : 0) +
              (c[4] != 0 ? c[4] * s->fpost[(long)i * N + nff] : 0) +
              c[5] * 2 * RHO0 * s->w[i] * eu / CS2;
      }
      s->f[(long)i * N + n] = fin;
      /* Eq. 17: F dt += f*_ib (e_ib - u_w) - f_i(t+1) (e_i - u_w) */
      double fs = s->fpost[(long)ib * N + n], dp[3];
      for (int a = 0; a < 3; a++)
        dp[a] = fs * (s->e[ib][a] - uw[a]) - fin * (s->e[i][a] - uw[a]);
      if (s->d == 2) dp[2] = 0;
      for (int a = 0; a < 3; a++) b->F[a] += dp[a];
      b->T[0] += xw[1] * dp[2] - xw[2] * dp[1];
      b->T[1] += xw[2] * dp[0] - xw[0] * dp[2];
      b->T[2] += xw[0] * dp[1] - xw[1] * dp[0];
    }
  }
  /* motion: prescribed, X(t+1) = X(t) + U dt; or free, new velocities from
   * this step's force and torque, then X(t+1) = X(t) + (U(t) + U(t+1))/2 */
  for (int k = 0; k < s->nsol; k++) {
    solid_t *b = &s->sol[k];
    if (b->free_) {
      double Un[3], On[3], Inow[6] = {0, 0, 0, 0, 0, 0};
      if (s->scheme == ORA_IBM && s->ibm_inertia == ORA_INERTIA_KEMPE) {
        /* Eq. 24 at time n, taken after ibm_forces and before the
         * streaming replaced f */
        for (int a = 0; a < 6; a++) Inow[a] = b->In[a];
        if (!b->have_Ip)
          for (int a = 0; a < 6; a++) b->Ip[a] = Inow[a];
      }
      free_motion(s, b, Inow, Un, On);
      if (s->scheme == ORA_IBM && s->ibm_inertia == ORA_INERTIA_KEMPE) {
        for (int a = 0; a < 6; a++) b->Ip[a] = Inow[a];
        b->have_Ip = 1;
      }
      for (int a = 0; a < 3; a++) {
        b->c[a] += 0.5 * (b->U[a] + Un[a]);
        b->Up[a] = b->U[a];
        b->Omp[a] = b->Om[a];
        b->U[a] = Un[a];
        b->Om[a] = On[a];
      }
    } else {
      for (int a = 0; a < 3; a++) b->c[a] += b->U[a];
    }
  }
  s->steps++;
}

void ora_step(ora_sim *s, int nsteps) {
  for (int k = 0; k < nsteps; k++) one_step(s);
}

/* The force field at the current time (external + IBM).  Under IBM the
 * markers and the forcing region follow the solids to the current time, as
 * the next step would see them; under bounce-back the geometry stays that of
 * the most recent streaming (the nodes that carry distributions). */
static void current_forces(ora_sim *s) {
  if (s->scheme == ORA_IBM) compute_inside(s, s->inside);
  ibm_forces(s);
}

void ora_density(ora_sim *s, double *rho) {
  current_forces(s);
  for (long n = 0; n < s->N; n++) {
    rho[n] = 0;
    if (!simulated(s, n)) continue;
    for (int i = 0; i < s->Q; i++) rho[n] += s->f[(long)i * s->N + n];
  }
}

static void node_velocity(const ora_sim *s, long n, double u[3], double F[3]) {
  double j[3] = {0, 0, 0};
  for (int i = 0; i < s->Q; i++)
    for (int a = 0; a < 3; a++) j[a] += s->f[(long)i * s->N + n] * s->e[i][a];
  gext(s, n, F);
  for (int a = 0; a < 3; a++) {
    F[a] += s->fibm[a * s->N + n];
    u[a] = (j[a] + 0.5 * F[a]) / RHO0;
  }
}

void ora_velocity(ora_sim *s, double *u) {
  current_forces(s);
  for (long n = 0; n < s->N; n++) {
    double un[3], F[3];
    if (simulated(s, n))
      node_velocity(s, n, un, F);
    else
      un[0] = un[1] = un[2] = 0;
    for (int a = 0; a < s->d; a++) u[a * s->N + n] = un[a];
  }
}

/* Strain rate from the non-equilibrium second moment with the forcing
 * correction (Sec. 3.1, Eq. 19 for D2Q9 MRT; the same Chapman-Enskog
 * relation written for the deviatoric (rate s_nu) and trace (rate s_b)
 * parts on either lattice):
 *   P = Pi_neq + (F u + u F)/2,
 *   S = -(1/(2 rho0 cs2)) [s_nu (P - tr(P)/d I) + s_b tr(P)/d I].
 * Output order: xx, yy, xy (2D); xx, yy, zz, xy, yz, xz (3D). */
void ora_strain_rate(ora_sim *s, double *S) {
  current_forces(s);
  int d = s->d, nc = d == 2 ? 3 : 6;
  double snu = 1.0 / s->tau, sb = 1.0 / s->tau;
  if (s->collision == ORA_MRT)
    for (int k = 0; k < s->Q; k++) {
      if (moment_kind(s->lattice, k) == 'v') snu = s->coll.s[k];
      if (moment_kind(s->lattice, k) == 'b') sb = s->coll.s[k];
    }
  static const int ca[6] = {0, 1, 2, 0, 1, 0}, cb[6] = {0, 1, 2, 1, 2, 2};
  static const int c2a[3] = {0, 1, 0}, c2b[3] = {0, 1, 1};
  for (long n = 0; n < s->N; n++) {
    for (int c = 0; c < nc; c++) S[c * s->N + n] = 0;
    if (!simulated(s, n)) continue;
    double u[3], F[3], rho = 0, feq[MAXQ], P[3][3];
    node_velocity(s, n, u, F);
    for (int i = 0; i < s->Q; i++) rho += s->f[(long)i * s->N + n];
    ora_equilibrium(s->lattice, rho, u, feq);
    for (int a = 0; a < 3; a++)
      for (int b2 = 0; b2 < 3; b2++) {
        P[a][b2] = 0.5 * (F[a] * u[b2] + u[a] * F[b2]);
        for (int i = 0; i < s->Q; i++)
          P[a][b2] += (s->f[(long)i * s->N + n] - feq[i]) * s->e[i][a] *
                      s->e[i][b2];
      }
    double tr = 0;
    for (int a = 0; a < d; a++) tr += P[a][a];
    for (int c = 0; c < nc; c++) {
      int a = d == 2 ? c2a[c] : ca[c], b2 = d == 2 ? c2b[c] : cb[c];
      double dev = P[a][b2] - (a == b2 ? tr / d : 0);
      double iso = a == b2 ? tr / d : 0;
      S[c * s->N + n] = -(snu * dev + sb * iso) / (2 * RHO0 * CS2);
    }
  }
}

/* Viscous dissipation rate (Sec. 3.1): epsilon = 2 nu s_ij s_ij, the strain
 * rate from the non-equilibrium moments as above, nu = (tau - 1/2) c_s^2. */
void ora_dissipation(ora_sim *s, double *eps) {
  const int d = s->d, nc = d == 2 ? 3 : 6;
  double *S = (double *)malloc(sizeof(double) * (size_t)nc * s->N);
  ora_strain_rate(s, S);
  const double nu = (s->tau - 0.5) * CS2;
  for (long n = 0; n < s->N; n++) {
    double ss = 0;
    for (int c = 0; c < nc; c++) {
      const double v = S[c * s->N + n];
      ss += (c < d ? 1.0 : 2.0) * v * v;  /* off-diagonal entries appear twice */
    }
    eps[n] = 2 * nu * ss;
  }
  free(S);
}

/* Stress (Sec. 3.1): sigma = -c_s^2 rho I + 2 rho0 nu S, the pressure of
 * the lattice equation of state p = c_s^2 rho plus the Newtonian viscous
 * stress of the strain rate above, nu = (tau - 1/2) c_s^2.  Same component
 * order as ora_strain_rate; 0 at nodes that are not simulated. */
void ora_stress(ora_sim *s, double *sig) {
  const int d = s->d, nc = d == 2 ? 3 : 6;
  double *S = (double *)malloc(sizeof(double) * (size_t)nc * s->N);
  double *rho = (double *)malloc(sizeof(double) * (size_t)s->N);
  ora_strain_rate(s, S);
  ora_density(s, rho);
  const double nu = (s->tau - 0.5) * CS2;
  for (long n = 0; n < s->N; n++)
    for (int c = 0; c < nc; c++) {
      double v = 0;
      if (simulated(s, n)) v = (c < d ? -CS2 * rho[n] : 0.0) + 2 * RHO0 * nu * S[c * s->N + n];
      sig[c * s->N + n] = v;
    }
  free(S);
  free(rho);
}

void ora_solid_mask(ora_sim *s, unsigned char *m) {
  for (long n = 0; n < s->N; n++) m[n] = simulated(s, n) ? 0 : 1;
}

void ora_force_torque(ora_sim *s, int id, double F[3], double T[3]) {
  if (s->scheme == ORA_IBM) current_forces(s);
  for (int a = 0; a < 3; a++) {
    F[a] = s->sol[id].F[a];
    T[a] = s->sol[id].T[a];
  }
}

int ora_num_markers(const ora_sim *s, int id) { return s->sol[id].nm; }

void ora_snapshot_velocity(ora_sim *s) { ora_velocity(s, s->usnap); }

/* || u^n - u^(n-K) ||_2 / || u^n ||_2 over simulated nodes */
double ora_residual(ora_sim *s) {
  double *u = (double *)calloc((size_t)3 * s->N, sizeof(double));
  ora_velocity(s, u);
  double num = 0, den = 0;
  for (int a = 0; a < s->d; a++)
    for (long n = 0; n < s->N; n++) {
      double du = u[a * s->N + n] - s->usnap[a * s->N + n];
      num += du * du;
      den += u[a * s->N + n] * u[a * s->N + n];
    }
  free(u);
  if (!isfinite(num) || !isfinite(den)) return NAN; /* a diverged field has no residual */
  return den > 0 ? sqrt(num / den) : 0;
}

long ora_steps_done(const ora_sim *s) { return s->steps; }

void ora_solid_centre(const ora_sim *s, int id, double c[3]) {
  for (int a = 0; a < 3; a++) c[a] = s->sol[id].c[a];
}

void ora_solid_velocity(const ora_sim *s, int id, double U[3], double Om[3]) {
  for (int a = 0; a < 3; a++) {
    U[a] = s->sol[id].U[a];
    Om[a] = s->sol[id].Om[a];
  }
}

void ora_set_solid_dynamics(ora_sim *s, int id, double rho_ratio, const double g[3]) {
  solid_t *b = &s->sol[id];
  b->have_Ip = 0;
  b->free_ = rho_ratio > 0;
  b->rho_p = rho_ratio;
  for (int a = 0; a < 3; a++) {
    b->g[a] = g ? g[a] : 0;
    b->Up[a] = b->U[a];
    b->Omp[a] = b->Om[a];
  }
  if (s->d == 2) b->g[2] = 0;
}

void ora_link_stats(const ora_sim *s, long counts[8]) {
  for (int k = 0; k < 8; k++) counts[k] = s->link_counts[k];
}
