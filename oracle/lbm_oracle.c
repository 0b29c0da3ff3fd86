/*
 * lbm_oracle.c -- plain FP64 CPU lattice Boltzmann oracle (TEST INFRASTRUCTURE).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this library. It shares no code with the CUDA path and is written to be
 * checked against the paper by eye: two full arrays, push streaming, one loop
 * per step of the method, no blocking or fusion.
 *
 * Paper: arXiv:2009.04604 (ELIBB single-node boundary condition).
 *   Lattice Boltzmann equation ............ Sec. II.A, Eq. LBE
 *   BGK collision, Omega = 1/tau .......... Sec. II.A, Eq. LB-BGK
 *   TRT collision (even/odd rates) ........ Sec. II.A, TRT paragraph, Eq. magic-parameter
 *   regularized wall non-equilibrium ...... appendix, Eqs. fi_neq, malaspinas, a12Eqlambda
 *   second-order equilibrium .............. Sec. II.A, Eq. Eq2ndOrder (c_s^2 = 1/3)
 *   generic interpolated bounce-back ...... Sec. II.B, Eq. general-ibb-linear
 *   BFL (linear Bouzidi) .................. Sec. II.B, Eq. bfl
 *   ELIBB general scheme .................. Sec. II.C, Eq. ELIBB-general
 *   wall population estimates ............. Sec. II.C.1 (Eqs. feq_approx-1, neqbb-s)
 *                                           and Sec. II.D (Eqs. ELIBB-approximation-*)
 *   s coordinate, Lagrange weights ........ Sec. II.C.2, Eqs. s, x_to_s_helper, poli_coeff
 *   ELIBB-U / -F / -UQ / -FQ .............. Sec. II.D, Eqs. unified_space_coordinates,
 *                                           linear_broken_method, elibbqu,
 *                                           quadratic_fragmented_method (q_cut = 0.01)
 *   moving-wall correction ................ Sec. II.E, Eq. ME-solid-to-fluid
 *   momentum-exchange force ............... Sec. II.F, Eq. force-boundary-node
 * Readings where the paper is silent or garbled (each also listed in the design notes):
 *   - body force: Guo forcing (the paper does not name a forcing scheme);
 *   - ELIBB-F weights are the Lagrange weights of Eq. poli_coeff at the points of
 *     Eq. x_to_s_helper (the printed q >= 1/2 weight (2-2q)/q is not a partition of unity);
 *   - the post-collision wall population uses (1 - 1/tau) f^neq, at s = 1;
 *     under TRT as well (omega+ = 1/tau: the wall non-equilibrium is even in c
 *     at first order);
 *   - TRT with Guo forcing: the even and odd parts of the forcing term take the
 *     factors (1 - omega+/2) and (1 - omega-/2);
 *   - regularized wall non-equilibrium (Eq. fi_neq, third-order truncation): the
 *     second Hermite coefficient is the node's non-equilibrium stress (Lambda at
 *     the wall taken as at x_F), the third follows from Eq. malaspinas with the
 *     wall's velocity at each wall point's time; open links keep Eq. neqbb-s;
 *   - the wall population index is i (incoming), as the paper's macros write it;
 *   - rho in the wall equilibria and the moving-wall term is rho_F(t);
 *   - the force uses the outgoing post-collision population f*_ibar (Wen et al.);
 *   - pressure outlet: f_i = f_i^eq(rho0, u_F) + f^neq_ibar(x_F) (single node,
 *     non-equilibrium bounce-back as in Eq. neqbb-s).
 * Parity unpinned: none of the functions here; each is pinned by the CPU tests
 * against closed forms, invariants or brute force.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define QMAX 27

/* ---- lattice tables (standard Gauss-Hermite sets; the paper does not print them) ---- */
static const int C_D2Q9[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const double W_D2Q9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                                 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int C_D3Q19[19][3] = {
    {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W_D3Q19[19] = {
    1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* D3Q27: rest 8/27, six axis links 2/27, twelve edge diagonals 1/54, eight
 * corner diagonals 1/216 (the lattice of the paper's 3-D cylindrical Couette runs) */
static const int C_D3Q27[27][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},  {1, 1, 1},   {-1, -1, -1},
    {1, 1, -1},  {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1}};
static const double W_D3Q27[27] = {
    8.0 / 27.0,  2.0 / 27.0,  2.0 / 27.0,  2.0 / 27.0,  2.0 / 27.0,  2.0 / 27.0,  2.0 / 27.0,
    1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,
    1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,  1.0 / 54.0,  1.0 / 216.0, 1.0 / 216.0,
    1.0 / 216.0, 1.0 / 216.0, 1.0 / 216.0, 1.0 / 216.0, 1.0 / 216.0, 1.0 / 216.0};

static const double CS2 = 1.0 / 3.0; /* lattice speed of sound squared */

typedef struct {
  int Q, D;
  int c[QMAX][3];
  double w[QMAX];
  int opp[QMAX];
} lat_t;

static int lat_load(int lattice, lat_t *L) {
  const int(*c)[3];
  const double *w;
  if (lattice == OR_D2Q9) { L->Q = 9; L->D = 2; c = C_D2Q9; w = W_D2Q9; }
  else if (lattice == OR_D3Q19) { L->Q = 19; L->D = 3; c = C_D3Q19; w = W_D3Q19; }
  else if (lattice == OR_D3Q27) { L->Q = 27; L->D = 3; c = C_D3Q27; w = W_D3Q27; }
  else return -1;
  for (int i = 0; i < L->Q; ++i) {
    for (int d = 0; d < 3; ++d) L->c[i][d] = c[i][d];
    L->w[i] = w[i];
  }
  for (int i = 0; i < L->Q; ++i)
    for (int j = 0; j < L->Q; ++j)
      if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
        L->opp[i] = j;
  return 0;
}

int or_lattice(int lattice, int *c, double *w, int *opp) {
  lat_t L;
  if (lat_load(lattice, &L)) return -1;
  for (int i = 0; i < L.Q; ++i) {
    for (int d = 0; d < 3; ++d) if (c) c[i * 3 + d] = L.c[i][d];
    if (w) w[i] = L.w[i];
    if (opp) opp[i] = L.opp[i];
  }
  return L.Q;
}

/* ---- index helpers: periodic index space with sheared x-wrap ---- */
static int imod(int a, int m) { int r = a % m; return r < 0 ? r + m : r; }

/* node reached from (x,y,z) by the displacement (dx,dy,dz) */
static long nbr(const or_params *p, int x, int y, int z, int dx, int dy, int dz) {
  int X = x + dx, Y = y + dy, Z = z + dz;
  if (X >= p->nx) { X -= p->nx; Y -= p->xshift; }
  else if (X < 0) { X += p->nx; Y += p->xshift; }
  Y = imod(Y, p->ny);
  Z = imod(Z, p->nz);
  return (long)X + (long)p->nx * ((long)Y + (long)p->ny * Z);
}

/* ---- Eq. Eq2ndOrder: w_i rho [1 + c.u/cs2 + u_a u_b (c_a c_b - cs2 delta_ab)/(2 cs2^2)] ---- */
static double feq(const lat_t *L, int i, double rho, const double u[3]) {
  double cu = 0.0, quad = 0.0;
  for (int a = 0; a < 3; ++a) cu += L->c[i][a] * u[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      quad += u[a] * u[b] * (L->c[i][a] * L->c[i][b] - (a == b ? CS2 : 0.0));
  return L->w[i] * rho * (1.0 + cu / CS2 + quad / (2.0 * CS2 * CS2));
}

/* Guo forcing term without its relaxation factor: w_i [(c_i - u)/cs2 + (c_i.u) c_i/cs2^2] . F */
static double guo_term(const lat_t *L, int i, const double u[3], const double F[3]) {
  double cu = 0.0, s = 0.0;
  for (int a = 0; a < 3; ++a) cu += L->c[i][a] * u[a];
  for (int a = 0; a < 3; ++a)
    s += ((L->c[i][a] - u[a]) / CS2 + cu * L->c[i][a] / (CS2 * CS2)) * F[a];
  return L->w[i] * s;
}

/* Guo forcing source of BGK: (1 - 1/(2 tau)) times the term above */
static double guo_source(const lat_t *L, int i, double tau, const double u[3], const double F[3]) {
  return (1.0 - 1.0 / (2.0 * tau)) * guo_term(L, i, u, F);
}

/* TRT collision of population i (Sec. II.A): the even parts a+ = (a_i + a_ibar)/2 of
 * f, f^eq and the forcing term relax with omega+, the odd parts a- = (a_i - a_ibar)/2
 * with omega-, each forcing part scaled by (1 - omega/2) of its own rate. */
static double trt_post(const lat_t *L, int i, const double *fn, double rho, const double u[3],
                       const double F[3], double omp, double omm) {
  const int ib = L->opp[i];
  const double fp = 0.5 * (fn[i] + fn[ib]), fm = 0.5 * (fn[i] - fn[ib]);
  const double ei = feq(L, i, rho, u), eb = feq(L, ib, rho, u);
  const double ep = 0.5 * (ei + eb), em = 0.5 * (ei - eb);
  const double si = guo_term(L, i, u, F), sb = guo_term(L, ib, u, F);
  const double sp = 0.5 * (si + sb), sm = 0.5 * (si - sb);
  return fn[i] - omp * (fp - ep) - omm * (fm - em) + (1.0 - 0.5 * omp) * sp + (1.0 - 0.5 * omm) * sm;
}

/* ---- regularized non-equilibrium (appendix, Eq. fi_neq) ----
 * Hermite tensors H2_ab = c_a c_b - cs2 d_ab and
 * H3_abc = c_a c_b c_c - cs2 (c_a d_bc + c_b d_ac + c_c d_ab). The first-order
 * population is rebuilt from its second Hermite coefficient a2 (the
 * non-equilibrium stress) and the third, a3_abc = u_c a2_ab + u_b a2_ac + u_a a2_bc
 * (Eq. malaspinas, isothermal):
 *   f1_i = w_i [ H2_i : a2 / (2 cs2^2) + H3_i : a3 / (6 cs2^3) ]                 */
static double kd(int a, int b) { return a == b ? 1.0 : 0.0; }

static double reg_neq(const lat_t *L, int i, const double a2[3][3], const double u[3]) {
  const int *c = L->c[i];
  double s2 = 0.0, s3 = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      s2 += (c[a] * c[b] - CS2 * kd(a, b)) * a2[a][b];
      for (int g = 0; g < 3; ++g) {
        const double h3 = c[a] * c[b] * c[g] - CS2 * (c[a] * kd(b, g) + c[b] * kd(a, g) + c[g] * kd(a, b));
        const double a3 = u[g] * a2[a][b] + u[b] * a2[a][g] + u[a] * a2[b][g];
        s3 += h3 * a3;
      }
    }
  return L->w[i] * (s2 / (2.0 * CS2 * CS2) + s3 / (6.0 * CS2 * CS2 * CS2));
}

/* density and Guo-corrected velocity u = (sum c f + F/2) / rho */
static void moments(const lat_t *L, const double *fn, const double F[3], double *rho, double u[3]) {
  double r = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < L->Q; ++i) {
    r += fn[i];
    for (int a = 0; a < 3; ++a) j[a] += L->c[i][a] * fn[i];
  }
  *rho = r;
  for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / r;
}

/* ---- Eq. poli_coeff: Lagrange interpolation through (s_j, v_j) evaluated at s_ref ---- */
static double lagrange(int np, const double *s, const double *v, double sref) {
  double r = 0.0;
  for (int j = 0; j < np; ++j) {
    double a = 1.0;
    for (int k = 0; k < np; ++k)
      if (k != j) a *= (sref - s[k]) / (s[j] - s[k]);
    r += a * v[j];
  }
  return r;
}

/* Interpolation points of each scheme, by the s coordinate of Eq. x_to_s_helper:
 *   P_F0: wall population  f~_i^{t+1}(x_W)   s = 0
 *   P_G : f*_ibar(x_F)                        s = 1 - q
 *   P_F1: wall population  f~*_i(x_W)         s = 1 (reading; exact: 1 + u_w.c_i/|c_i|^2)
 *   P_H : f*_i(x_F)                           s = 1 + q
 *   P_FF: f*_ibar(x_FF), x_FF = x_F + c_i     s = -q                                  */
enum { P_F0 = 0, P_G = 1, P_F1 = 2, P_H = 3, P_FF = 4 };

static int bc_points(int bc, double q, double qcut, int ff_fluid, int *pt) {
  switch (bc) {
    case OR_BC_HWBB: pt[0] = P_G; return 1;
    case OR_BC_ELIBB_F:
      if (q < 0.5) { pt[0] = P_F0; pt[1] = P_G; } else { pt[0] = P_G; pt[1] = P_F1; }
      return 2;
    case OR_BC_ELIBB_FQ:
      if (q < qcut) return bc_points(OR_BC_ELIBB_F, q, qcut, ff_fluid, pt);
      if (q < 0.5) { pt[0] = P_F0; pt[1] = P_G; pt[2] = P_F1; }
      else { pt[0] = P_G; pt[1] = P_F1; pt[2] = P_H; }
      return 3;
    case OR_BC_BFL:
      if (q < 0.5) {
        if (!ff_fluid) { pt[0] = P_G; return 1; } /* no second node: half-way bounce-back */
        pt[0] = P_FF; pt[1] = P_G; return 2;
      }
      pt[0] = P_G; pt[1] = P_H; return 2;
    case OR_BC_ELIBB_U: pt[0] = P_F0; pt[1] = P_F1; return 2;
    case OR_BC_ELIBB_UQ:
      /* reading: as q -> 1 the point s = 1 - q meets s = 0; below the same cutoff the
       * unified linear rule is used (mirror of the ELIBB-FQ cutoff at q -> 0) */
      if (1.0 - q < qcut) return bc_points(OR_BC_ELIBB_U, q, qcut, ff_fluid, pt);
      pt[0] = P_F0; pt[1] = P_G; pt[2] = P_F1; return 3;
    default: return 0;
  }
}

static double point_s(int pt, double q, double s1) {
  switch (pt) {
    case P_F0: return 0.0;
    case P_G: return 1.0 - q;
    case P_F1: return s1;
    case P_H: return 1.0 + q;
    default: return -q; /* P_FF */
  }
}

int or_bc_weights(int bc, double q, double qcut, double *s, double *a) {
  int pt[3];
  int np = bc_points(bc, q, qcut, 1, pt);
  double ss[3];
  for (int j = 0; j < np; ++j) ss[j] = point_s(pt[j], q, 1.0);
  for (int j = 0; j < np; ++j) {
    double v[3] = {0.0, 0.0, 0.0};
    v[j] = 1.0;
    s[j] = ss[j];
    a[j] = lagrange(np, ss, v, q);
  }
  return np;
}

/* ---- initial state ---- */
void or_init_eq(const or_params *p, const uint8_t *flags, const double *rho, const double *u,
                double *f) {
  lat_t L;
  if (lat_load(p->lattice, &L)) return;
  long N = (long)p->nx * p->ny * p->nz;
  for (long n = 0; n < N; ++n) {
    double r = rho ? rho[n] : p->rho0;
    double uu[3] = {0.0, 0.0, 0.0};
    if (u) for (int a = 0; a < 3; ++a) uu[a] = u[n * 3 + a];
    for (int i = 0; i < L.Q; ++i)
      f[n * L.Q + i] = (flags[n] == OR_FLUID) ? feq(&L, i, r, uu) : 0.0;
  }
}

/* ---- one time step ---- */
int or_step(const or_params *p, const uint8_t *flags, const double *q, const uint8_t *shell,
            const double *uw, const double *uw1, const double *f, double *fout, double *flink) {
  lat_t L;
  if (lat_load(p->lattice, &L) || p->tau <= 0.5 || !flags || !f || !fout) return -1;
  const int Q = L.Q;
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const long N = (long)nx * ny * nz;
  const double omega = 1.0 / p->tau;
  const int trt = p->collision == OR_COLL_TRT;
  if (trt && !(p->magic > 0.0)) return -1;
  /* Eq. magic-parameter solved for omega- */
  const double omega_m = trt ? 1.0 / (0.5 + p->magic / (p->tau - 0.5)) : omega;
  if (!uw1) uw1 = uw;

  double *fpost = (double *)calloc((size_t)N * Q, sizeof(double));
  double *rho = (double *)calloc((size_t)N, sizeof(double));
  double *vel = (double *)calloc((size_t)N * 3, sizeof(double));
  if (!fpost || !rho || !vel) { free(fpost); free(rho); free(vel); return -1; }

  /* 1. collision at every fluid node: f* = f - Omega (f - f^eq) + S (Eq. LB-BGK) */
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; ++n) {
    if (flags[n] != OR_FLUID) continue;
    double r, u[3];
    moments(&L, f + n * Q, p->force, &r, u);
    rho[n] = r;
    for (int a = 0; a < 3; ++a) vel[n * 3 + a] = u[a];
    for (int i = 0; i < Q; ++i) {
      double fi = f[n * Q + i];
      fpost[n * Q + i] = trt ? trt_post(&L, i, f + n * Q, r, u, p->force, omega, omega_m)
                             : fi - omega * (fi - feq(&L, i, r, u)) + guo_source(&L, i, p->tau, u, p->force);
    }
  }

  for (long n = 0; n < N * Q; ++n) fout[n] = 0.0;

  /* 2. streaming: f_i(x + c_i, t+1) = f*_i(x, t) between fluid nodes (Eq. LBE),
   * except across a thin shell (link i of x + c_i marked in shell) */
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; ++n) {
    if (flags[n] != OR_FLUID) continue;
    int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long)nx * ny));
    for (int i = 0; i < Q; ++i) {
      long m = nbr(p, x, y, z, L.c[i][0], L.c[i][1], L.c[i][2]);
      if (flags[m] == OR_FLUID && !(shell && shell[m * Q + i])) fout[m * Q + i] = fpost[n * Q + i];
    }
  }

  /* 3. boundary rule for every cut link (x_F, i): x_F - c_i is not fluid, or lies
   * across a thin shell. A shell is a wall seen from both of its sides, so each
   * side applies the rule to the population coming back to it. */
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; ++n) {
    if (flags[n] != OR_FLUID) continue;
    int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long)nx * ny));
    const double rF = rho[n];
    const double *uF = vel + n * 3;
    /* non-equilibrium stress of the node, sum_j c_j c_j (f_j - f^eq_j), for the
     * regularized wall estimate (the stress at the wall is taken as the node's) */
    double a2[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    if (p->wall_neq == OR_NEQ_REGULARIZED)
      for (int j = 0; j < Q; ++j) {
        const double fn = f[n * Q + j] - feq(&L, j, rF, uF);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) a2[a][b] += L.c[j][a] * L.c[j][b] * fn;
      }
    for (int i = 1; i < Q; ++i) {
      long m = nbr(p, x, y, z, -L.c[i][0], -L.c[i][1], -L.c[i][2]);
      if (flags[m] == OR_FLUID && !(shell && shell[n * Q + i])) continue;
      const int ib = L.opp[i];
      /* pre-collision non-equilibrium of the outgoing population (Eq. neqbb-s) */
      const double fneq_ib = f[n * Q + ib] - feq(&L, ib, rF, uF);
      double result;
      if (flags[m] == OR_OPEN) {
        double r0 = p->rho0;
        result = feq(&L, i, r0, uF) + fneq_ib;
        fout[n * Q + i] = result;
        continue;
      }
      const double qq = q ? q[n * Q + i] : 0.5;
      double u0[3] = {0.0, 0.0, 0.0}, u1[3] = {0.0, 0.0, 0.0};
      if (uw) for (int a = 0; a < 3; ++a) u0[a] = uw[(n * Q + i) * 3 + a];
      if (uw1) for (int a = 0; a < 3; ++a) u1[a] = uw1[(n * Q + i) * 3 + a];
      /* Eq. ME-solid-to-fluid: + 2 w_i rho c_i.u_w / cs2 on nodal points with s < 1 */
      double cu = 0.0, c2 = 0.0;
      for (int a = 0; a < 3; ++a) { cu += L.c[i][a] * u0[a]; c2 += L.c[i][a] * L.c[i][a]; }
      const double rme = p->me_rho0 ? p->rho0 : rF;
      const double me = 2.0 * L.w[i] * rme * cu / CS2;
      /* wall populations (Eqs. f=eq+neq, ELIBB-approximation-eq1/eq2, neqbb-s) */
      /* reading: under TRT the wall non-equilibrium, even in c at first order, decays
       * with omega+ = 1/tau as under BGK */
      const double post = p->wall_neq_same ? 1.0 : (1.0 - omega);
      /* wall non-equilibrium: f^neq_ibar(x_F) (Eq. neqbb-s), or the regularized
       * estimate with the wall's velocity at each time (Eq. fi_neq) */
      const int reg = p->wall_neq == OR_NEQ_REGULARIZED;
      const double fn0 = reg ? reg_neq(&L, i, (const double(*)[3])a2, u1) : fneq_ib;
      const double fn1 = reg ? reg_neq(&L, i, (const double(*)[3])a2, u0) : fneq_ib;
      const double f0 = feq(&L, i, rF, u1) + fn0;
      const double f1 = feq(&L, i, rF, u0) + post * fn1;
      const double s1 = p->s1_exact ? 1.0 + cu / c2 : 1.0;
      /* second fluid node along the link (BFL only), on the node's side of any shell */
      long ff = nbr(p, x, y, z, L.c[i][0], L.c[i][1], L.c[i][2]);
      int ff_fluid = flags[ff] == OR_FLUID && !(shell && shell[n * Q + ib]);
      int pt[3];
      int np = bc_points(p->bc, qq, p->qcut, ff_fluid, pt);
      double s[3], v[3];
      for (int j = 0; j < np; ++j) {
        s[j] = point_s(pt[j], qq, s1);
        switch (pt[j]) {
          case P_F0: v[j] = f0; break;
          case P_F1: v[j] = f1; break;
          case P_G: v[j] = fpost[n * Q + ib]; break;
          case P_H: v[j] = fpost[n * Q + i]; break;
          default: v[j] = fpost[ff * Q + ib]; break;
        }
        if (pt[j] != P_F0 && pt[j] != P_F1 && s[j] < 1.0) v[j] += me;
      }
      result = lagrange(np, s, v, qq);
      fout[n * Q + i] = result;
      if (flink) {
        /* Eq. force-boundary-node: (c_ibar - u_w) f*_ibar(x_F,t) - (c_i - u_w) f_i(x_F,t+1) */
        for (int a = 0; a < 3; ++a)
          flink[(n * Q + i) * 3 + a] =
              (L.c[ib][a] - u0[a]) * fpost[n * Q + ib] - (L.c[i][a] - u0[a]) * result;
      }
    }
  }
  if (flink) {
    /* links that are not wall links carry no force; of a thin shell's links only
     * those on its outer side count (the fluid inside moves with the body) */
    for (long n = 0; n < N; ++n) {
      int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long)nx * ny));
      for (int i = 0; i < Q; ++i) {
        long m = nbr(p, x, y, z, -L.c[i][0], -L.c[i][1], -L.c[i][2]);
        const int sh = shell ? shell[n * Q + i] : 0;
        int wall = flags[n] == OR_FLUID && i > 0 && ((flags[m] == OR_SOLID && !sh) || sh == 1);
        if (!wall) for (int a = 0; a < 3; ++a) flink[(n * Q + i) * 3 + a] = 0.0;
      }
    }
  }
  free(fpost);
  free(rho);
  free(vel);
  return 0;
}

void or_macros(const or_params *p, const uint8_t *flags, const double *f, double *rho, double *u) {
  lat_t L;
  if (lat_load(p->lattice, &L)) return;
  long N = (long)p->nx * p->ny * p->nz;
  for (long n = 0; n < N; ++n) {
    double r = 0.0, uu[3] = {0.0, 0.0, 0.0};
    if (flags[n] == OR_FLUID) moments(&L, f + n * L.Q, p->force, &r, uu);
    if (rho) rho[n] = r;
    if (u) for (int a = 0; a < 3; ++a) u[n * 3 + a] = uu[a];
  }
}

double or_mass(const or_params *p, const uint8_t *flags, const double *f) {
  lat_t L;
  if (lat_load(p->lattice, &L)) return 0.0;
  long N = (long)p->nx * p->ny * p->nz;
  double m = 0.0;
  for (long n = 0; n < N; ++n)
    if (flags[n] == OR_FLUID)
      for (int i = 0; i < L.Q; ++i) m += f[n * L.Q + i];
  return m;
}

void or_refill(const or_params *p, const uint8_t *flags_old, const uint8_t *flags_new,
               const double *un, double *f) {
  lat_t L;
  if (lat_load(p->lattice, &L)) return;
  long N = (long)p->nx * p->ny * p->nz;
  for (long n = 0; n < N; ++n) {
    if (flags_old[n] == OR_FLUID || flags_new[n] != OR_FLUID) continue;
    double uu[3] = {0.0, 0.0, 0.0};
    if (un) for (int a = 0; a < 3; ++a) uu[a] = un[n * 3 + a];
    for (int i = 0; i < L.Q; ++i) f[n * L.Q + i] = feq(&L, i, p->rho0, uu);
  }
}

/* post-collision population i of a node with pre-collision populations fn (the
 * collision of or_step: BGK with Guo forcing, or TRT) */
static double post_one(const or_params *p, const lat_t *L, const double *fn, int i) {
  double r, u[3];
  moments(L, fn, p->force, &r, u);
  const double omega = 1.0 / p->tau;
  if (p->collision == OR_COLL_TRT) {
    const double omega_m = 1.0 / (0.5 + p->magic / (p->tau - 0.5));
    return trt_post(L, i, fn, r, u, p->force, omega, omega_m);
  }
  return fn[i] - omega * (fn[i] - feq(L, i, r, u)) + guo_source(L, i, p->tau, u, p->force);
}

/* the same collision with the node's velocity set to uw (its density from fn) */
static double post_at(const or_params *p, const lat_t *L, const double *fn, int i, const double uw[3]) {
  double r = 0.0;
  for (int j = 0; j < L->Q; ++j) r += fn[j];
  const double omega = 1.0 / p->tau;
  if (p->collision == OR_COLL_TRT) {
    const double omega_m = 1.0 / (0.5 + p->magic / (p->tau - 0.5));
    return trt_post(L, i, fn, r, uw, p->force, omega, omega_m);
  }
  return fn[i] - omega * (fn[i] - feq(L, i, r, uw)) + guo_source(L, i, p->tau, uw, p->force);
}

void or_refill_lir(const or_params *p, const uint8_t *flags_old, const uint8_t *flags_new,
                   const double *un, const double *fprev, int K, double *f) {
  lat_t L;
  if (lat_load(p->lattice, &L)) return;
  const int Q = L.Q;
  const int nx = p->nx, ny = p->ny;
  const long N = (long)nx * ny * p->nz;
  for (long n = 0; n < N; ++n) {
    if (flags_old[n] == OR_FLUID || flags_new[n] != OR_FLUID) continue;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long)nx * ny));
    double uw[3] = {0.0, 0.0, 0.0};
    if (un) for (int a = 0; a < 3; ++a) uw[a] = un[n * 3 + a];
    double fn[27];
    int unknown[27];
    for (int i = 0; i < Q; ++i) {
      const long m = nbr(p, x, y, z, -L.c[i][0], -L.c[i][1], -L.c[i][2]);
      unknown[i] = flags_old[m] != OR_FLUID;
      fn[i] = unknown[i] ? feq(&L, i, p->rho0, uw) : post_one(p, &L, fprev + m * Q, i);
    }
    for (int k = 0; k < K; ++k) {
      double r = 0.0, post[27];
      for (int i = 0; i < Q; ++i) r += fn[i];
      for (int i = 0; i < Q; ++i) post[i] = post_at(p, &L, fn, i, uw);
      for (int i = 0; i < Q; ++i) {
        if (!unknown[i]) continue;
        double cu = 0.0;
        for (int a = 0; a < 3; ++a) cu += L.c[i][a] * uw[a];
        fn[i] = post[L.opp[i]] + 2.0 * L.w[i] * r * cu / CS2;
      }
    }
    for (int i = 0; i < Q; ++i) f[n * Q + i] = fn[i];
  }
}

/* ---- link geometry ---- */

/* point inside the solid of shape s (ties count as solid) */
static int shape_solid(const or_shape *s, int D, const double x[3]) {
  double d0 = x[0] - s->c[0], d1 = x[1] - s->c[1], d2 = D == 3 ? x[2] - s->c[2] : 0.0;
  switch (s->type) {
    case OR_SHAPE_SPHERE: return d0 * d0 + d1 * d1 + d2 * d2 <= s->r[0] * s->r[0];
    case OR_SHAPE_SPHERE_OUT: return d0 * d0 + d1 * d1 + d2 * d2 >= s->r[0] * s->r[0];
    case OR_SHAPE_ELLIPSOID: {
      /* offset in the body frame: rotated by -ang about z */
      const double ca = cos(s->ang), sa = sin(s->ang);
      const double b0 = ca * d0 + sa * d1, b1 = ca * d1 - sa * d0;
      double t0 = b0 / s->r[0], t1 = b1 / s->r[1], t2 = D == 3 ? d2 / s->r[2] : 0.0;
      return t0 * t0 + t1 * t1 + t2 * t2 <= 1.0;
    }
    case OR_SHAPE_STRIP: {
      double v = s->nrm[0] * x[0] + s->nrm[1] * x[1] + (D == 3 ? s->nrm[2] * x[2] : 0.0) - s->off;
      if (s->period > 0.0) v = v - s->period * floor(v / s->period + 0.5);
      return fabs(v) >= 0.5 * s->width;
    }
    default: return 0;
  }
}

/* Inside a thin shell: strictly closer to the centre than r0. */
static int shell_inside(const or_shape *s, int D, const double x[3]) {
  double d0 = x[0] - s->c[0], d1 = x[1] - s->c[1], d2 = D == 3 ? x[2] - s->c[2] : 0.0;
  return d0 * d0 + d1 * d1 + d2 * d2 < s->r[0] * s->r[0];
}

/* Smallest t in (0,1] where x - t c enters the solid of shape s (or, for a thin
 * shell, meets its surface), or -1.
 * Quadratic roots use the cancellation-free form (Numerical Recipes, Sec. 5.6). */
static double shape_cross(const or_shape *s, int D, const double x[3], const int c[3]) {
  double d[3], e[3];
  for (int a = 0; a < 3; ++a) { d[a] = (a < D) ? x[a] - s->c[a] : 0.0; e[a] = (a < D) ? c[a] : 0.0; }
  switch (s->type) {
    case OR_SHAPE_SPHERE:
    case OR_SHAPE_SPHERE_OUT:
    case OR_SHAPE_SHELL:
    case OR_SHAPE_ELLIPSOID: {
      double R2 = 1.0;
      if (s->type == OR_SHAPE_ELLIPSOID) {
        /* offset and link direction in the body frame, scaled to the unit sphere */
        const double ca = cos(s->ang), sa = sin(s->ang);
        const double d0 = ca * d[0] + sa * d[1], d1 = ca * d[1] - sa * d[0];
        const double e0 = ca * e[0] + sa * e[1], e1 = ca * e[1] - sa * e[0];
        d[0] = d0; d[1] = d1; e[0] = e0; e[1] = e1;
        for (int a = 0; a < D; ++a) { d[a] /= s->r[a]; e[a] /= s->r[a]; }
      } else {
        R2 = s->r[0] * s->r[0];
      }
      /* |d - t e|^2 = R2  <=>  A t^2 - 2 B t + C = 0 */
      double A = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
      double B = d[0] * e[0] + d[1] * e[1] + d[2] * e[2];
      double Cc = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - R2;
      double disc = B * B - A * Cc;
      if (disc < 0.0) return -1.0;
      double sq = sqrt(disc), t;
      if (s->type == OR_SHAPE_SHELL) {
        /* both roots, B -/+ sq over A, in the cancellation-free form; the smaller
         * one in (0,1] */
        double qq = B >= 0.0 ? B + sq : B - sq;
        double ta = qq != 0.0 ? Cc / qq : -1.0, tb = qq / A;
        double lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
        t = (lo > 0.0 && lo <= 1.0) ? lo : hi;
      } else if (s->type != OR_SHAPE_SPHERE_OUT) {
        if (Cc <= 0.0 || B <= 0.0) return -1.0; /* start inside, or moving away */
        t = Cc / (B + sq);                       /* entry root (B - sq)/A */
      } else {
        if (Cc >= 0.0) return -1.0;
        t = (B >= 0.0) ? (B + sq) / A : Cc / (B - sq); /* exit root (B + sq)/A */
      }
      return (t > 0.0 && t <= 1.0) ? t : -1.0;
    }
    case OR_SHAPE_STRIP: {
      double v = s->nrm[0] * x[0] + s->nrm[1] * x[1] + (D == 3 ? s->nrm[2] * x[2] : 0.0) - s->off;
      if (s->period > 0.0) v = v - s->period * floor(v / s->period + 0.5);
      double a = s->nrm[0] * e[0] + s->nrm[1] * e[1] + s->nrm[2] * e[2];
      double h = 0.5 * s->width, t;
      if (a > 0.0) t = (v + h) / a;       /* moving towards -h */
      else if (a < 0.0) t = (v - h) / a;  /* moving towards +h */
      else return -1.0;
      return (t > 0.0 && t <= 1.0) ? t : -1.0;
    }
    default: return -1.0;
  }
}

long or_geometry(const or_params *p, const uint8_t *base, const double *base_u,
                 const or_shape *shapes, int nshapes, uint8_t *flags, double *q, double *uw,
                 double *uw1, int32_t *tag, uint8_t *shell) {
  lat_t L;
  if (lat_load(p->lattice, &L)) return -1;
  const int Q = L.Q, D = L.D;
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const long N = (long)nx * ny * nz;
  int on_shell = 0;
#pragma omp parallel for schedule(static) reduction(| : on_shell)
  for (long n = 0; n < N; ++n) {
    int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long)nx * ny));
    double X[3] = {(double)x, (double)y, (double)z};
    uint8_t fl = base ? base[n] : OR_FLUID;
    if (fl == OR_FLUID)
      for (int k = 0; k < nshapes; ++k)
        if (shape_solid(&shapes[k], D, X)) { fl = OR_SOLID; break; }
    if (fl == OR_FLUID)
      for (int k = 0; k < nshapes; ++k) {
        if (shapes[k].type != OR_SHAPE_SHELL) continue;
        double d0 = X[0] - shapes[k].c[0], d1 = X[1] - shapes[k].c[1],
               d2 = D == 3 ? X[2] - shapes[k].c[2] : 0.0;
        if (d0 * d0 + d1 * d1 + d2 * d2 == shapes[k].r[0] * shapes[k].r[0]) on_shell = 1;
      }
    flags[n] = fl;
  }
  if (on_shell) return -2;
  long ncut = 0;
#pragma omp parallel for schedule(static) reduction(+ : ncut)
  for (long n = 0; n < N; ++n) {
    int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long)nx * ny));
    double X[3] = {(double)x, (double)y, (double)z};
    for (int i = 0; i < Q; ++i) {
      long li = n * Q + i;
      double qq = 0.0, u0[3] = {0.0, 0.0, 0.0}, u1[3] = {0.0, 0.0, 0.0};
      int tg = 0, sh = 0;
      if (flags[n] == OR_FLUID && i > 0) {
        long m = nbr(p, x, y, z, -L.c[i][0], -L.c[i][1], -L.c[i][2]);
        double Y[3];
        for (int a = 0; a < 3; ++a) Y[a] = X[a] - L.c[i][a];
        /* a thin shell between two fluid nodes: 1 seen from outside, 2 from inside */
        if (flags[m] == OR_FLUID)
          for (int k = 0; k < nshapes && !sh; ++k)
            if (shapes[k].type == OR_SHAPE_SHELL) {
              const int in_x = shell_inside(&shapes[k], D, X), in_y = shell_inside(&shapes[k], D, Y);
              if (in_x != in_y) sh = in_x ? 2 : 1;
            }
        if (flags[m] != OR_FLUID || sh) {
          ++ncut;
          if (sh || !base || base[m] == OR_FLUID) {
            /* cut by a shape: nearest crossing along x_F - t c_i */
            double best = 2.0;
            int kb = -1;
            for (int k = 0; k < nshapes; ++k) {
              double t = shape_cross(&shapes[k], D, X, L.c[i]);
              if (t > 0.0 && t < best) { best = t; kb = k; }
            }
            if (kb < 0) {
              best = 1.0; /* rounding left no root: the wall sits on the far node */
              for (int k = 0; k < nshapes; ++k) {
                const int shell_k = shapes[k].type == OR_SHAPE_SHELL &&
                                    shell_inside(&shapes[k], D, X) != shell_inside(&shapes[k], D, Y);
                if (shape_solid(&shapes[k], D, Y) || shell_k) { kb = k; break; }
              }
            }
            qq = best;
            if (kb >= 0) {
              const or_shape *s = &shapes[kb];
              double r[3];
              for (int a = 0; a < 3; ++a) r[a] = (a < D) ? X[a] - qq * L.c[i][a] - s->c[a] : 0.0;
              /* rigid motion at the wall point: v + om x r */
              u0[0] = s->v[0] + s->om[1] * r[2] - s->om[2] * r[1];
              u0[1] = s->v[1] + s->om[2] * r[0] - s->om[0] * r[2];
              u0[2] = s->v[2] + s->om[0] * r[1] - s->om[1] * r[0];
              u1[0] = s->v1[0] + s->om1[1] * r[2] - s->om1[2] * r[1];
              u1[1] = s->v1[1] + s->om1[2] * r[0] - s->om1[0] * r[2];
              u1[2] = s->v1[2] + s->om1[0] * r[1] - s->om1[1] * r[0];
              if (D == 2) { u0[2] = 0.0; u1[2] = 0.0; }
              tg = sh == 2 ? -1 : s->tag;
            }
          } else {
            qq = 0.5; /* base-flag wall: half-way */
            if (base_u && base[m] == OR_SOLID)
              for (int a = 0; a < 3; ++a) { u0[a] = base_u[m * 3 + a]; u1[a] = u0[a]; }
          }
        }
      }
      if (q) q[li] = qq;
      if (uw) for (int a = 0; a < 3; ++a) uw[li * 3 + a] = u0[a];
      if (uw1) for (int a = 0; a < 3; ++a) uw1[li * 3 + a] = u1[a];
      if (tag) tag[li] = tg;
      if (shell) shell[li] = (uint8_t)sh;
    }
  }
  return ncut;
}

void or_torque(const or_params *p, const double *q, const int32_t *tag, const double *flink, int want_tag,
               const double c[3], double T[3]) {
  lat_t L;
  T[0] = T[1] = T[2] = 0.0;
  if (lat_load(p->lattice, &L)) return;
  const int Q = L.Q;
  const int nx = p->nx, ny = p->ny;
  const long N = (long)nx * ny * p->nz;
  for (long n = 0; n < N; ++n) {
    const double X[3] = {(double)(n % nx), (double)((n / nx) % ny), (double)(n / ((long)nx * ny))};
    for (int i = 0; i < Q; ++i) {
      const long li = n * Q + i;
      if (q[li] <= 0.0) continue;                       /* not a cut link */
      if (want_tag >= 0 && tag[li] != want_tag) continue;
      double r[3];
      for (int a = 0; a < 3; ++a) r[a] = X[a] - q[li] * L.c[i][a] - c[a];  /* x_W - c */
      if (L.D == 2) r[2] = 0.0;
      const double *F = flink + li * 3;
      T[0] += r[1] * F[2] - r[2] * F[1];
      T[1] += r[2] * F[0] - r[0] * F[2];
      T[2] += r[0] * F[1] - r[1] * F[0];
    }
  }
}

/* ---- threads ---- */

int or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
