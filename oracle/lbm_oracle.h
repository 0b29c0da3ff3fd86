/*
 * lbm_oracle.h -- plain FP64 CPU lattice Boltzmann oracle (TEST INFRASTRUCTURE).
 *
 * This header belongs to the oracle only. Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load the oracle; the CUDA
 * library shares no code, header or table with it.
 *
 * Paper: Marson, Thorimbert, Latt, Chopard, "Enhanced single-node boundary
 * condition for the Lattice Boltzmann Method" (arXiv:2009.04604).
 *
 * Conventions (all arrays are caller-owned, row-major, FP64 unless stated):
 *   node index   n = x + nx*(y + ny*z)           (nz = 1 for D2Q9)
 *   populations  f[n*Q + i]                      (array of structures)
 *   per link     q[n*Q + i], uw[(n*Q + i)*3 + d] (link i of node n points from
 *                n towards n - c_i, i.e. the node the population i comes from)
 *   node flags   0 = fluid, 1 = solid wall, 2 = open (pressure) ghost node
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_D2Q9 = 0, OR_D3Q19 = 1, OR_D3Q27 = 2 };
enum { OR_FLUID = 0, OR_SOLID = 1, OR_OPEN = 2 };
/* Boundary schemes: ELIBB fragmented linear / quadratic (Sec. II.E),
 * linear Bouzidi-Firdaouss-Lallemand (Eq. bfl), half-way bounce-back,
 * ELIBB unified linear / quadratic (Sec. II.E). */
enum { OR_BC_ELIBB_F = 0, OR_BC_ELIBB_FQ = 1, OR_BC_BFL = 2, OR_BC_HWBB = 3,
       OR_BC_ELIBB_U = 4, OR_BC_ELIBB_UQ = 5 };
/* Collision operators: single relaxation time (Eq. LB-BGK) and two relaxation
 * times (Sec. II.A, TRT paragraph). */
enum { OR_COLL_BGK = 0, OR_COLL_TRT = 1 };
/* Estimates of the non-equilibrium part of a wall population (Sec. II.C.1 and
 * the appendix on the regularized reconstruction). */
enum { OR_NEQ_BOUNCE_BACK = 0, OR_NEQ_REGULARIZED = 1 };
/* Analytic shapes for the link geometry. */
enum { OR_SHAPE_SPHERE = 0,      /* solid inside |x-c| <= r0 (circle in 2D)        */
       OR_SHAPE_SPHERE_OUT = 1,  /* solid outside |x-c| >= r0                      */
       OR_SHAPE_ELLIPSOID = 2,   /* solid inside sum((x-c)'_d/r_d)^2 <= 1, with (x-c)' the offset
                                    in the body frame: rotated by -ang about the z axis */
       OR_SHAPE_STRIP = 3,       /* fluid strip |nrm.x - off| < width/2, periodic along nrm
                                    with period 'period' (0 = not periodic); solid elsewhere */
       OR_SHAPE_SHELL = 4 };     /* thin spherical shell |x-c| = r0 (a circle in 2D) with fluid
                                    on both sides (the thin-shell cylinders of Sec. III.B) */

typedef struct {
  int lattice;        /* OR_D2Q9 or OR_D3Q19 */
  int nx, ny, nz;     /* lattice extents; index space is periodic in every axis */
  int xshift;         /* sheared periodicity: (x + nx, y + xshift) is the same node as (x, y) */
  int bc;             /* OR_BC_* */
  double tau;         /* BGK relaxation time; Omega = 1/tau (Eq. LB-BGK) */
  double rho0;        /* reference density (open boundaries, refill) */
  double force[3];    /* constant body-force density F (Guo forcing) */
  double qcut;        /* ELIBB-FQ cutoff below which ELIBB-F is used (paper: 0.01) */
  int wall_neq_same;  /* 0: post-collision wall neq = (1 - 1/tau) f^neq (default reading);
                         1: the same f^neq for both wall populations */
  int me_rho0;        /* 0: rho in the moving-wall term is rho_F(t) (default); 1: rho0 */
  int s1_exact;       /* 0: s of the post-collision wall population is 1 (default);
                         1: s = 1 + u_w.c_i/|c_i|^2 (Eq. x_to_s_helper as printed) */
  int collision;      /* OR_COLL_BGK, or OR_COLL_TRT (two relaxation times, Sec. II.A) */
  int wall_neq;       /* OR_NEQ_BOUNCE_BACK (Eq. neqbb-s) or OR_NEQ_REGULARIZED (Eq. fi_neq):
                         the estimate of the wall non-equilibrium in the ELIBB wall populations */
  double magic;       /* TRT: Lambda = (1/omega+ - 1/2)(1/omega- - 1/2) (Eq. magic-parameter),
                         omega+ = 1/tau */
} or_params;

typedef struct {
  int type;           /* OR_SHAPE_* */
  int tag;            /* force accumulation tag, copied to every link the shape cuts */
  double c[3];        /* centre (sphere, ellipsoid) */
  double r[3];        /* radius in r[0] (sphere) or semi-axes (ellipsoid) */
  double nrm[3];      /* unit normal of the strip */
  double off, width, period;   /* strip: centre-line offset, width, normal period */
  double v[3], om[3];          /* rigid velocity and angular velocity at time t */
  double v1[3], om1[3];        /* the same at time t + 1 */
  double ang;                  /* ellipsoid: rotation about the z axis (radians); its
                                  semi-axes r[0], r[1] lie along (cos, sin) and (-sin, cos) */
} or_shape;

/* Lattice tables in the oracle's own order: c[i*3 + d], w[i], opp[i]. Returns Q. */
int or_lattice(int lattice, int *c, double *w, int *opp);

/* f = f^eq(rho[n], u[n*3..]) at fluid nodes; 0 elsewhere. rho/u may be NULL
 * (then rho0 and zero velocity). */
void or_init_eq(const or_params *p, const uint8_t *flags, const double *rho,
                const double *u, double *f);

/* One collide-stream-boundary update t -> t+1 (push form, two arrays).
 *   flags, q, uw, uw1 describe the geometry at time t; uw1 is the wall velocity
 *   at t+1 (NULL: same as uw; uw NULL: walls at rest).
 *   shell (N*Q or NULL): nonzero where link i of node n crosses a thin shell to
 *   the fluid node n - c_i: 1 when n lies outside the shell, 2 inside. Such a
 *   link is a wall link from both sides: neither node streams across it, and
 *   each writes its boundary value for the population coming back to it.
 *   f: pre-collision populations at t; fout: pre-collision populations at t+1.
 *   flink (N*Q*3 or NULL): momentum-exchange force of every wall link.
 * Returns 0, or -1 on bad arguments. */
int or_step(const or_params *p, const uint8_t *flags, const double *q,
            const uint8_t *shell, const double *uw, const double *uw1, const double *f,
            double *fout, double *flink);

/* rho[n], u[n*3 + d] (Guo-corrected velocity) at fluid nodes, 0 elsewhere. */
void or_macros(const or_params *p, const uint8_t *flags, const double *f,
               double *rho, double *u);

/* Sum of f over fluid nodes. */
double or_mass(const or_params *p, const uint8_t *flags, const double *f);

/* Nodes solid or open in flags_old and fluid in flags_new get f^eq(rho0, un[n]). */
void or_refill(const or_params *p, const uint8_t *flags_old, const uint8_t *flags_new,
               const double *un, double *f);

/* Local iteration refill (App. D, modified LIR; the paper gives it as a figure:
 * this is the reading the library follows). A node that is not fluid in
 * flags_old and fluid in flags_new (a fresh node) gets, for each direction i:
 *   - when its upstream node x - c_i was fluid at t: the post-collision value
 *     f*_i(x - c_i, t) computed from fprev, the state at t (what the step would
 *     have streamed to it);
 *   - otherwise: the value found by K local iterations of collide and bounce
 *     back at the node, which start from f^eq_i(rho0, un[n]) and then set the
 *     unknown f_i to the node's own post-collision f*_ibar plus the moving-wall
 *     term 2 w_i rho c_i.un[n] / c_s^2. The fluid at a fresh node moves with the
 *     body: the local collision is the step's (BGK or TRT, with the body force)
 *     at the node's density and the velocity un[n]. With the velocity held, each
 *     iteration contracts the error by |1 - 1/tau| or better (with the node's
 *     own velocity, bounce-back would flip its momentum every iteration).
 * f is the state at t+1, changed in place at fresh nodes only. */
void or_refill_lir(const or_params *p, const uint8_t *flags_old, const uint8_t *flags_new,
                   const double *un, const double *fprev, int K, double *f);

/* Link geometry from analytic shapes.
 *   base: caller flags (walls, inlet, outlet); a fluid base node inside any shape
 *   becomes solid. Links cut by a base-flag node get q = 1/2 and the wall
 *   velocity base_u[m*3..] of that node m (NULL: at rest), tag 0. Links cut by a
 *   shape get the exact q and u_w = v + om x (x_W - c) of the nearest crossing.
 *   A link between two fluid nodes on different sides of a thin shell (one
 *   inside, |x-c| < r0, one not) is cut from both sides; the inner side's
 *   links carry tag -1 (their momentum exchange is not counted as a force on
 *   the shell).
 *   Outputs: flags[N], q[N*Q], uw[N*Q*3], uw1[N*Q*3], tag[N*Q], shell[N*Q] (the
 *   marks or_step takes; any output but flags may be NULL). Returns the number
 *   of cut links, or -2 when a fluid node lies exactly on a thin shell (its
 *   links would have q = 0 on one side). */
long or_geometry(const or_params *p, const uint8_t *base, const double *base_u,
                 const or_shape *shapes, int nshapes, uint8_t *flags, double *q,
                 double *uw, double *uw1, int32_t *tag, uint8_t *shell);

/* Torque about the point c of the momentum exchange (flink from or_step) of the
 * links with the given tag (tag < 0: every wall link): T = sum (x_W - c) x F_link,
 * with x_W = x_F - q c_i the link's wall point (Sec. II.F; the moment of the
 * link forces of Eq. force-boundary-node). q and tag as or_geometry writes them. */
/* Number of OpenMP threads of the oracle's loops (n <= 0 keeps the current
 * setting); returns the number in use (1 without OpenMP). Used to time the
 * oracle on one core. */
int or_set_threads(int n);

void or_torque(const or_params *p, const double *q, const int32_t *tag, const double *flink, int want_tag,
               const double c[3], double T[3]);

/* Interpolation weights the boundary rule applies to its points, for tests:
 * writes up to 3 (s, a) pairs for the scheme at this q and returns their count. */
int or_bc_weights(int bc, double q, double qcut, double *s, double *a);

#ifdef __cplusplus
}
#endif
#endif
