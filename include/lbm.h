/*
 * lbm.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann library liblbm.so.
 *
 * The library advances the lattice Boltzmann equation with BGK or TRT collision on
 * D2Q9, D3Q19 and D3Q27 lattices (Sec. II.A, Eqs. LBE, LB-BGK, Eq2ndOrder, magic-parameter
 * of arXiv:2009.04604) in one fused stream-collide kernel. On boundary nodes the
 * same kernel applies a link-wise curved-wall Dirichlet rule. The rules are ELIBB-F,
 * -FQ, -U and -UQ (Sec. II.D), linear BFL (Sec. II.B, Eq. bfl) and half-way bounce-back,
 * with the moving-wall term of Sec. II.E. Every rule takes its per-link wall
 * distance q and wall velocity u_w from the geometry. The momentum-exchange wall
 * force (Sec. II.F) and the total mass are reduced in FP64.
 *
 * Conventions for every call:
 *   - Every call returns an lbm_status (0 = LBM_OK). No call aborts or exits.
 *     lbm_last_error() gives a message for the last failing call on a handle.
 *   - Node index n = x + nx*(y + ny*z), with x fastest. D2Q9 uses nz = 1.
 *     The index space is periodic in every axis. Walls, inlets and outlets are
 *     nodes flagged non-fluid. Optionally the x axis is sheared-periodic: node
 *     (x + nx, y + xshift) is node (x, y).
 *   - Per-link arrays are indexed [n*Q + i]. Link i of node n joins n to
 *     n - c_i, the node its population i streams from. Directions follow this
 *     library's own order, which lbm_lattice_info() returns. Opposite
 *     directions satisfy opp(i) = Q - 1 - i.
 *   - Host arrays passed in are read during the call and copied. The caller
 *     keeps ownership. Device buffers passed in (lbm_macros) are caller-owned
 *     and are written on the handle's stream.
 *   - The handle owns all device state: populations, flags, boundary records
 *     and scratch. lbm_step() only enqueues work on the stream. Errors raised
 *     on the device show up at the next call that synchronises.
 *   - A handle must not be used by two host threads at the same time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_sim *lbm_handle;

enum lbm_lattice { LBM_D2Q9 = 0, LBM_D3Q19 = 1, LBM_D3Q27 = 2 };

/* Storage type of the populations. F64 computes in FP64. The others keep the
 * shifted value f_i - w_i rho0 in the stated format and compute in FP32. */
enum lbm_dtype { LBM_F64 = 0, LBM_F32 = 1, LBM_F16 = 2, LBM_BF16 = 3 };

/* Boundary rule on wall links:
 *   ELIBB_F  fragmented linear single-node rule (Sec. II.D, Eq. linear_broken_method);
 *   ELIBB_FQ fragmented quadratic rule, which falls back to ELIBB_F for
 *            q < 0.01 (Sec. II.D, Eq. quadratic_fragmented_method);
 *   BFL      linear Bouzidi rule (Sec. II.B, Eq. bfl). It falls back to half-way
 *            bounce-back where the second fluid node along the link is missing;
 *   HWBB     half-way bounce-back (Sec. II.B);
 *   ELIBB_U  unified linear rule through the two wall populations
 *            (Sec. II.D, Eq. unified_space_coordinates);
 *   ELIBB_UQ unified quadratic rule (Sec. II.D, Eq. elibbqu), which falls back
 *            to ELIBB_U for 1 - q < 0.01, where two of its points meet. */
enum lbm_bc { LBM_BC_ELIBB_F = 0, LBM_BC_ELIBB_FQ = 1, LBM_BC_BFL = 2, LBM_BC_HWBB = 3,
              LBM_BC_ELIBB_U = 4, LBM_BC_ELIBB_UQ = 5 };
/* Collision operators: BGK (Sec. II.A, Eq. LB-BGK) and two relaxation times
 * (Sec. II.A, TRT paragraph, Eq. magic-parameter). */
enum lbm_collision { LBM_COLL_BGK = 0, LBM_COLL_TRT = 1 };
/* Estimates of the non-equilibrium part of the ELIBB wall populations (Sec. II.D). */
enum lbm_wall_neq { LBM_NEQ_BOUNCE_BACK = 0, LBM_NEQ_REGULARIZED = 1 };

/* Node kinds. A link into an OPEN node gets the single-node pressure rule
 * f_i = f_i^eq(rho0, u_F) + f^neq_ibar(x_F), the non-equilibrium bounce-back of
 * Eq. neqbb-s applied at the reference density. */
enum lbm_node { LBM_FLUID = 0, LBM_SOLID = 1, LBM_OPEN = 2 };

enum lbm_status {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,       /* bad argument: null pointer, size, tau <= 1/2, q outside (0,1] */
  LBM_ERR_CUDA = -2,      /* a CUDA runtime call failed */
  LBM_ERR_OOM = -3,       /* device allocation failed */
  LBM_ERR_NONFINITE = -4, /* a reduction found NaN or Inf in the state */
  LBM_ERR_TIMEOUT = -5,   /* a bounded device wait ran out */
  LBM_ERR_STATE = -6,     /* call out of order, e.g. stepping before set_geometry */
  LBM_ERR_BOUNDS = -7     /* debug builds: a population index out of range (not accessed) */
};

/* Analytic shapes for lbm_build_geometry. A node is solid where the shape's test
 * holds (ties count as solid). A thin shell makes no node solid (see
 * lbm_build_geometry). */
enum lbm_shape_type {
  LBM_SHAPE_SPHERE = 0,     /* solid inside |x - c| <= r[0] (a circle on D2Q9)            */
  LBM_SHAPE_SPHERE_OUT = 1, /* solid outside |x - c| >= r[0]                               */
  LBM_SHAPE_ELLIPSOID = 2,  /* solid inside sum_d ((x - c)'_d / r[d])^2 <= 1, (x - c)' the
                               offset turned by -ang about the z axis (ang = 0: axis-aligned) */
  LBM_SHAPE_STRIP = 3,      /* fluid where |v| < width/2, with v = nrm.x - off. When
                               period > 0, v is first wrapped into [-period/2, period/2) */
  LBM_SHAPE_SHELL = 4       /* thin spherical shell |x - c| = r[0] >= 1 (a circle on D2Q9)
                               with fluid on both sides (Sec. III.B-III.C thin shells) */
};

typedef struct {
  int type;                 /* lbm_shape_type */
  int tag;                  /* force tag 0..7 given to every link the shape cuts */
  double c[3], r[3];        /* centre; radius r[0] or semi-axes r[0..2] */
  double nrm[3];            /* strip unit normal */
  double off, width, period;/* strip parameters */
  double v[3], om[3];       /* rigid velocity, angular velocity at time t */
  double v1[3], om1[3];     /* the same at time t+1 (wall population at s = 0) */
  double ang;               /* ellipsoid: rotation about the z axis (radians); its semi-axes
                               r[0], r[1] lie along (cos ang, sin ang) and (-sin ang, cos ang) */
} lbm_shape;

/* Lattice tables in this library's direction order: c[i*3 + d], w[i].
 * Either output may be NULL. Writes *Q. */
int lbm_lattice_info(int lattice, int *Q, int *c, double *w);

/* Create a simulation on the current CUDA device. dims = {nx, ny, nz}; nz must
 * be 1 for D2Q9. tau > 1/2 is the BGK relaxation time, Omega = 1/tau (Eq. LB-BGK).
 * stream is a cudaStream_t (NULL = legacy default stream). Allocates the two
 * population buffers and the flags. The state starts uninitialised: call
 * lbm_set_geometry or lbm_build_geometry, then lbm_init or lbm_set_populations. */
int lbm_create(int lattice, const int dims[3], double tau, int dtype, void *stream,
               lbm_handle *out);
int lbm_destroy(lbm_handle h);

/* Boundary rule (lbm_bc), reference density rho0 (default 1), constant body-force
 * density F (Guo forcing; NULL = none) and the x-wrap shear (0 = plain periodic). */
int lbm_set_options(lbm_handle h, int bc, double rho0, const double force[3], int xshift);

/* Collision operator (lbm_collision; BGK by default). Under TRT the even parts of
 * the populations relax with omega+ = 1/tau and the odd parts with omega-, from
 * the magic parameter Lambda = (1/omega+ - 1/2)(1/omega- - 1/2) (Eq.
 * magic-parameter; the paper uses Lambda = 3/16, with which half-way bounce-back
 * puts a flat wall exactly half-way at any tau). With Guo forcing, the even and
 * odd parts of the source take the factors (1 - omega+/2) and (1 - omega-/2).
 * The boundary rules use the TRT post-collision values; their post-collision
 * wall estimate keeps the factor (1 - omega+). magic is ignored for BGK and must
 * be positive for TRT; otherwise LBM_ERR_ARG. Takes effect at the next step. */
int lbm_set_collision(lbm_handle h, int model, double magic);

/* Non-equilibrium part of the ELIBB wall populations (lbm_wall_neq):
 *   NEQ_BOUNCE_BACK (default): f^neq_ibar(x_F), the node's own opposite
 *     population (Eq. neqbb-s);
 *   NEQ_REGULARIZED: the Hermite reconstruction of the appendix's Eq. fi_neq,
 *     truncated at third order. The second-order coefficient is the node's
 *     non-equilibrium stress (the wall's stress taken as the node's); the third
 *     follows from the isothermal recursion (Eq. malaspinas) with the wall
 *     velocity at each wall population's time. On D3Q19, which lacks part of the
 *     third-order Hermite set, the reconstruction is exact up to O(Ma^2).
 * Open (outlet) links keep the bounce-back estimate. Takes effect at the next
 * step; LBM_ERR_ARG for an unknown mode. */
int lbm_set_wall_neq(lbm_handle h, int mode);

/* Explicit geometry from host arrays.
 *   flags[N]: lbm_node per node.
 *   q[N*Q]: wall distance of each wall link (a fluid node n with a SOLID node
 *     n - c_i), as a fraction of |c_i| in (0,1]. NULL means every wall link has q = 1/2.
 *   uw[N*Q*3], uw1[N*Q*3]: wall velocity at the wall point at t and at t+1.
 *     NULL uw means walls at rest. NULL uw1 means the same as uw.
 *   tag[N*Q]: force tag 0..7 of each wall link. NULL means tag 0.
 * Entries of links that are not wall links are ignored. Returns LBM_ERR_ARG
 * for a wall link with q outside (0,1] or a tag outside 0..7. */
int lbm_set_geometry(lbm_handle h, const uint8_t *flags, const double *q, const double *uw,
                     const double *uw1, const int32_t *tag);

/* Geometry computed on the device from analytic shapes (link-geometry kernel).
 *   base[N] (host, may be NULL): the caller's nodes (walls, inlet, outlet). A
 *     fluid base node inside any shape becomes SOLID.
 *   base_u[N*3] (host, may be NULL): velocity of the SOLID base nodes.
 * A wall link cut by a base node gets q = 1/2 and that node's velocity, tag 0.
 * A link cut by a shape gets the exact crossing q, the smallest t in (0,1] at
 * which x_F - t c_i reaches the shape, and the rigid-motion velocity
 * v + om x (x_W - c) at the wall point x_W = x_F - q c_i. At most 65536 shapes.
 * Thin shells: a link between two fluid nodes, one strictly inside the shell
 * (|x - c| < r[0]) and one not, is a wall link of both nodes, each with its own
 * q (the two add up to 1). Neither node streams across it: each applies the
 * boundary rule to the population coming back to it, and writes that value into
 * the slot the other node would have stored. The links on the inner side carry
 * no force (lbm_wall_force counts the outer fluid only, as for the filled body
 * of Sec. III.C) and read back with tag -1 from lbm_get_geometry. A shell must
 * keep at least one node away from the lattice's edges and from other shapes
 * (two crossings within one link are not represented). LBM_ERR_ARG when a fluid
 * node lies exactly on a shell (its links would have q = 0 on one side).
 * lbm_set_geometry cannot express thin shells, and a geometry with thin shells
 * takes no moving body. */
int lbm_build_geometry(lbm_handle h, const uint8_t *base, const double *base_u,
                       const lbm_shape *shapes, int nshapes);

/* A rigid body moving on a prescribed trajectory: a sphere or an axis-aligned
 * ellipsoid (body->type, r, tag; its c, v and om fields are ignored).
 *   traj[ntraj*9] (host, FP64): for pose k, the centre c[3], velocity v[3] and
 *     angular velocity om[3]. Step t uses pose (t0 + t) mod ntraj, so a periodic
 *     path needs one period of poses.
 * After every step the library rebuilds the body's link geometry on the device
 * (the link-geometry kernel, restricted to a region box that covers the whole
 * trajectory): node kinds, q and u_w = v + om x (x_W - c) at the new pose, and
 * u_w at the following pose for the wall population at s = 0 (Sec. II.D-II.E).
 * A node that turns fluid is refilled (lbm_set_refill: f^eq(rho0, u_body) by
 * default, or the local iteration refill of App. D). A node that turns solid is
 * dropped. The region, widened
 * by one node, must lie inside the lattice and hold only fluid nodes of the
 * static geometry; otherwise LBM_ERR_ARG. BFL is not available with a moving
 * body. Call after lbm_build_geometry/lbm_set_geometry; a new static geometry
 * removes the body. lbm_wall_force includes the body's links (its tag). */
int lbm_set_moving_body(lbm_handle h, const lbm_shape *body, const double *traj, int ntraj, int t0);

/* A rigid body turning freely about the z axis through its centre under the
 * fluid's torque, the coupling of Sec. III.C (Jeffery's orbit): a sphere or an
 * ellipsoid (body->type, c, r, ang = initial rotation about z, om[2] = initial
 * angular velocity, tag). inertia: its moment of inertia about that axis, in
 * lattice units (mass x length^2; per unit length on D2Q9). After every step the
 * library reduces, on the device and in FP64, the torque T about the centre of
 * the momentum exchange of the body's links (as lbm_wall_torque), then turns the
 * body: omega += T / inertia, angle += omega (semi-implicit Euler, unit time
 * step), and rebuilds its link geometry at the new angle, with wall velocity
 * omega x (x_W - c) at t and t+1 alike (the next torque is not known yet). Nodes
 * it uncovers are refilled as for lbm_set_moving_body. The centre does not move.
 * history: number of steps of (angle, omega, torque) kept on the device (read
 * with lbm_get_body_history). The same conditions as lbm_set_moving_body apply to
 * the region the body sweeps (a disc of its largest in-plane semi-axis). */
int lbm_set_free_body(lbm_handle h, const lbm_shape *body, double inertia, int history);

/* The last min(*n, steps taken, history) entries of a free body's history, in
 * step order: out[3*k + {0, 1, 2}] = angle and angular velocity after the step,
 * and the torque of the step. out NULL: writes the number available into *n.
 * Synchronises. LBM_ERR_STATE without a free body. */
int lbm_get_body_history(lbm_handle h, double *out, int64_t *n);

/* Refill of the nodes a moving or free body uncovers (fresh nodes):
 *   REFILL_EQUILIBRIUM (default): every population of a fresh node becomes
 *     f^eq_i(rho0, u_b), u_b the body's velocity at the node;
 *   REFILL_LIR: local iteration refill, the reading of the paper's modified LIR
 *     (App. D, given there as a figure): the populations streamed to the node
 *     from upstream nodes that were fluid are kept; the others are found by
 *     `iterations` local iterations of collide-and-bounce-back at the node,
 *     from f^eq(rho0, u_b), colliding at the node's density and the velocity
 *     u_b and bouncing back the node's own post-collision values with the
 *     moving-wall term. Each iteration contracts the error by about |1 - 1/tau|
 *     or better; nodes with few streamed values converge slowest.
 * Applies to the body set now and to bodies set later. LBM_ERR_ARG for an unknown
 * mode or iterations outside 0..100000. */
enum lbm_refill { LBM_REFILL_EQUILIBRIUM = 0, LBM_REFILL_LIR = 1 };
int lbm_set_refill(lbm_handle h, int mode, int iterations);

/* Equilibrium start f = f^eq(rho, u) on every fluid node. */
int lbm_init(lbm_handle h, double rho, const double u[3]);

/* Pre-collision populations at the current time, as host FP64 arrays
 * f[n*Q + i], unshifted, in this library's direction order. Non-fluid entries are
 * ignored on set and written as 0 on get. */
int lbm_set_populations(lbm_handle h, const double *f);
int lbm_get_populations(lbm_handle h, double *f);

/* Enqueue n fused stream-collide-boundary steps on the handle's stream. The
 * steps are replayed from a captured CUDA graph. */
int lbm_step(lbm_handle h, int n);

/* Density rho[N] and Guo-corrected velocity u[N*3] ((sum c f + F/2)/rho, Guo
 * forcing) of the current state. Both are device FP64 buffers owned by the
 * caller; either may be NULL. Non-fluid nodes get 0. Asynchronous on the stream. */
int lbm_macros(lbm_handle h, double *rho, double *u);

/* Momentum-exchange force (Sec. II.F, Eq. force-boundary-node, outgoing
 * population f*_ibar as in Wen et al.) of the last step. It sums
 * (c_ibar - u_w) f*_ibar(x_F, t) - (c_i - u_w) f_i(x_F, t+1) over the wall links
 * with this tag (tag = -1 sums every tag). Accumulated in FP64 in a fixed
 * order, so the result is deterministic. Synchronises the stream. On the outer
 * side of a thin shell f*_ibar(x_F, t) is not kept in memory (the slot holds the
 * value written from the other side): it is computed again from the state the
 * last step read, so call this right after a step. */
int lbm_wall_force(lbm_handle h, int tag, double F[3]);

/* Torque about the point centre[3] of the momentum exchange of the last step
 * (Sec. II.F): the sum over the static geometry's wall links with this tag (-1:
 * every tag) of (x_W - centre) x F_link, where F_link is the link's term of
 * lbm_wall_force and x_W = x_F - q c_i the link's wall point. FP64, fixed order,
 * deterministic. Synchronises the stream. A free body's own torque is in
 * lbm_get_body_history. */
int lbm_wall_torque(lbm_handle h, int tag, const double centre[3], double T[3]);

/* Total mass sum of rho over the fluid nodes, in FP64. Deterministic. Synchronises.
 * Returns LBM_ERR_NONFINITE if the sum is NaN or Inf. */
int lbm_mass(lbm_handle h, double *m);

/* Capacity of the static scratch array of lbm_mass_noalloc, in per-block
 * partial sums: 131072 doubles (1 MiB). Every GPU that loads the library holds
 * it until the process exits. */
#define LBM_NOALLOC_MAX_PARTIALS 131072

/* Total mass, as lbm_mass computes it, without allocating device memory. The
 * paper has no counterpart: this exists for callers that cannot call cudaMalloc.
 * Examples are monitoring code inside a step loop that must not stall on the
 * allocator (cudaMalloc and cudaFree can synchronise the device), and processes
 * where another allocator already holds the device memory.
 *   mass_dev: caller-owned device pointer to one double. The sum is written there
 *     on the handle's stream; the call does not wait for it. Unlike lbm_mass, it
 *     does not check the value for NaN or Inf.
 * The per-block partial sums live in a file-scope static device array of
 * LBM_NOALLOC_MAX_PARTIALS doubles. The reduction uses one block per 32 x 8
 * nodes of a z-plane, (nx rounded up to 32)/32 * ceil(ny/8) * nz blocks. A
 * lattice that needs more (above about 33.5 million padded nodes) gets
 * LBM_ERR_ARG. The first call on a device looks up the array's device address,
 * once per device: make that call with the handle's device current and before
 * any stream capture. Every call reuses the same array, and each call writes
 * every partial it reads. Calls whose work overlaps on the GPU, for instance on
 * two streams, race on the array and give wrong sums: serialise them. */
int lbm_mass_noalloc(lbm_handle h, double *mass_dev);

/* Read back the geometry the library holds, for checks: flags[N] (lbm_node),
 * q/uw/uw1/tag per link [N*Q(*3)]. Non-wall links read 0; links on the inner
 * side of a thin shell read tag -1. Any pointer may be NULL. */
int lbm_get_geometry(lbm_handle h, uint8_t *flags, double *q, double *uw, double *uw1,
                     int32_t *tag);

/* Counts of the current geometry: fluid nodes, boundary nodes, wall links. */
int lbm_get_counts(lbm_handle h, int64_t *n_fluid, int64_t *n_boundary, int64_t *n_links);

/* Checkpoint and resume. The paper has no counterpart: these keep a run's state
 * so that a resumed run continues bit for bit.
 * lbm_save writes the state into the caller's host buffer buf of *bytes bytes:
 * a header (lattice, storage type, size, boundary rule, reference density, a
 * 64-bit hash of the static geometry, the moving body's identity and pose
 * index) and the raw stored populations of the current time, the values the
 * last step wrote ahead for the next one included. With buf NULL it only writes
 * the size needed into *bytes. LBM_ERR_ARG when *bytes is too small;
 * LBM_ERR_STATE before a state exists. Synchronises.
 * lbm_load restores such a state into a handle built with the same lattice,
 * storage type, size, boundary rule, reference density, static geometry and
 * moving body (checked against the header: LBM_ERR_ARG otherwise). Relaxation
 * time, body force and collision are not checked; a resumed run is bitwise
 * identical to an uninterrupted one when they are the same. A moving body
 * resumes at the saved pose. The wall force of the step before the save is not
 * part of the state. Synchronises. */
int lbm_save(lbm_handle h, void *buf, size_t *bytes);
int lbm_load(lbm_handle h, const void *buf, size_t bytes);

/* Testing aid for failure detection: how many times a first wait of the
 * TMA-staged step (launch variant 4) polls its mbarrier before it counts as
 * hung (default 2^24; a negative value restores it; 0 makes every such wait
 * run out at once). A wait that runs out sets the handle's device error word,
 * the block waits for its own copies in flight (always with the default limit)
 * and leaves, and the next lbm_synchronize returns LBM_ERR_TIMEOUT and clears
 * the word. The state is then incomplete: re-initialise it. The paper has no
 * counterpart. */
int lbm_set_wait_limit(lbm_handle h, long long polls);

/* Bounds-checked builds. A library compiled with LBM_DEBUG checks every element
 * index of a population load or store in the step, set-up, read-out and force
 * kernels against [0, limit), limit = Q x padded nodes (the buffer's size) by
 * default. An index outside is not accessed (a load reads 0); the first one, with
 * the source line of the access, is kept in a device word per handle, and the
 * next lbm_synchronize returns LBM_ERR_BOUNDS and clears it. The state is then
 * wrong: re-initialise it. The paper has no counterpart; this stands in for a
 * memory checker.
 * lbm_is_debug_build: 1 for such a build, 0 otherwise.
 * lbm_set_debug_limit: testing aid, sets the limit (negative: the default); a
 * limit below the buffer's size makes accesses inside the buffer count as out of
 * range, which exercises the checks without touching memory outside the
 * buffers. LBM_ERR_STATE in a build without LBM_DEBUG. */
int lbm_is_debug_build(void);
int lbm_set_debug_limit(lbm_handle h, long long elements);

/* Launch configuration of the step kernel:
 *   bx x by threads per block: bx a multiple of 32 that divides the padded row
 *     length, bx*by <= 256;
 *   variant 0..3: the register budget. Variant v guarantees v+1 resident
 *     256-thread blocks per SM;
 *   variant 4: the TMA-staged persistent kernel. The first warp of a block copies
 *     each lattice tile's source rows into shared memory with bulk asynchronous
 *     copies, several tiles ahead, and the block computes from there. FP32,
 *     FP16 and BF16 only;
 *   variant 5..7: two nodes per thread along x, with vector loads and stores,
 *     at least 1..3 resident 256-thread blocks per SM. A block covers 2*bx nodes
 *     of a row, which must divide the padded row. FP32/FP16/BF16, not with BFL
 *     (switching to BFL moves the launch back to variant 0);
 *   variant 8: as 5..7, for blocks of exactly 128 threads, at least 7 resident
 *     per SM (72 registers a thread);
 *   variant 9, 10: the split step. The lattice tiles and the boundary-record
 *     tiles run as two kernels side by side in each step: the boundary kernel
 *     on a second stream of the handle (highest priority), forked from and
 *     joined back into the handle's stream around every step, so that nothing
 *     after the step starts before both finish. The lattice kernel keeps at
 *     least 6 (variant 9: 40 registers a thread) or 5 (variant 10: 48) resident
 *     256-thread blocks per SM, the boundary kernel at least 4. One node per
 *     thread; FP32/FP16/BF16. The results are those of variants 0..3;
 *   variant 11, 12: as 0..3, with at least 5 (48 registers a thread) or 6 (40)
 *     resident 256-thread blocks per SM. FP32/FP16/BF16;
 *   tiles 1..4: consecutive entries of the step kernel's tile table that one
 *     block processes. The table lists, plane by plane, the lattice tiles and
 *     then the boundary-record tiles (variants 9, 10: the lattice tiles; each
 *     block of the boundary kernel takes one boundary-record tile).
 * FP64 storage accepts variant 0 only, and on D3Q27 at most 128 threads per block
 * (27 x 256 doubles of boundary staging would exceed the static shared memory).
 * The default is the widest bx <= 128 that divides the row, by = 256/bx (128/bx
 * for FP64 on D3Q27), variant 0, tiles 4. LBM_ERR_ARG for an invalid
 * configuration. */
int lbm_set_launch(lbm_handle h, int bx, int by, int variant, int tiles);
int lbm_get_launch(lbm_handle h, int *bx, int *by, int *variant, int *tiles);

/* Autotuner: runs `steps` steps with each candidate configuration and keeps the
 * fastest. The candidates are 128- and 256-thread blocks, every admissible bx,
 * every register variant, and 1, 2 or 4 tiles per block. Each is timed with
 * CUDA events. The simulation advances by every trial step. Writes the chosen
 * configuration and its time per step in ms; any output may be NULL.
 * Synchronises the stream. */
int lbm_autotune(lbm_handle h, int steps, int *bx, int *by, int *variant, int *tiles,
                 double *ms_per_step);

/* ---- Batches: many independent simulations advanced by one launch per step ----
 * The simulations of a batch share one lattice, one storage type and one stream,
 * and each keeps its own geometry, parameters and state. A batched step runs the
 * same per-node code as lbm_step, so each simulation gets exactly the results it
 * would get alone. The blocks of the launch take the tiles of every simulation
 * (lattice tiles and boundary-record tiles, plane by plane), and the steps replay
 * from captured CUDA graphs. This is for workloads of many small or uneven grids,
 * where one launch per simulation would leave the GPU idle between launches. The
 * handles stay usable on their own; lbm_batch_step picks up their current state. */
typedef struct lbm_batch_s *lbm_batch;

/* sims: n distinct handles, each with geometry and state, all with the same
 * lattice, dtype and stream, none with a moving body. Returns LBM_ERR_ARG or
 * LBM_ERR_STATE otherwise. The batch does not own the handles: destroy the batch
 * first. */
int lbm_batch_create(const lbm_handle *sims, int n, lbm_batch *out);
int lbm_batch_destroy(lbm_batch b);

/* Enqueue n steps of every simulation of the batch on the shared stream. */
int lbm_batch_step(lbm_batch b, int n);

/* Launch configuration and autotuner of the batched step, as lbm_set_launch and
 * lbm_autotune. bx must divide the padded row length of every simulation. The
 * autotuner advances every simulation by its trial steps. */
int lbm_batch_set_launch(lbm_batch b, int bx, int by, int variant, int tiles);
int lbm_batch_autotune(lbm_batch b, int steps, int *bx, int *by, int *variant, int *tiles,
                       double *ms_per_step);

/* Message of the last error on a batch. */
const char *lbm_batch_last_error(lbm_batch b);

/* Wait for all work on the handle's stream. */
int lbm_synchronize(lbm_handle h);

/* Message of the last error on this handle (or of the last failed lbm_create
 * when h is NULL). The string stays valid until the next call on h. */
const char *lbm_last_error(lbm_handle h);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
