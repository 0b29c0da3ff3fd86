// sim.hpp -- the simulation handle behind lbm_handle (host side).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "lattice.cuh"
#include "launch.hpp"

namespace lbm {
struct HostGeometry;
}

// A rigid body moving along a prescribed trajectory. Its link geometry is
// rebuilt on the device after every step, inside a fixed region box that covers
// the whole trajectory. The records are double-buffered by the population
// buffer index: set k serves the step that reads buffer k.
struct MovingBody {
  bool on = false;
  void *shape = nullptr;           // device copy of the body's shape (geometry kernels' type)
  double *traj = nullptr;          // device [ntraj][9]: centre, velocity, angular velocity per step
  int ntraj = 0;
  int ox = 0, oy = 0, oz = 0, rx = 1, ry = 1, rz = 1;  // region box
  long long rsize = 0, rpad = 0;   // region nodes; rounded up to 32
  lbm::Rec *rec[2] = {nullptr, nullptr};
  uint32_t *rnode[2] = {nullptr, nullptr};
  void *lq[2] = {nullptr, nullptr}, *luw[2] = {nullptr, nullptr}, *luw1[2] = {nullptr, nullptr};
  uint8_t *ltag[2] = {nullptr, nullptr};
  int *count[2] = {nullptr, nullptr};  // device: records in each set
  uint32_t *crec = nullptr, *clink = nullptr, *tot = nullptr, *totals = nullptr;  // scan scratch
  int *step = nullptr;             // device: index of the body's current pose
  long long cap_rec = 0, cap_link = 0;
  int tag = 0;
  double *fpart = nullptr;         // device: per-block momentum-exchange partials of the last step
  long long nfpart = 0;            // blocks
  unsigned long long hash = 0;     // FNV-1a of the body's shape and trajectory table
  // free rotation about a fixed axis through the body's centre, driven by the fluid torque
  bool free_rot = false;
  double *state = nullptr;         // device [angle, omega, c0, c1, c2, inertia]
  double centre[3] = {0.0, 0.0, 0.0};
  double *tpart = nullptr;         // device: per-block torque partials (about centre) of the last step
  double *hist = nullptr;          // device [hist_cap][3]: angle, omega, torque after each step
  int hist_cap = 0;
  int refill_mode = 0, refill_iters = 10;  // lbm_refill of fresh nodes, LIR iterations
  uint8_t *nkind = nullptr;        // device [rpad]: the region's kinds at the new pose (LIR)
};

struct lbm_sim {
  static constexpr int kGraphSteps = 32;  // steps per captured CUDA graph (even)

  int lattice = 0, Q = 9, dtype = 1;
  int nx = 1, ny = 1, nz = 1, nxp = 32;
  long long np = 0;  // padded nodes (population plane length)
  long long N = 0;   // nodes
  double tau = 1.0, rho0 = 1.0, qcut = 0.01;
  int collision = LBM_COLL_BGK;     // lbm_collision
  double magic = 3.0 / 16.0;        // TRT magic parameter Lambda
  int wall_neq = LBM_NEQ_BOUNCE_BACK;  // lbm_wall_neq
  double F[3] = {0.0, 0.0, 0.0};
  int has_force = 0, bc = 0, xshift = 0;

  cudaStream_t stream = nullptr;
  bool own_stream = false;

  void *f[2] = {nullptr, nullptr};  // population buffers; f[cur] holds the current state
  int cur = 0;
  uint8_t *flags = nullptr;
  uint32_t *amask = nullptr;  // [np] planes of a non-fluid node that take written-ahead values
  uint32_t *cbase = nullptr;
  lbm::Rec *rec = nullptr;
  uint32_t *rnode = nullptr;
  void *lq = nullptr, *luw = nullptr, *luw1 = nullptr;
  uint8_t *ltag = nullptr;
  long long nb = 0, nl = 0, nfluid = 0;
  int has_uw = 0;
  int has_shell = 0;  // the static geometry has links across thin shells
  unsigned long long geom_hash = 0;  // FNV-1a of the static geometry (flags, records, link data)

  double *dres = nullptr;     // reduction results (device)
  int *err_dev = nullptr;     // device error word (bit 0: a bounded wait ran out)
  unsigned long long *dbg_dev = nullptr;  // LBM_DEBUG builds: first out-of-range population index
  long long dbg_limit = -1;   // LBM_DEBUG builds: index limit of the checks (-1: Q x padded nodes)
  double *scratch = nullptr;  // per-block reduction partials (device)
  long long scratch_len = 0;
  double *stage_f = nullptr;  // FP64 staging of lbm_set/get_populations (N*Q, device; kept)
  long long wait_limit = 1LL << 24;  // first-wait poll limit of the TMA-staged step
  int refill_mode = 0, refill_iters = 10;  // lbm_set_refill, kept for bodies set later

  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // captured step loops, by starting buffer
  int2 *tiles = nullptr;      // step-kernel tile table (device)
  long long ntiles = 0;
  int2 *btiles = nullptr;     // split step (variants 9, 10): the boundary entries (device)
  long long nbtiles = 0;
  cudaStream_t aux = nullptr;                         // split step: the boundary kernel's stream
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;   // split step: orders aux around each step
  int tiles_bx = 0, tiles_by = 0;  // launch shape the table was built for (0: stale)
  int tiles_per_block = 4;          // consecutive table entries per step-kernel block (1..4)
  int tiles_var = -1;               // register variant the launch data was prepared for
  int tma_blocks = 0, tma_smem = 0; // persistent grid and shared memory of the TMA-staged step
  int step_bx = 32, step_by = 8, variant = 0;
  bool geom_ok = false, state_ok = false;
  int version = 0;  // bumped whenever the kernel view changes (options, geometry)
  MovingBody mb;
  std::string err;

  int npt() const { return variant >= 5 && variant <= 8 ? 2 : 1; }  // nodes per thread along x in lattice tiles
  bool split() const { return variant == 9 || variant == 10; }      // lattice and boundary kernels apart
  size_t elem_size() const;
  size_t link_size() const;
  void lattice_c(int i, int &x, int &y, int &z) const;
  double lattice_w(int i) const;
  lbm::View view() const;
  lbm::Launch shape(int bx, int by) const;
  lbm::Launch step_shape() const;
  lbm::Launch aux_shape() const;
  void tune_default();
  int ensure_scratch(long long doubles);
  void free_geometry();
  void drop_graphs();
  int launch_steps(int n);
  int ensure_tiles();
  int move_after_step(void *fout, int set);  // body geometry for the next step (geometry.cu)
  int move_rebuild(long long pose);          // body at pose index `pose`, records for f[cur] (geometry.cu)
  void free_moving_body();
  int capture(int parity);
  int upload(const lbm::HostGeometry &g);
  int download(lbm::HostGeometry &g);
  int finish_geometry();  // written-ahead masks and hash of the static geometry just set
  int ensure_stage_f();
};

int lbm_fail(lbm_sim *h, int code, const std::string &msg);
