// sim.hpp -- the simulation handle behind lbm_handle (host side).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "lattice.cuh"
#include "launch.hpp"

namespace lbm {
struct HostGeometry;
}

struct lbm_sim {
  static constexpr int kGraphSteps = 32;  // steps per captured CUDA graph (even)

  int lattice = 0, Q = 9, dtype = 1;
  int nx = 1, ny = 1, nz = 1, nxp = 32;
  long long np = 0;  // padded nodes (population plane length)
  long long N = 0;   // nodes
  double tau = 1.0, rho0 = 1.0, qcut = 0.01;
  double F[3] = {0.0, 0.0, 0.0};
  int has_force = 0, bc = 0, xshift = 0;

  cudaStream_t stream = nullptr;
  bool own_stream = false;

  void *f[2] = {nullptr, nullptr};  // population buffers; f[cur] holds the current state
  int cur = 0;
  uint8_t *flags = nullptr;
  uint32_t *cbase = nullptr;
  lbm::Rec *rec = nullptr;
  uint32_t *rnode = nullptr;
  void *lq = nullptr, *luw = nullptr, *luw1 = nullptr;
  uint8_t *ltag = nullptr;
  long long nb = 0, nl = 0, nfluid = 0;
  int has_uw = 0;

  double *dres = nullptr;     // reduction results (device)
  double *scratch = nullptr;  // per-block reduction partials (device)
  long long scratch_len = 0;

  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // captured step loops, by starting buffer
  int2 *tiles = nullptr;      // step-kernel tile table (device)
  long long ntiles = 0;
  int tiles_bx = 0, tiles_by = 0;  // launch shape the table was built for (0: stale)
  int tiles_per_block = 4;          // consecutive table entries per step-kernel block (1..4)
  int step_bx = 32, step_by = 8, variant = 0;
  bool geom_ok = false, state_ok = false;
  int version = 0;  // bumped whenever the kernel view changes (options, geometry)
  std::string err;

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
  int capture(int parity);
  int upload(const lbm::HostGeometry &g);
  int download(lbm::HostGeometry &g);
};

int lbm_fail(lbm_sim *h, int code, const std::string &msg);
