// runtime.cu -- host runtime of liblbm: the C ABI of include/lbm.h.
//
// Owns the device state of a simulation: the two population buffers (A-B
// pull), node flags, boundary records and per-link wall data, and the scratch
// for the FP64 reductions. It builds boundary records from explicit host
// geometry and captures the step loop in CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "geometry.hpp"
#include "launch.hpp"
#include "sim.hpp"
#include "kernels.cuh"

using namespace lbm;

static std::string g_create_error;

int lbm_fail(lbm_sim *h, int code, const std::string &msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return code;
}

#define LBM_CUDA(h, call)                                                                        \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return lbm_fail((h), e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,         \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

// ---------------------------------------------------------------- lattice info
template <class L>
static void fill_info(int *c, double *w) {
  for (int i = 0; i < L::Q; ++i) {
    if (c) { c[i * 3] = L::cx(i); c[i * 3 + 1] = L::cy(i); c[i * 3 + 2] = L::cz(i); }
    if (w) w[i] = weight<L>(i);
  }
}

extern "C" int lbm_lattice_info(int lattice, int *Q, int *c, double *w) {
  if (lattice == LBM_D2Q9) { if (Q) *Q = 9; fill_info<D2Q9>(c, w); return LBM_OK; }
  if (lattice == LBM_D3Q19) { if (Q) *Q = 19; fill_info<D3Q19>(c, w); return LBM_OK; }
  if (lattice == LBM_D3Q27) { if (Q) *Q = 27; fill_info<D3Q27>(c, w); return LBM_OK; }
  return lbm_fail(nullptr, LBM_ERR_ARG, "unknown lattice");
}

void lbm_sim::lattice_c(int i, int &x, int &y, int &z) const {
  if (lattice == LBM_D2Q9) { x = D2Q9::cx(i); y = D2Q9::cy(i); z = 0; }
  else if (lattice == LBM_D3Q19) { x = D3Q19::cx(i); y = D3Q19::cy(i); z = D3Q19::cz(i); }
  else { x = D3Q27::cx(i); y = D3Q27::cy(i); z = D3Q27::cz(i); }
}

double lbm_sim::lattice_w(int i) const {
  return lattice == LBM_D2Q9 ? weight<D2Q9>(i) : (lattice == LBM_D3Q19 ? weight<D3Q19>(i) : weight<D3Q27>(i));
}

size_t lbm_sim::elem_size() const {
  return dtype == LBM_F64 ? 8 : (dtype == LBM_F32 ? 4 : 2);
}

size_t lbm_sim::link_size() const { return dtype == LBM_F64 ? 8 : 4; }

// ---------------------------------------------------------------- create / destroy
extern "C" int lbm_create(int lattice, const int dims[3], double tau, int dtype, void *stream,
                          lbm_handle *out) {
  if (!out || !dims) return lbm_fail(nullptr, LBM_ERR_ARG, "null argument");
  *out = nullptr;
  if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19 && lattice != LBM_D3Q27)
    return lbm_fail(nullptr, LBM_ERR_ARG, "unknown lattice");
  if (dtype < LBM_F64 || dtype > LBM_BF16) return lbm_fail(nullptr, LBM_ERR_ARG, "unknown dtype");
  if (!(tau > 0.5)) return lbm_fail(nullptr, LBM_ERR_ARG, "tau must exceed 1/2");
  if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return lbm_fail(nullptr, LBM_ERR_ARG, "dims must be positive");
  if (lattice == LBM_D2Q9 && dims[2] != 1) return lbm_fail(nullptr, LBM_ERR_ARG, "D2Q9 needs nz = 1");
  const long long nxp = (dims[0] + 31) / 32 * 32;
  const long long np = nxp * dims[1] * (long long)dims[2];
  const long long Qn = lattice == LBM_D2Q9 ? 9 : (lattice == LBM_D3Q19 ? 19 : 27);
  if (np * Qn >= (1LL << 31))
    return lbm_fail(nullptr, LBM_ERR_ARG, "grid too large: Q x padded nodes must stay below 2^31");
  lbm_sim *h = new lbm_sim();
  h->lattice = lattice;
  h->Q = (int)Qn;
  h->dtype = dtype;
  h->nx = dims[0]; h->ny = dims[1]; h->nz = dims[2];
  h->nxp = (int)nxp;
  h->np = np;
  h->N = (long long)dims[0] * dims[1] * dims[2];
  h->tau = tau;
  if (stream) {
    h->stream = static_cast<cudaStream_t>(stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete h; return lbm_fail(nullptr, LBM_ERR_CUDA, cudaGetErrorString(e)); }
    h->own_stream = true;
  }
  const size_t bytes = (size_t)h->Q * np * h->elem_size();
  cudaError_t e = cudaMalloc(&h->f[0], bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->f[1], bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->flags, np);
  if (e == cudaSuccess) e = cudaMalloc(&h->amask, np * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->amask, 0xff, np * sizeof(uint32_t), h->stream);
  if (e == cudaSuccess) e = cudaMalloc(&h->cbase, (np / 32 + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->dres, 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->err_dev, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaMalloc(&h->dbg_dev, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->dbg_dev, 0, sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->flags, K_PAD, np, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->f[0], 0, bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->f[1], 0, bytes, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    std::string msg = std::string("allocation: ") + cudaGetErrorString(e);
    lbm_destroy(h);
    return lbm_fail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, msg);
  }
  h->tune_default();
  *out = h;
  return LBM_OK;
}

void lbm_sim::free_geometry() {
  cudaFree(rec); cudaFree(rnode); cudaFree(lq); cudaFree(luw); cudaFree(luw1); cudaFree(ltag);
  rec = nullptr; rnode = nullptr; lq = nullptr; luw = nullptr; luw1 = nullptr; ltag = nullptr;
  nb = nl = 0;
  has_uw = 0;
  geom_hash = 0;
}

int lbm_sim::ensure_stage_f() {
  if (stage_f) return LBM_OK;
  LBM_CUDA(this, cudaMalloc(&stage_f, (size_t)N * Q * sizeof(double)));
  return LBM_OK;
}

// 64-bit FNV-1a over 8-byte words (the tail byte by byte)
static unsigned long long fnv_words(unsigned long long h, const void *p, size_t n) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  size_t k = 0;
  for (; k + 8 <= n; k += 8) {
    unsigned long long w;
    std::memcpy(&w, b + k, 8);
    h = (h ^ w) * 0x100000001b3ULL;
  }
  for (; k < n; ++k) h = (h ^ b[k]) * 0x100000001b3ULL;
  return h;
}

// After a static geometry is in place: the written-ahead masks of the non-fluid
// nodes (View::amask) and the geometry's hash (for lbm_save / lbm_load).
int lbm_sim::finish_geometry() {
  LBM_CUDA(this, launch_amask(lattice, view(), amask, stream));
  HostGeometry g;
  int rc = download(g);
  if (rc) return rc;
  unsigned long long h = 0xcbf29ce484222325ULL;
  const long long dims[5] = {lattice, nx, ny, nz, dtype};
  h = fnv_words(h, dims, sizeof(dims));
  h = fnv_words(h, g.flags.data(), g.flags.size());
  h = fnv_words(h, g.rec.data(), g.rec.size() * sizeof(Rec));
  h = fnv_words(h, g.rnode.data(), g.rnode.size() * sizeof(uint32_t));
  h = fnv_words(h, g.lq.data(), g.lq.size());
  h = fnv_words(h, g.ltag.data(), g.ltag.size());
  h = fnv_words(h, g.luw.data(), g.luw.size());
  h = fnv_words(h, g.luw1.data(), g.luw1.size());
  geom_hash = h;
  return LBM_OK;
}

void lbm_sim::drop_graphs() {
  for (int k = 0; k < 2; ++k)
    if (graph[k]) { cudaGraphExecDestroy(graph[k]); graph[k] = nullptr; }
}

extern "C" int lbm_destroy(lbm_handle h) {
  if (!h) return LBM_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  h->drop_graphs();
  h->free_geometry();
  cudaFree(h->f[0]); cudaFree(h->f[1]); cudaFree(h->flags); cudaFree(h->cbase);
  cudaFree(h->dres); cudaFree(h->scratch); cudaFree(h->tiles); cudaFree(h->err_dev); cudaFree(h->dbg_dev);
  cudaFree(h->btiles);
  cudaFree(h->amask); cudaFree(h->stage_f);
  h->free_moving_body();
  if (h->aux) { cudaStreamSynchronize(h->aux); cudaStreamDestroy(h->aux); }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return LBM_OK;
}

extern "C" const char *lbm_last_error(lbm_handle h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

extern "C" int lbm_synchronize(lbm_handle h) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  int err = 0;
  LBM_CUDA(h, cudaMemcpy(&err, h->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    cudaMemset(h->err_dev, 0, sizeof(int));
    return lbm_fail(h, LBM_ERR_TIMEOUT, "a bounded wait in the step kernel ran out; the step is incomplete");
  }
#ifdef LBM_DEBUG
  unsigned long long word = 0;
  LBM_CUDA(h, cudaMemcpy(&word, h->dbg_dev, sizeof(word), cudaMemcpyDeviceToHost));
  if (word) {
    cudaMemset(h->dbg_dev, 0, sizeof(word));
    char msg[160];
    std::snprintf(msg, sizeof msg,
                  "population index %lld (mod 2^40) out of range [0, %lld) at kernels.cuh line %llu; not accessed",
                  (long long)(word & ((1ull << 40) - 1ull)), h->view().dbg_limit, word >> 40);
    return lbm_fail(h, LBM_ERR_BOUNDS, msg);
  }
#endif
  return LBM_OK;
}

extern "C" int lbm_set_options(lbm_handle h, int bc, double rho0, const double force[3], int xshift) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  if (bc < LBM_BC_ELIBB_F || bc > LBM_BC_ELIBB_UQ) return lbm_fail(h, LBM_ERR_ARG, "unknown boundary rule");
  if (bc == LBM_BC_BFL && h->mb.on)
    return lbm_fail(h, LBM_ERR_ARG, "BFL needs a second node along the link, which a moving body's records do not carry");
  if (!(rho0 > 0.0) || !std::isfinite(rho0)) return lbm_fail(h, LBM_ERR_ARG, "rho0 must be positive");
  if (h->geom_ok && h->state_ok && rho0 != h->rho0)
    return lbm_fail(h, LBM_ERR_STATE, "rho0 changes the stored shift: set it before the state");
  if (h->geom_ok && h->state_ok && (bc == LBM_BC_BFL) != (h->bc == LBM_BC_BFL)) {
    // BFL keeps a partial value in its written-ahead slots: re-encode the state
    int rc = h->ensure_stage_f();
    if (rc) return rc;
    double *d = h->stage_f;
    cudaError_t e = launch_read(h->lattice, h->dtype, h->view(), h->f[h->cur], d, nullptr, nullptr,
                                nullptr, h->aux_shape());
    const int old_bc = h->bc;
    h->bc = bc;
    if (e == cudaSuccess) e = launch_set_pop(h->lattice, h->dtype, h->view(), h->f[h->cur], d, h->aux_shape());
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { h->bc = old_bc; return lbm_fail(h, LBM_ERR_CUDA, cudaGetErrorString(e)); }
  }
  h->bc = bc;
  if (bc == LBM_BC_BFL && h->npt() == 2) { h->variant = 0; h->tune_default(); }  // pairs have no BFL path
  h->rho0 = rho0;
  h->has_force = 0;
  for (int a = 0; a < 3; ++a) {
    h->F[a] = force ? force[a] : 0.0;
    if (h->F[a] != 0.0) h->has_force = 1;
  }
  if (h->lattice == LBM_D2Q9) { h->F[2] = 0.0; }
  h->xshift = xshift;
  h->drop_graphs();
  h->tiles_var = -1;  // the TMA-staged step is prepared per force path
  ++h->version;
  return LBM_OK;
}

extern "C" int lbm_set_wall_neq(lbm_handle h, int mode) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  if (mode != LBM_NEQ_BOUNCE_BACK && mode != LBM_NEQ_REGULARIZED)
    return lbm_fail(h, LBM_ERR_ARG, "unknown wall non-equilibrium estimate");
  h->wall_neq = mode;
  h->drop_graphs();
  ++h->version;
  return LBM_OK;
}

extern "C" int lbm_set_collision(lbm_handle h, int model, double magic) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  if (model != LBM_COLL_BGK && model != LBM_COLL_TRT) return lbm_fail(h, LBM_ERR_ARG, "unknown collision model");
  if (model == LBM_COLL_TRT && !(magic > 0.0 && std::isfinite(magic)))
    return lbm_fail(h, LBM_ERR_ARG, "the TRT magic parameter must be positive");
  h->collision = model;
  if (model == LBM_COLL_TRT) h->magic = magic;
  h->drop_graphs();
  h->tiles_var = -1;  // the TMA-staged step is prepared per collision
  ++h->version;
  return LBM_OK;
}

// ---------------------------------------------------------------- kernel view, launch shapes
// Multiplier and shift of the quotient t / d by one wide multiply (div_by in
// kernels.cuh): l = floor(log2 d), m = ceil(2^(32+l) / d) and s = 32 + l, or
// m = 2^31 and s = 31 + l for a power of two.
static void invariant_divisor(long long dd, uint32_t *m, uint32_t *s) {
  const unsigned long long d = (unsigned long long)(dd > 0 ? dd : 1);
  unsigned l = 0;
  while ((2ull << l) <= d) ++l;
  if ((d & (d - 1)) == 0) { *m = 1u << 31; *s = 31 + l; }
  else { *m = (uint32_t)(((1ull << (32 + l)) + d - 1) / d); *s = 32 + l; }
}

View lbm_sim::view() const {
  View v;
  v.nx = nx; v.ny = ny; v.nz = nz; v.nxp = nxp; v.np = np;
  v.xshift = xshift; v.bc = bc;
  v.omega = 1.0 / tau; v.rho0 = rho0; v.qcut = qcut;
  for (int a = 0; a < 3; ++a) v.F[a] = F[a];
  v.has_force = has_force; v.has_uw = has_uw;
  v.trt = collision == LBM_COLL_TRT ? 1 : 0;
  v.wall_neq = wall_neq == LBM_NEQ_REGULARIZED ? 1 : 0;
  // Eq. magic-parameter with omega+ = 1/tau, solved for omega-
  v.omega_m = v.trt ? 1.0 / (0.5 + magic / (tau - 0.5)) : v.omega;
  v.omega_f = (float)v.omega; v.rho0_f = (float)rho0; v.qcut_f = (float)qcut;
  v.omega_m_f = (float)v.omega_m;
  for (int a = 0; a < 3; ++a) v.F_f[a] = (float)F[a];
  const double unit = dtype == LBM_F16 ? (double)kF16Scale : 1.0;  // stored units (lattice.cuh, Units)
  v.rho0_u = (float)(rho0 * unit);
  for (int a = 0; a < 3; ++a) v.F_u[a] = (float)(F[a] * unit);
  v.flags = flags; v.amask = amask; v.cbase = cbase; v.rec = rec; v.rnode = rnode; v.nb = nb;
  v.err = err_dev;
  v.wait_limit = wait_limit;
  v.dbg = dbg_dev;
  v.dbg_limit = dbg_limit >= 0 ? dbg_limit : (long long)Q * np;
  v.tiles = tiles; v.gx = nxp / (step_bx * npt());
  invariant_divisor(v.gx, &v.gx_m, &v.gx_s);
  invariant_divisor(nxp, &v.nxp_m, &v.nxp_s);
  invariant_divisor((long long)nxp * ny, &v.pl_m, &v.pl_s);
  for (int i = 0; i < Q; ++i) {
    int c[3];
    lattice_c(i, c[0], c[1], c[2]);
    v.soff[i] = (int)((long long)i * np);
    v.loff[i] = (int)((long long)i * np - (c[0] + (long long)c[1] * nxp + (long long)c[2] * nxp * ny));
  }
  v.ntiles = (int)ntiles; v.tpb_tiles = tiles_per_block;
  v.btiles = btiles;
  if (mb.on) {
    v.dyn = RecSet{mb.rec[cur], mb.rnode[cur], mb.lq[cur], mb.luw[cur], mb.luw1[cur], mb.ltag[cur]};
    v.dyn_count = mb.count[cur];
  } else {
    v.dyn = RecSet{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    v.dyn_count = nullptr;
  }
  v.lq = lq; v.luw = luw; v.luw1 = luw1; v.ltag = ltag;
  return v;
}

// Launch shape: bx (multiple of 32 dividing nxp) by by rows.
Launch lbm_sim::shape(int bx, int by) const {
  Launch l;
  l.block = dim3(bx, by, 1);
  l.grid = dim3(nxp / bx, (ny + by - 1) / by, nz);
  l.stream = stream;
  return l;
}

void lbm_sim::tune_default() {
  // widest power-of-two multiple of 32 (<= 128) that divides the padded row
  int bx = 32;
  while (bx < 128 && nxp % (bx * 2) == 0) bx *= 2;
  step_bx = bx;
  const int threads = (dtype == LBM_F64 && lattice == LBM_D3Q27) ? 128 : 256;  // shared staging
  step_by = std::max(1, threads / bx);
}

Launch lbm_sim::step_shape() const {
  Launch l;
  l.block = dim3(step_bx, step_by, 1);
  l.grid = dim3((unsigned)((ntiles + tiles_per_block - 1) / tiles_per_block), 1, 1);
  l.stream = stream;
  if (variant == 4) {
    l.grid = dim3((unsigned)tma_blocks, 1, 1);
    l.smem = tma_smem;
  }
  return l;
}

// Tile table of the step kernel for the current geometry and launch shape: for
// each plane z, its lattice tiles {z, t} (t = tile in the plane), then its
// boundary tiles {-1 - count, first record}. The split step keeps the boundary
// tiles in a table of their own (btiles), in the same order.
int lbm_sim::ensure_tiles() {
  if (tiles && tiles_bx == step_bx && tiles_by == step_by && tiles_var == variant) return LBM_OK;
  const int tpb = step_bx * step_by;
  const int gx = nxp / (step_bx * npt()), gy = (ny + step_by - 1) / step_by;
  std::vector<uint32_t> hc(np / 32 + 1, 0u);
  if (nb > 0)
    LBM_CUDA(this, cudaMemcpyAsync(hc.data(), cbase, hc.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
  LBM_CUDA(this, cudaStreamSynchronize(stream));
  std::vector<int2> t, bt;
  std::vector<int2> &bdst = split() ? bt : t;
  t.reserve((size_t)nz * gx * gy + nb / tpb + nz + 1);
  const long long pchunks = (long long)nxp * ny / 32;
  for (int z = 0; z < nz; ++z) {
    for (int k = 0; k < gx * gy; ++k) t.push_back(make_int2(z, k));
    if (nb == 0) continue;
    const long long r0 = hc[z * pchunks], r1 = hc[(z + 1) * pchunks];
    for (long long r = r0; r < r1; r += tpb)
      bdst.push_back(make_int2(-1 - (int)std::min<long long>(tpb, r1 - r), (int)r));
  }
  if (mb.on)  // the moving body's records: as many tiles as the region could need
    for (long long r = 0; r < mb.cap_rec; r += tpb) bdst.push_back(make_int2(DYN_TILE, (int)r));
  cudaFree(tiles);
  tiles = nullptr;
  cudaFree(btiles);
  btiles = nullptr;
  ntiles = (long long)t.size();
  nbtiles = (long long)bt.size();
  LBM_CUDA(this, cudaMalloc(&tiles, ntiles * sizeof(int2)));
  LBM_CUDA(this, cudaMemcpyAsync(tiles, t.data(), ntiles * sizeof(int2), cudaMemcpyHostToDevice, stream));
  if (nbtiles > 0) {
    LBM_CUDA(this, cudaMalloc(&btiles, nbtiles * sizeof(int2)));
    LBM_CUDA(this, cudaMemcpyAsync(btiles, bt.data(), nbtiles * sizeof(int2), cudaMemcpyHostToDevice, stream));
    if (!aux) {  // highest priority: the boundary blocks start as soon as the step does
      int lo = 0, hi = 0;
      LBM_CUDA(this, cudaDeviceGetStreamPriorityRange(&lo, &hi));
      LBM_CUDA(this, cudaStreamCreateWithPriority(&aux, cudaStreamNonBlocking, hi));
      LBM_CUDA(this, cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
      LBM_CUDA(this, cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
    }
  }
  LBM_CUDA(this, cudaStreamSynchronize(stream));
  tiles_bx = step_bx;
  tiles_by = step_by;
  tiles_var = variant;
  if (variant == 4) {
    const int phys = (has_force ? PH_FORCE : 0) | (collision == LBM_COLL_TRT ? PH_TRT : 0);
    cudaError_t e = prepare_step_tma(lattice, dtype, phys, step_bx, step_by, ntiles, &tma_blocks, &tma_smem);
    if (e != cudaSuccess) {
      tiles_bx = 0;
      return lbm_fail(this, LBM_ERR_CUDA, std::string("TMA-staged step: ") + cudaGetErrorString(e));
    }
  }
  return LBM_OK;
}
Launch lbm_sim::aux_shape() const { return shape(32, 8); }

// ---------------------------------------------------------------- scratch
int lbm_sim::ensure_scratch(long long doubles) {
  if (doubles <= scratch_len) return LBM_OK;
  cudaFree(scratch);
  scratch = nullptr;
  scratch_len = 0;
  LBM_CUDA(this, cudaMalloc(&scratch, doubles * sizeof(double)));
  scratch_len = doubles;
  return LBM_OK;
}

// ---------------------------------------------------------------- state
extern "C" int lbm_init(lbm_handle h, double rho, const double u[3]) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  if (!h->geom_ok) return lbm_fail(h, LBM_ERR_STATE, "set the geometry first");
  if (!(rho > 0.0)) return lbm_fail(h, LBM_ERR_ARG, "rho must be positive");
  double ux = u ? u[0] : 0.0, uy = u ? u[1] : 0.0, uz = (u && h->lattice != LBM_D2Q9) ? u[2] : 0.0;
  LBM_CUDA(h, launch_init(h->lattice, h->dtype, h->view(), h->f[h->cur], rho, ux, uy, uz, h->aux_shape()));
  h->state_ok = true;
  return LBM_OK;
}

// Both calls stage the FP64 host layout in a device buffer that the handle
// allocates on first use and keeps, so that repeated transfers never reach the
// allocator.
extern "C" int lbm_set_populations(lbm_handle h, const double *f) {
  if (!h || !f) return lbm_fail(h, LBM_ERR_ARG, "null argument");
  if (!h->geom_ok) return lbm_fail(h, LBM_ERR_STATE, "set the geometry first");
  int rc = h->ensure_stage_f();
  if (rc) return rc;
  const size_t bytes = (size_t)h->N * h->Q * sizeof(double);
  cudaError_t e = cudaMemcpyAsync(h->stage_f, f, bytes, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = launch_set_pop(h->lattice, h->dtype, h->view(), h->f[h->cur], h->stage_f, h->aux_shape());
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return lbm_fail(h, LBM_ERR_CUDA, cudaGetErrorString(e));
  h->state_ok = true;
  return LBM_OK;
}

extern "C" int lbm_get_populations(lbm_handle h, double *f) {
  if (!h || !f) return lbm_fail(h, LBM_ERR_ARG, "null argument");
  if (!h->geom_ok) return lbm_fail(h, LBM_ERR_STATE, "set the geometry first");
  int rc = h->ensure_stage_f();
  if (rc) return rc;
  const size_t bytes = (size_t)h->N * h->Q * sizeof(double);
  cudaError_t e = launch_read(h->lattice, h->dtype, h->view(), h->f[h->cur], h->stage_f, nullptr, nullptr,
                              nullptr, h->aux_shape());
  if (e == cudaSuccess) e = cudaMemcpyAsync(f, h->stage_f, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return lbm_fail(h, LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}

extern "C" int lbm_macros(lbm_handle h, double *rho, double *u) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  if (!h->geom_ok || !h->state_ok) return lbm_fail(h, LBM_ERR_STATE, "no state yet");
  LBM_CUDA(h, launch_read(h->lattice, h->dtype, h->view(), h->f[h->cur], nullptr, rho, u, nullptr,
                          h->aux_shape()));
  return LBM_OK;
}

extern "C" int lbm_mass(lbm_handle h, double *m) {
  if (!h || !m) return lbm_fail(h, LBM_ERR_ARG, "null argument");
  if (!h->geom_ok || !h->state_ok) return lbm_fail(h, LBM_ERR_STATE, "no state yet");
  Launch l = h->aux_shape();
  const long long nblk = (long long)l.grid.x * l.grid.y * l.grid.z;
  int rc = h->ensure_scratch(nblk);
  if (rc) return rc;
  LBM_CUDA(h, launch_read(h->lattice, h->dtype, h->view(), h->f[h->cur], nullptr, nullptr, nullptr,
                          h->scratch, l));
  LBM_CUDA(h, launch_reduce_final(h->scratch, nblk, 1, h->dres, h->stream));
  LBM_CUDA(h, cudaMemcpyAsync(m, h->dres, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  if (!std::isfinite(*m)) return lbm_fail(h, LBM_ERR_NONFINITE, "mass is not finite");
  return LBM_OK;
}

extern "C" int lbm_wall_force(lbm_handle h, int tag, double F[3]) {
  if (!h || !F) return lbm_fail(h, LBM_ERR_ARG, "null argument");
  if (!h->geom_ok || !h->state_ok) return lbm_fail(h, LBM_ERR_STATE, "no state yet");
  if (tag < -1 || tag > 7) return lbm_fail(h, LBM_ERR_ARG, "tag must be -1..7");
  F[0] = F[1] = F[2] = 0.0;
  const int bs = 256;
  const long long nblk1 = (h->nb + bs - 1) / bs;
  const long long nblk2 = h->mb.on ? h->mb.nfpart : 0;
  if (nblk1 + nblk2 == 0) return LBM_OK;
  int rc = h->ensure_scratch((nblk1 + nblk2) * 3);
  if (rc) return rc;
  Launch l;
  l.block = dim3(bs);
  l.stream = h->stream;
  const View v = h->view();
  if (nblk1) {
    l.grid = dim3((unsigned)nblk1);
    LBM_CUDA(h, launch_force(h->lattice, h->dtype, v, h->f[h->cur], h->f[h->cur ^ 1], v.stat(), h->nb,
                             nullptr, tag, h->scratch, l));
  }
  if (nblk2) {
    // the moving body's partials, taken during the last step before its refill
    if (tag < 0 || tag == h->mb.tag)
      LBM_CUDA(h, cudaMemcpyAsync(h->scratch + nblk1 * 3, h->mb.fpart, nblk2 * 3 * sizeof(double),
                                  cudaMemcpyDeviceToDevice, h->stream));
    else
      LBM_CUDA(h, cudaMemsetAsync(h->scratch + nblk1 * 3, 0, nblk2 * 3 * sizeof(double), h->stream));
  }
  LBM_CUDA(h, launch_reduce_final(h->scratch, nblk1 + nblk2, 3, h->dres, h->stream));
  LBM_CUDA(h, cudaMemcpyAsync(F, h->dres, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

extern "C" int lbm_wall_torque(lbm_handle h, int tag, const double centre[3], double T[3]) {
  if (!h || !T || !centre) return lbm_fail(h, LBM_ERR_ARG, "null argument");
  if (!h->geom_ok || !h->state_ok) return lbm_fail(h, LBM_ERR_STATE, "no state yet");
  if (tag < -1 || tag > 7) return lbm_fail(h, LBM_ERR_ARG, "tag must be -1..7");
  T[0] = T[1] = T[2] = 0.0;
  const int bs = 256;
  const long long nblk = (h->nb + bs - 1) / bs;
  if (nblk == 0) return LBM_OK;
  int rc = h->ensure_scratch(nblk * 6);
  if (rc) return rc;
  Launch l;
  l.block = dim3(bs);
  l.grid = dim3((unsigned)nblk);
  l.stream = h->stream;
  const View v = h->view();
  LBM_CUDA(h, launch_force(h->lattice, h->dtype, v, h->f[h->cur], h->f[h->cur ^ 1], v.stat(), h->nb, nullptr, tag,
                           h->scratch, l, h->scratch + nblk * 3, centre[0], centre[1], centre[2]));
  LBM_CUDA(h, launch_reduce_final(h->scratch + nblk * 3, nblk, 3, h->dres, h->stream));
  LBM_CUDA(h, cudaMemcpyAsync(T, h->dres, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

extern "C" int lbm_get_counts(lbm_handle h, int64_t *n_fluid, int64_t *n_boundary, int64_t *n_links) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  if (n_fluid) *n_fluid = h->nfluid;
  if (n_boundary) *n_boundary = h->nb;
  if (n_links) *n_links = h->nl;
  return LBM_OK;
}

// ---------------------------------------------------------------- stepping
int lbm_sim::launch_steps(int n) {
  if (n > 0) {
    int rc = ensure_tiles();
    if (rc) return rc;
  }
  for (int k = 0; k < n; ++k) {
    cudaError_t e;
    if (split() && nbtiles > 0) {
      // the boundary kernel forks onto aux and joins before anything after the step
      Launch lb;
      lb.grid = dim3((unsigned)nbtiles, 1, 1);
      lb.block = dim3(step_bx, step_by, 1);
      lb.stream = aux;
      e = cudaEventRecord(ev_fork, stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev_fork, 0);
      if (e == cudaSuccess) e = launch_step(lattice, dtype, variant, view(), f[cur], f[cur ^ 1], step_shape(), &lb);
      if (e == cudaSuccess) e = cudaEventRecord(ev_join, aux);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev_join, 0);
    } else {
      e = launch_step(lattice, dtype, variant, view(), f[cur], f[cur ^ 1], step_shape());
    }
    if (e != cudaSuccess) return lbm_fail(this, LBM_ERR_CUDA, cudaGetErrorString(e));
    if (mb.on) {
      int rc = move_after_step(f[cur ^ 1], cur ^ 1);
      if (rc) return rc;
    }
    cur ^= 1;
  }
  return LBM_OK;
}

int lbm_sim::capture(int parity) {
  // a graph of kGraphSteps (even) steps starting from buffer `parity`
  const int save = cur;
  cur = parity;
  cudaGraph_t g = nullptr;
  LBM_CUDA(this, cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
  int rc = launch_steps(kGraphSteps);
  cudaError_t e = cudaStreamEndCapture(stream, &g);
  cur = save;
  if (rc) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) return lbm_fail(this, LBM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&graph[parity], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { graph[parity] = nullptr; return lbm_fail(this, LBM_ERR_CUDA, cudaGetErrorString(e)); }
  return LBM_OK;
}

extern "C" int lbm_step(lbm_handle h, int n) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  if (n < 0) return lbm_fail(h, LBM_ERR_ARG, "negative step count");
  if (!h->geom_ok || !h->state_ok) return lbm_fail(h, LBM_ERR_STATE, "set geometry and state first");
  int reps = n / lbm_sim::kGraphSteps;
  int rest = n % lbm_sim::kGraphSteps;
  if (n > 0) {
    int rc = h->ensure_tiles();  // never inside a capture
    if (rc) return rc;
  }
  if (reps > 0) {
    if (!h->graph[h->cur]) {
      int rc = h->capture(h->cur);
      if (rc) return rc;
    }
    for (int k = 0; k < reps; ++k) LBM_CUDA(h, cudaGraphLaunch(h->graph[h->cur], h->stream));
  }
  return h->launch_steps(rest);
}

// ---------------------------------------------------------------- explicit geometry
extern "C" int lbm_set_geometry(lbm_handle h, const uint8_t *flags, const double *q, const double *uw,
                                const double *uw1, const int32_t *tag) {
  if (!h || !flags) return lbm_fail(h, LBM_ERR_ARG, "null argument");
  HostGeometry g;
  std::string msg;
  int rc = build_records_host(*h, flags, q, uw, uw1, tag, g, msg);
  if (rc) return lbm_fail(h, rc, msg);
  return h->upload(g);
}

int lbm_sim::upload(const HostGeometry &g) {
  ++version;
  free_moving_body();
  drop_graphs();
  free_geometry();
  tiles_bx = tiles_by = 0;
  geom_ok = false;
  LBM_CUDA(this, cudaMemcpyAsync(flags, g.flags.data(), np, cudaMemcpyHostToDevice, stream));
  LBM_CUDA(this, cudaMemcpyAsync(cbase, g.cbase.data(), g.cbase.size() * sizeof(uint32_t),
                                 cudaMemcpyHostToDevice, stream));
  nb = (long long)g.rec.size();
  nl = (long long)g.ltag.size();
  nfluid = g.nfluid;
  has_uw = g.has_uw;
  has_shell = 0;
  if (nb > 0) {
    LBM_CUDA(this, cudaMalloc(&rec, nb * sizeof(Rec)));
    LBM_CUDA(this, cudaMalloc(&rnode, nb * sizeof(uint32_t)));
    LBM_CUDA(this, cudaMemcpyAsync(rec, g.rec.data(), nb * sizeof(Rec), cudaMemcpyHostToDevice, stream));
    LBM_CUDA(this, cudaMemcpyAsync(rnode, g.rnode.data(), nb * sizeof(uint32_t), cudaMemcpyHostToDevice, stream));
  }
  if (nl > 0) {
    const size_t ls = link_size();
    LBM_CUDA(this, cudaMalloc(&lq, nl * ls));
    LBM_CUDA(this, cudaMalloc(&ltag, nl));
    LBM_CUDA(this, cudaMemcpyAsync(lq, g.lq.data(), nl * ls, cudaMemcpyHostToDevice, stream));
    LBM_CUDA(this, cudaMemcpyAsync(ltag, g.ltag.data(), nl, cudaMemcpyHostToDevice, stream));
    if (has_uw) {
      LBM_CUDA(this, cudaMalloc(&luw, nl * 3 * ls));
      LBM_CUDA(this, cudaMalloc(&luw1, nl * 3 * ls));
      LBM_CUDA(this, cudaMemcpyAsync(luw, g.luw.data(), nl * 3 * ls, cudaMemcpyHostToDevice, stream));
      LBM_CUDA(this, cudaMemcpyAsync(luw1, g.luw1.data(), nl * 3 * ls, cudaMemcpyHostToDevice, stream));
    }
  }
  LBM_CUDA(this, cudaStreamSynchronize(stream));
  int rc = finish_geometry();
  if (rc) return rc;
  geom_ok = true;
  return LBM_OK;
}

extern "C" int lbm_get_geometry(lbm_handle h, uint8_t *flags, double *q, double *uw, double *uw1,
                                int32_t *tag) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  if (!h->geom_ok) return lbm_fail(h, LBM_ERR_STATE, "no geometry yet");
  HostGeometry g;
  int rc = h->download(g);
  if (rc) return rc;
  unpack_geometry(*h, g, flags, q, uw, uw1, tag);
  return LBM_OK;
}

int lbm_sim::download(HostGeometry &g) {
  g.flags.resize(np);
  g.cbase.resize(np / 32 + 1);
  g.rec.resize(nb);
  g.rnode.resize(nb);
  const size_t ls = link_size();
  g.lq.resize(nl * ls);
  g.ltag.resize(nl);
  g.has_uw = has_uw;
  g.nfluid = nfluid;
  LBM_CUDA(this, cudaMemcpyAsync(g.flags.data(), flags, np, cudaMemcpyDeviceToHost, stream));
  if (nb) {
    LBM_CUDA(this, cudaMemcpyAsync(g.rec.data(), rec, nb * sizeof(Rec), cudaMemcpyDeviceToHost, stream));
    LBM_CUDA(this, cudaMemcpyAsync(g.rnode.data(), rnode, nb * sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
  }
  if (nl) {
    LBM_CUDA(this, cudaMemcpyAsync(g.lq.data(), lq, nl * ls, cudaMemcpyDeviceToHost, stream));
    LBM_CUDA(this, cudaMemcpyAsync(g.ltag.data(), ltag, nl, cudaMemcpyDeviceToHost, stream));
    if (has_uw) {
      g.luw.resize(nl * 3 * ls);
      g.luw1.resize(nl * 3 * ls);
      LBM_CUDA(this, cudaMemcpyAsync(g.luw.data(), luw, nl * 3 * ls, cudaMemcpyDeviceToHost, stream));
      LBM_CUDA(this, cudaMemcpyAsync(g.luw1.data(), luw1, nl * 3 * ls, cudaMemcpyDeviceToHost, stream));
    }
  }
  LBM_CUDA(this, cudaStreamSynchronize(stream));
  return LBM_OK;
}

// ---------------------------------------------------------------- launch configuration
static bool valid_launch(const lbm_sim *h, int bx, int by, int variant, int tiles) {
  if (bx < 32 || bx % 32 || h->nxp % bx || by < 1 || bx * by > 256) return false;
  if (variant < 0 || variant > 12 || tiles < 1 || tiles > 4) return false;
  if (variant == 8 && bx * by != 128) return false;  // compiled for blocks of 128 threads
  if (h->dtype == LBM_F64 && variant != 0) return false;
  if (h->dtype == LBM_F64 && h->lattice == LBM_D3Q27 && bx * by > 128) return false;  // shared staging
  if (variant >= 5 && variant <= 8 && (h->nxp % (2 * bx) || h->bc == LBM_BC_BFL))
    return false;  // pairs: whole rows, no BFL
  return true;
}

extern "C" int lbm_set_launch(lbm_handle h, int bx, int by, int variant, int tiles) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  if (!valid_launch(h, bx, by, variant, tiles)) return lbm_fail(h, LBM_ERR_ARG, "invalid launch configuration");
  h->step_bx = bx;
  h->step_by = by;
  h->variant = variant;
  h->tiles_per_block = tiles;
  h->drop_graphs();
  return LBM_OK;
}

extern "C" int lbm_get_launch(lbm_handle h, int *bx, int *by, int *variant, int *tiles) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  if (bx) *bx = h->step_bx;
  if (by) *by = h->step_by;
  if (variant) *variant = h->variant;
  if (tiles) *tiles = h->tiles_per_block;
  return LBM_OK;
}

extern "C" int lbm_autotune(lbm_handle h, int steps, int *bx, int *by, int *variant, int *tiles,
                            double *ms_per_step) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  if (steps < 1) return lbm_fail(h, LBM_ERR_ARG, "steps must be positive");
  if (!h->geom_ok || !h->state_ok) return lbm_fail(h, LBM_ERR_STATE, "set geometry and state first");
  cudaEvent_t e0, e1;
  LBM_CUDA(h, cudaEventCreate(&e0));
  LBM_CUDA(h, cudaEventCreate(&e1));
  const int save[4] = {h->step_bx, h->step_by, h->variant, h->tiles_per_block};
  int best[4] = {save[0], save[1], save[2], save[3]};
  float best_ms = 1e30f;
  int rc = LBM_OK;
  const int nvar = h->dtype == LBM_F64 ? 1 : 13;  // 4: TMA; 5-8: node pairs; 9-10: split; 11-12: 5, 6 blocks
  const int tile_opts[3] = {1, 2, 4};
  for (int threads = 128; threads <= 256 && rc == LBM_OK; threads *= 2)
    for (int bxx = 32; bxx <= threads && rc == LBM_OK; bxx *= 2) {
      if (h->nxp % bxx) continue;
      for (int var = 0; var < nvar && rc == LBM_OK; ++var)
        for (int k = 0; k < 3 && rc == LBM_OK; ++k) {
          if (var == 4 && k > 0) continue;  // the persistent kernel ignores tiles per block
          if (!valid_launch(h, bxx, threads / bxx, var, tile_opts[k])) continue;
          h->step_bx = bxx;
          h->step_by = threads / bxx;
          h->variant = var;
          h->tiles_per_block = tile_opts[k];
          rc = h->launch_steps(2);  // warm (and build the tile table)
          if (rc) break;
          cudaEventRecord(e0, h->stream);
          rc = h->launch_steps(steps);
          cudaEventRecord(e1, h->stream);
          if (rc) break;
          cudaError_t e = cudaEventSynchronize(e1);
          if (e != cudaSuccess) { rc = lbm_fail(h, LBM_ERR_CUDA, cudaGetErrorString(e)); break; }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best_ms) { best_ms = ms; best[0] = bxx; best[1] = threads / bxx; best[2] = var; best[3] = tile_opts[k]; }
        }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    h->step_bx = save[0]; h->step_by = save[1]; h->variant = save[2]; h->tiles_per_block = save[3];
    return rc;
  }
  h->step_bx = best[0];
  h->step_by = best[1];
  h->variant = best[2];
  h->tiles_per_block = best[3];
  h->drop_graphs();
  if (bx) *bx = best[0];
  if (by) *by = best[1];
  if (variant) *variant = best[2];
  if (tiles) *tiles = best[3];
  if (ms_per_step) *ms_per_step = best_ms / steps;
  return LBM_OK;
}

// ---------------------------------------------------------------- save / load
// A saved state is a header followed by the raw contents of the current
// population buffer, byte for byte as the kernels keep them (the values written
// ahead for the next step included), so that a resumed run continues bit for bit.
namespace {
struct SaveHeader {
  char magic[8];  // "LBMSTATE"
  uint32_t version;
  int32_t lattice, dtype, nx, ny, nz, bc, has_body;
  double rho0;
  uint64_t geom_hash, body_hash;
  int64_t pose;  // the moving body's pose index, -1 without a body
  double body_state[6];  // free body: angle, omega, centre, inertia
  uint64_t pop_bytes;
};
constexpr uint32_t kSaveVersion = 1;
}  // namespace

extern "C" int lbm_save(lbm_handle h, void *buf, size_t *bytes) {
  if (!h || !bytes) return lbm_fail(h, LBM_ERR_ARG, "null argument");
  if (!h->geom_ok || !h->state_ok) return lbm_fail(h, LBM_ERR_STATE, "no state yet");
  SaveHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "LBMSTATE", 8);
  hd.version = kSaveVersion;
  hd.lattice = h->lattice; hd.dtype = h->dtype; hd.nx = h->nx; hd.ny = h->ny; hd.nz = h->nz; hd.bc = h->bc;
  hd.has_body = h->mb.on ? 1 : 0;
  hd.rho0 = h->rho0;
  hd.geom_hash = h->geom_hash;
  hd.body_hash = h->mb.on ? h->mb.hash : 0;
  hd.pose = -1;
  hd.pop_bytes = (uint64_t)h->Q * h->np * h->elem_size();
  const size_t total = sizeof(SaveHeader) + hd.pop_bytes;
  if (!buf) { *bytes = total; return LBM_OK; }
  if (*bytes < total)
    return lbm_fail(h, LBM_ERR_ARG, "buffer too small for the saved state: " + std::to_string(total) + " bytes needed");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->mb.on) {
    int k = 0;
    LBM_CUDA(h, cudaMemcpy(&k, h->mb.step, sizeof(int), cudaMemcpyDeviceToHost));
    hd.pose = k;
    if (h->mb.free_rot) LBM_CUDA(h, cudaMemcpy(hd.body_state, h->mb.state, sizeof(hd.body_state), cudaMemcpyDeviceToHost));
  }
  unsigned char *p = static_cast<unsigned char *>(buf);
  std::memcpy(p, &hd, sizeof(hd));
  LBM_CUDA(h, cudaMemcpyAsync(p + sizeof(hd), h->f[h->cur], hd.pop_bytes, cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  *bytes = total;
  return LBM_OK;
}

extern "C" int lbm_load(lbm_handle h, const void *buf, size_t bytes) {
  if (!h || !buf) return lbm_fail(h, LBM_ERR_ARG, "null argument");
  if (!h->geom_ok) return lbm_fail(h, LBM_ERR_STATE, "set the same geometry first");
  SaveHeader hd;
  if (bytes < sizeof(hd)) return lbm_fail(h, LBM_ERR_ARG, "not a saved state: too short");
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, "LBMSTATE", 8) != 0 || hd.version != kSaveVersion)
    return lbm_fail(h, LBM_ERR_ARG, "not a saved state of this library version");
  if (hd.lattice != h->lattice || hd.dtype != h->dtype || hd.nx != h->nx || hd.ny != h->ny || hd.nz != h->nz)
    return lbm_fail(h, LBM_ERR_ARG, "the saved state has another lattice, storage type or size");
  if (hd.bc != h->bc || hd.rho0 != h->rho0)
    return lbm_fail(h, LBM_ERR_ARG, "the saved state has another boundary rule or reference density");
  if (hd.geom_hash != h->geom_hash) return lbm_fail(h, LBM_ERR_ARG, "the saved state has another geometry");
  if ((hd.has_body != 0) != h->mb.on || (h->mb.on && hd.body_hash != h->mb.hash))
    return lbm_fail(h, LBM_ERR_ARG, "the saved state has another moving body");
  const uint64_t pop = (uint64_t)h->Q * h->np * h->elem_size();
  if (hd.pop_bytes != pop || bytes < sizeof(hd) + pop) return lbm_fail(h, LBM_ERR_ARG, "the saved state is truncated");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  const unsigned char *p = static_cast<const unsigned char *>(buf);
  LBM_CUDA(h, cudaMemcpyAsync(h->f[h->cur], p + sizeof(hd), pop, cudaMemcpyHostToDevice, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->mb.on) {
    if (h->mb.free_rot)
      LBM_CUDA(h, cudaMemcpy(h->mb.state, hd.body_state, sizeof(hd.body_state), cudaMemcpyHostToDevice));
    int rc = h->move_rebuild(hd.pose);
    if (rc) return rc;
  }
  h->state_ok = true;
  return LBM_OK;
}

extern "C" int lbm_is_debug_build(void) {
#ifdef LBM_DEBUG
  return 1;
#else
  return 0;
#endif
}

extern "C" int lbm_set_debug_limit(lbm_handle h, long long elements) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
#ifdef LBM_DEBUG
  h->dbg_limit = elements < 0 ? -1 : elements;
  h->drop_graphs();
  return LBM_OK;
#else
  (void)elements;
  return lbm_fail(h, LBM_ERR_STATE, "not a debug build (compile with LBM_DEBUG)");
#endif
}

extern "C" int lbm_set_wait_limit(lbm_handle h, long long polls) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  h->wait_limit = polls < 0 ? (1LL << 24) : polls;
  h->drop_graphs();
  return LBM_OK;
}
