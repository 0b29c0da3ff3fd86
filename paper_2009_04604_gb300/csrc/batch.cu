// batch.cu -- batched stepping of many independent simulations (lbm_batch_*).
//
// One launch per step and physics class (body force on or off, BGK or TRT; a
// batch of like simulations has one class) advances every simulation of the
// batch. Its blocks run the tiles of the class's simulations, one simulation
// after another, each one's table plane-interleaved as in the single-simulation
// step. The steps replay from captured CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "lbm.h"
#include "sim.hpp"

using namespace lbm;

struct lbm_batch_s {
  std::vector<lbm_sim *> sims;
  std::vector<int> base_cur;  // each simulation's buffer index when the entries were built
  std::vector<int> base_ver;  // each simulation's version when the entries were built
  int lattice = 0, dtype = 1;
  cudaStream_t stream = nullptr;
  BatchEntry *entries = nullptr;
  int4 *tiles = nullptr;
  long long ntiles = 0;
  long long cls_first[4] = {0, 0, 0, 0}, cls_count[4] = {0, 0, 0, 0};  // tile range per physics class
  int bx = 32, by = 4, variant = 3, T = 1;
  bool tiles_ok = false;
  int parity = 0;  // batch steps taken since the entries were built, mod 2
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  std::string err;
};

static constexpr int kBatchGraphSteps = 32;

static int bfail(lbm_batch b, int code, const std::string &msg) {
  if (b) b->err = msg;
  return code;
}

#define B_CUDA(b, call)                                                                          \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return bfail((b), e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,           \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                          \
  } while (0)

template <class L, typename S, typename M, int MINB, int PHYS>
static cudaError_t batch_class(const lbm_batch_s *b, int parity) {
  const long long n = b->cls_count[PHYS];
  if (n == 0) return cudaSuccess;
  const dim3 block(b->bx, b->by, 1);
  const unsigned grid = (unsigned)((n + b->T - 1) / b->T);
  k_step_batch<L, S, M, MINB, PHYS><<<grid, block, 0, b->stream>>>(b->entries, b->tiles + b->cls_first[PHYS],
                                                                    (int)n, b->T, parity);
  return cudaGetLastError();
}

template <class L, typename S, typename M, int MINB>
static cudaError_t batch_variant(const lbm_batch_s *b, int parity) {
  cudaError_t e = batch_class<L, S, M, MINB, 0>(b, parity);
  if (e == cudaSuccess) e = batch_class<L, S, M, MINB, PH_FORCE>(b, parity);
  if (e == cudaSuccess) e = batch_class<L, S, M, MINB, PH_TRT>(b, parity);
  if (e == cudaSuccess) e = batch_class<L, S, M, MINB, PH_FORCE | PH_TRT>(b, parity);
  return e;
}

template <class L, typename S, typename M>
static cudaError_t batch_launch_t(const lbm_batch_s *b, int parity) {
  if constexpr (sizeof(M) == 8) {
    return batch_variant<L, S, M, 1>(b, parity);
  } else {
    switch (b->variant) {
      case 1: return batch_variant<L, S, M, 2>(b, parity);
      case 2: return batch_variant<L, S, M, 3>(b, parity);
      case 3: return batch_variant<L, S, M, 4>(b, parity);
      default: return batch_variant<L, S, M, 1>(b, parity);
    }
  }
}

static cudaError_t batch_launch(const lbm_batch_s *b, int parity) {
  if (b->lattice == LBM_D2Q9) {
    switch (b->dtype) {
      case LBM_F64: return batch_launch_t<D2Q9, double, double>(b, parity);
      case LBM_F32: return batch_launch_t<D2Q9, float, float>(b, parity);
      case LBM_F16: return batch_launch_t<D2Q9, __half, float>(b, parity);
      default: return batch_launch_t<D2Q9, __nv_bfloat16, float>(b, parity);
    }
  }
  if (b->lattice == LBM_D3Q27) {
    switch (b->dtype) {
      case LBM_F64: return batch_launch_t<D3Q27, double, double>(b, parity);
      case LBM_F32: return batch_launch_t<D3Q27, float, float>(b, parity);
      case LBM_F16: return batch_launch_t<D3Q27, __half, float>(b, parity);
      default: return batch_launch_t<D3Q27, __nv_bfloat16, float>(b, parity);
    }
  }
  switch (b->dtype) {
    case LBM_F64: return batch_launch_t<D3Q19, double, double>(b, parity);
    case LBM_F32: return batch_launch_t<D3Q19, float, float>(b, parity);
    case LBM_F16: return batch_launch_t<D3Q19, __half, float>(b, parity);
    default: return batch_launch_t<D3Q19, __nv_bfloat16, float>(b, parity);
  }
}

static void drop_batch_graphs(lbm_batch b) {
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) { cudaGraphExecDestroy(b->graph[k]); b->graph[k] = nullptr; }
}

// Entries (views and buffers at the current buffer index of each simulation) and
// the tile table for the batch's launch shape.
static int build_batch(lbm_batch b) {
  const int n = (int)b->sims.size();
  std::vector<BatchEntry> e(n);
  std::vector<int4> t;
  b->base_cur.resize(n);
  b->base_ver.resize(n);
  const int tpb = b->bx * b->by;
  // simulations by physics class, in batch order within a class
  std::vector<int> order;
  for (int c = 0; c < 4; ++c)
    for (int k = 0; k < n; ++k) {
      const lbm_sim *s = b->sims[k];
      if (((s->has_force ? PH_FORCE : 0) | (s->collision == LBM_COLL_TRT ? PH_TRT : 0)) == c) order.push_back(k);
    }
  for (int c = 0; c < 4; ++c) b->cls_count[c] = 0;
  for (int k : order) {
    lbm_sim *s = b->sims[k];
    const int c = (s->has_force ? PH_FORCE : 0) | (s->collision == LBM_COLL_TRT ? PH_TRT : 0);
    if (b->cls_count[c] == 0) b->cls_first[c] = (long long)t.size();
    const size_t t0 = t.size();
    const int save_bx = s->step_bx, save_var = s->variant;
    s->step_bx = b->bx;        // the view's tile-row count follows the batch's block width
    s->variant = b->variant;   // and its one-node lattice tiles (a simulation may be set to node pairs)
    e[k].v = s->view();
    s->step_bx = save_bx;
    s->variant = save_var;
    e[k].v.tiles = nullptr;
    e[k].f0 = s->f[s->cur];
    e[k].f1 = s->f[s->cur ^ 1];
    b->base_cur[k] = s->cur;
    b->base_ver[k] = s->version;
    const int gx = s->nxp / b->bx, gy = (s->ny + b->by - 1) / b->by;
    std::vector<uint32_t> hc(s->np / 32 + 1, 0u);
    if (s->nb > 0) {
      B_CUDA(b, cudaMemcpyAsync(hc.data(), s->cbase, hc.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream));
      B_CUDA(b, cudaStreamSynchronize(b->stream));
    }
    const long long pchunks = (long long)s->nxp * s->ny / 32;
    for (int z = 0; z < s->nz; ++z) {
      for (int i = 0; i < gx * gy; ++i) t.push_back(make_int4(k, z, i, 0));
      if (s->nb == 0) continue;
      const long long r0 = hc[z * pchunks], r1 = hc[(z + 1) * pchunks];
      for (long long r = r0; r < r1; r += tpb)
        t.push_back(make_int4(k, -1, (int)r, (int)std::min<long long>(tpb, r1 - r)));
    }
    b->cls_count[c] += (long long)(t.size() - t0);
  }
  drop_batch_graphs(b);
  cudaFree(b->entries);
  cudaFree(b->tiles);
  b->entries = nullptr;
  b->tiles = nullptr;
  b->ntiles = (long long)t.size();
  if (b->ntiles >= (1LL << 31)) return bfail(b, LBM_ERR_ARG, "batch too large: more than 2^31 tiles");
  B_CUDA(b, cudaMalloc(&b->entries, n * sizeof(BatchEntry)));
  B_CUDA(b, cudaMalloc(&b->tiles, std::max<long long>(1, b->ntiles) * sizeof(int4)));
  B_CUDA(b, cudaMemcpyAsync(b->entries, e.data(), n * sizeof(BatchEntry), cudaMemcpyHostToDevice, b->stream));
  if (b->ntiles)
    B_CUDA(b, cudaMemcpyAsync(b->tiles, t.data(), b->ntiles * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  b->parity = 0;
  b->tiles_ok = true;
  return LBM_OK;
}

// The entries are valid while every simulation is still at its recorded buffer
// index shifted by the batch's own steps, with unchanged options and geometry.
static bool entries_current(const lbm_batch_s *b) {
  if (!b->tiles_ok || b->base_cur.size() != b->sims.size()) return false;
  for (size_t k = 0; k < b->sims.size(); ++k)
    if (b->sims[k]->cur != (b->base_cur[k] ^ b->parity) || b->sims[k]->version != b->base_ver[k] ||
        !b->sims[k]->geom_ok)
      return false;
  return b->tiles_ok;
}

static int batch_direct(lbm_batch b, int n) {
  for (int k = 0; k < n; ++k) {
    cudaError_t e = batch_launch(b, b->parity);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, cudaGetErrorString(e));
    b->parity ^= 1;
    for (lbm_sim *s : b->sims) s->cur ^= 1;
  }
  return LBM_OK;
}

extern "C" int lbm_batch_create(const lbm_handle *sims, int n, lbm_batch *out) {
  if (!out || !sims || n < 1) return LBM_ERR_ARG;
  *out = nullptr;
  lbm_batch b = new lbm_batch_s();
  for (int k = 0; k < n; ++k) {
    lbm_sim *s = sims[k];
    if (!s) { delete b; return LBM_ERR_ARG; }
    if (!s->geom_ok || !s->state_ok) { delete b; return LBM_ERR_STATE; }
    if (s->mb.on) { delete b; return LBM_ERR_ARG; }  // moving bodies step alone
    if (k == 0) {
      b->lattice = s->lattice;
      b->dtype = s->dtype;
      b->stream = s->stream;
    } else if (s->lattice != b->lattice || s->dtype != b->dtype || s->stream != b->stream) {
      delete b;
      return LBM_ERR_ARG;  // one lattice, one storage type and one stream per batch
    }
    for (int j = 0; j < k; ++j)
      if (sims[j] == s) { delete b; return LBM_ERR_ARG; }
    b->sims.push_back(s);
  }
  if (b->dtype == LBM_F64) b->variant = 0;
  *out = b;
  return LBM_OK;
}

extern "C" int lbm_batch_destroy(lbm_batch b) {
  if (!b) return LBM_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_batch_graphs(b);
  cudaFree(b->entries);
  cudaFree(b->tiles);
  delete b;
  return LBM_OK;
}

extern "C" const char *lbm_batch_last_error(lbm_batch b) { return b ? b->err.c_str() : ""; }

extern "C" int lbm_batch_set_launch(lbm_batch b, int bx, int by, int variant, int tiles) {
  if (!b) return LBM_ERR_ARG;
  if (bx < 32 || bx % 32 || by < 1 || bx * by > 256 || variant < 0 || variant > 3 || tiles < 1 || tiles > 4)
    return bfail(b, LBM_ERR_ARG, "invalid launch configuration");
  if (b->dtype == LBM_F64 && variant != 0) return bfail(b, LBM_ERR_ARG, "FP64 takes variant 0 only");
  if (b->dtype == LBM_F64 && b->lattice == LBM_D3Q27 && bx * by > 128)
    return bfail(b, LBM_ERR_ARG, "FP64 on D3Q27 takes at most 128 threads per block (shared staging)");
  for (lbm_sim *s : b->sims)
    if (s->nxp % bx) return bfail(b, LBM_ERR_ARG, "bx must divide the padded row length of every simulation");
  b->bx = bx; b->by = by; b->variant = variant; b->T = tiles;
  b->tiles_ok = false;
  drop_batch_graphs(b);
  return LBM_OK;
}

extern "C" int lbm_batch_step(lbm_batch b, int n) {
  if (!b) return LBM_ERR_ARG;
  if (n < 0) return bfail(b, LBM_ERR_ARG, "negative step count");
  if (n == 0) return LBM_OK;
  for (lbm_sim *s : b->sims) {
    if (!s->geom_ok || !s->state_ok) return bfail(b, LBM_ERR_STATE, "a simulation lost its geometry or state");
    if (s->mb.on) return bfail(b, LBM_ERR_ARG, "a simulation with a moving body cannot be batched");
  }
  if (!entries_current(b)) {
    int rc = build_batch(b);
    if (rc) return rc;
  }
  int reps = n / kBatchGraphSteps, rest = n % kBatchGraphSteps;
  if (reps > 0) {
    const int p = b->parity;
    if (!b->graph[p]) {
      cudaGraph_t g = nullptr;
      B_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      for (int k = 0; k < kBatchGraphSteps; ++k) batch_launch(b, (p + k) & 1);
      cudaError_t e = cudaStreamEndCapture(b->stream, &g);
      if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&b->graph[p], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { b->graph[p] = nullptr; return bfail(b, LBM_ERR_CUDA, cudaGetErrorString(e)); }
    }
    for (int k = 0; k < reps; ++k) B_CUDA(b, cudaGraphLaunch(b->graph[p], b->stream));
    // kBatchGraphSteps is even: parities and buffer indices are unchanged
  }
  return batch_direct(b, rest);
}

extern "C" int lbm_batch_autotune(lbm_batch b, int steps, int *bx, int *by, int *variant, int *tiles,
                                  double *ms_per_step) {
  if (!b || steps < 1) return LBM_ERR_ARG;
  cudaEvent_t e0, e1;
  B_CUDA(b, cudaEventCreate(&e0));
  B_CUDA(b, cudaEventCreate(&e1));
  int best[4] = {b->bx, b->by, b->variant, b->T};
  float best_ms = 1e30f;
  int rc = LBM_OK;
  const int nvar = b->dtype == LBM_F64 ? 1 : 4;
  const int topts[3] = {1, 2, 4};
  const int max_threads = (b->dtype == LBM_F64 && b->lattice == LBM_D3Q27) ? 128 : 256;  // shared staging
  for (int threads = 128; threads <= max_threads && rc == LBM_OK; threads *= 2)
    for (int bxx = 32; bxx <= threads && rc == LBM_OK; bxx *= 2) {
      bool ok = true;
      for (lbm_sim *s : b->sims) ok = ok && (s->nxp % bxx == 0);
      if (!ok) continue;
      for (int var = 0; var < nvar && rc == LBM_OK; ++var)
        for (int k = 0; k < 3 && rc == LBM_OK; ++k) {
          rc = lbm_batch_set_launch(b, bxx, threads / bxx, var, topts[k]);
          if (rc) break;
          rc = build_batch(b);
          if (rc) break;
          rc = batch_direct(b, 2);
          if (rc) break;
          cudaEventRecord(e0, b->stream);
          rc = batch_direct(b, steps);
          cudaEventRecord(e1, b->stream);
          if (rc) break;
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best_ms) { best_ms = ms; best[0] = bxx; best[1] = threads / bxx; best[2] = var; best[3] = topts[k]; }
        }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  rc = lbm_batch_set_launch(b, best[0], best[1], best[2], best[3]);
  if (rc) return rc;
  if (bx) *bx = best[0];
  if (by) *by = best[1];
  if (variant) *variant = best[2];
  if (tiles) *tiles = best[3];
  if (ms_per_step) *ms_per_step = best_ms / steps;
  return LBM_OK;
}
