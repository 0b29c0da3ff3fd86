// geometry.hpp -- boundary records in host memory: build from explicit per-link
// arrays, and unpack back to dense per-link arrays.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "lattice.cuh"

struct lbm_sim;

namespace lbm {

struct HostGeometry {
  std::vector<uint8_t> flags;   // [np] padded node flags
  std::vector<uint32_t> cbase;  // [np/32 + 1]
  std::vector<Rec> rec;         // [nb]
  std::vector<uint32_t> rnode;  // [nb]
  std::vector<uint8_t> lq;      // [nl] q, as the link type (float or double) in raw bytes
  std::vector<uint8_t> luw, luw1;
  std::vector<uint8_t> ltag;    // [nl]
  long long nfluid = 0;
  int has_uw = 0;
};

// flags/q/uw/uw1/tag in the layout of lbm_set_geometry. Returns 0 or an lbm_status.
int build_records_host(const lbm_sim &s, const uint8_t *flags, const double *q, const double *uw,
                       const double *uw1, const int32_t *tag, HostGeometry &g, std::string &msg);

void unpack_geometry(const lbm_sim &s, const HostGeometry &g, uint8_t *flags, double *q, double *uw,
                     double *uw1, int32_t *tag);

// padded index of the node reached from (x, y, z) by (dx, dy, dz), periodic with x-shear
long long host_neighbour(const lbm_sim &s, int x, int y, int z, int dx, int dy, int dz);

}  // namespace lbm
