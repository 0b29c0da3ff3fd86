// geometry_host.cu -- boundary records from explicit host geometry (lbm_set_geometry).
//
// Records are sorted by padded node index. cbase[c] counts the records of the
// nodes before 32-node chunk c. A warp that covers chunk c then finds the
// record of its lane from the ballot of the boundary flag.
#include <cmath>
#include <cstring>

#include "lbm.h"
#include "geometry.hpp"
#include "sim.hpp"

namespace lbm {

long long host_neighbour(const lbm_sim &s, int x, int y, int z, int dx, int dy, int dz) {
  int X = x + dx, Y = y + dy, Z = z + dz;
  if (X >= s.nx) { X -= s.nx; Y -= s.xshift; }
  else if (X < 0) { X += s.nx; Y += s.xshift; }
  Y %= s.ny;
  if (Y < 0) Y += s.ny;
  Z %= s.nz;
  if (Z < 0) Z += s.nz;
  return ((long long)Z * s.ny + Y) * s.nxp + X;
}

template <typename T>
static void push_val(std::vector<uint8_t> &v, double x) {
  T t = (T)x;
  const uint8_t *p = reinterpret_cast<const uint8_t *>(&t);
  v.insert(v.end(), p, p + sizeof(T));
}

template <typename T>
static double get_val(const std::vector<uint8_t> &v, size_t k) {
  T t;
  std::memcpy(&t, v.data() + k * sizeof(T), sizeof(T));
  return (double)t;
}

int build_records_host(const lbm_sim &s, const uint8_t *flags, const double *q, const double *uw,
                       const double *uw1, const int32_t *tag, HostGeometry &g, std::string &msg) {
  const int Q = s.Q;
  const bool dbl = s.link_size() == 8;
  g.flags.assign(s.np, K_PAD);
  g.cbase.assign(s.np / 32 + 1, 0);
  g.rec.clear(); g.rnode.clear(); g.lq.clear(); g.luw.clear(); g.luw1.clear(); g.ltag.clear();
  g.nfluid = 0;
  for (int z = 0; z < s.nz; ++z)
    for (int y = 0; y < s.ny; ++y)
      for (int x = 0; x < s.nx; ++x) {
        const long long hn = ((long long)z * s.ny + y) * s.nx + x;
        if (flags[hn] > LBM_OPEN) { msg = "flags must be 0 (fluid), 1 (solid) or 2 (open)"; return LBM_ERR_ARG; }
        g.flags[((long long)z * s.ny + y) * s.nxp + x] = flags[hn];
      }
  // wall velocities are stored only when some wall link moves
  bool moving = false;
  std::vector<int> cx(Q), cy(Q), cz(Q);
  for (int i = 0; i < Q; ++i) s.lattice_c(i, cx[i], cy[i], cz[i]);
  for (int pass = 0; pass < 2; ++pass) {
    long long nrec = 0;
    for (long long n = 0; n < s.np; ++n) {
      if (pass == 1 && (n & 31) == 0) g.cbase[n >> 5] = (uint32_t)nrec;
      if (g.flags[n] & 3) continue;  // not fluid (the boundary bit is set below)
      if (pass == 0 && (g.flags[n] & 3) == K_FLUID) ++g.nfluid;
      const int x = (int)(n % s.nxp), y = (int)((n / s.nxp) % s.ny), z = (int)(n / ((long long)s.nxp * s.ny));
      const long long hn = ((long long)z * s.ny + y) * s.nx + x;
      Rec r = {0u, 0u, 0u, 0u, 0u};
      for (int i = 0; i < Q; ++i) {
        if (cx[i] == 0 && cy[i] == 0 && cz[i] == 0) continue;
        const long long m = host_neighbour(s, x, y, z, -cx[i], -cy[i], -cz[i]);
        const uint8_t k = g.flags[m] & 3;
        if (k == K_SOLID) r.cut |= 1u << i;
        else if (k == K_OPEN) r.open |= 1u << i;
        else continue;
        const long long ff = host_neighbour(s, x, y, z, cx[i], cy[i], cz[i]);
        if ((g.flags[ff] & 3) == K_FLUID) r.ffok |= 1u << i;
      }
      if (!(r.cut | r.open)) continue;
      ++nrec;
      if (pass == 0) {
        for (int i = 0; i < Q; ++i) {
          if (!(r.cut & (1u << i))) continue;
          const long long li = hn * Q + i;
          const double qq = q ? q[li] : 0.5;
          if (!(qq > 0.0 && qq <= 1.0)) { msg = "q must lie in (0, 1] on every wall link"; return LBM_ERR_ARG; }
          const int tg = tag ? tag[li] : 0;
          if (tg < 0 || tg > 7) { msg = "tags must be 0..7"; return LBM_ERR_ARG; }
          for (int a = 0; a < 3; ++a) {
            if (uw && uw[li * 3 + a] != 0.0) moving = true;
            if (uw1 && uw1[li * 3 + a] != 0.0) moving = true;
          }
        }
        continue;
      }
      r.link0 = (uint32_t)(g.ltag.size());
      if (moving)
        for (int i = 0; i < Q; ++i) {
          if (!(r.cut & (1u << i))) continue;
          const long long li = hn * Q + i;
          for (int a = 0; a < 3; ++a)
            if ((uw && uw[li * 3 + a] != 0.0) || (uw1 && uw1[li * 3 + a] != 0.0)) r.open |= REC_MOVING;
        }
      g.rec.push_back(r);
      g.rnode.push_back((uint32_t)n);
      g.flags[n] |= F_BOUNDARY;
      for (int i = 0; i < Q; ++i) {
        if (!(r.cut & (1u << i))) continue;
        const long long li = hn * Q + i;
        const double qq = q ? q[li] : 0.5;
        if (dbl) push_val<double>(g.lq, qq); else push_val<float>(g.lq, qq);
        g.ltag.push_back((uint8_t)(tag ? tag[li] : 0));
        if (moving) {
          for (int a = 0; a < 3; ++a) {
            const double u0 = uw ? uw[li * 3 + a] : 0.0;
            const double u1 = uw1 ? uw1[li * 3 + a] : u0;
            if (dbl) { push_val<double>(g.luw, u0); push_val<double>(g.luw1, u1); }
            else { push_val<float>(g.luw, u0); push_val<float>(g.luw1, u1); }
          }
        }
      }
    }
    if (pass == 1) g.cbase[s.np >> 5] = (uint32_t)nrec;
  }
  g.has_uw = moving ? 1 : 0;
  return LBM_OK;
}

void unpack_geometry(const lbm_sim &s, const HostGeometry &g, uint8_t *flags, double *q, double *uw,
                     double *uw1, int32_t *tag) {
  const int Q = s.Q;
  const bool dbl = s.link_size() == 8;
  if (flags)
    for (int z = 0; z < s.nz; ++z)
      for (int y = 0; y < s.ny; ++y)
        for (int x = 0; x < s.nx; ++x)
          flags[((long long)z * s.ny + y) * s.nx + x] = g.flags[((long long)z * s.ny + y) * s.nxp + x] & 3;
  if (q) std::memset(q, 0, sizeof(double) * s.N * Q);
  if (uw) std::memset(uw, 0, sizeof(double) * s.N * Q * 3);
  if (uw1) std::memset(uw1, 0, sizeof(double) * s.N * Q * 3);
  if (tag) std::memset(tag, 0, sizeof(int32_t) * s.N * Q);
  for (size_t k = 0; k < g.rec.size(); ++k) {
    const Rec &r = g.rec[k];
    const long long n = g.rnode[k];
    const int x = (int)(n % s.nxp), y = (int)((n / s.nxp) % s.ny), z = (int)(n / ((long long)s.nxp * s.ny));
    const long long hn = ((long long)z * s.ny + y) * s.nx + x;
    uint32_t li = r.link0;
    for (int i = 0; i < Q; ++i) {
      if (!(r.cut & (1u << i))) continue;
      if (q) q[hn * Q + i] = dbl ? get_val<double>(g.lq, li) : get_val<float>(g.lq, li);
      if (tag) tag[hn * Q + i] = g.ltag[li] == TAG_INNER ? -1 : g.ltag[li];
      for (int a = 0; a < 3; ++a) {
        if (g.has_uw) {
          const double u0 = dbl ? get_val<double>(g.luw, li * 3 + a) : get_val<float>(g.luw, li * 3 + a);
          const double u1 = dbl ? get_val<double>(g.luw1, li * 3 + a) : get_val<float>(g.luw1, li * 3 + a);
          if (uw) uw[(hn * Q + i) * 3 + a] = u0;
          if (uw1) uw1[(hn * Q + i) * 3 + a] = u1;
        }
      }
      ++li;
    }
  }
}

}  // namespace lbm
