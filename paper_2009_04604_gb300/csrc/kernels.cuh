// kernels.cuh -- device code of the fused lattice Boltzmann step and its companions.
//
// Layout: populations are stored structure-of-arrays, plane i of buffer f holds
// f[i][z][y][x] with rows padded to nxp (a multiple of 32). Values are shifted,
// f~_i = f_i - w_i rho0, so the reduced-precision formats spend their bits on
// the deviation from rest.
//
// Pull scheme with two buffers (A-B): the thread of node x reads f_i(x,t) from
// slot fin[i][x - c_i] (Eq. LBE: exact on-grid streaming), relaxes with BGK
// (Eq. LB-BGK, equilibrium Eq. Eq2ndOrder, Guo forcing), and writes f*_i(x,t) to
// fout[i][x].
//
// Single-node boundary rule, written ahead. Let link i of a boundary node x_F be
// cut, so x_F - c_i is not fluid. The thread of x_F evaluates the unknown incoming
// population f_i(x_F, t+1) from its own registers alone (Sec. II.C-II.E: f*_ibar(x_F),
// f*_i(x_F), rho_F, u_F, f^neq_ibar(x_F) and the wall data q, u_w). It stores the
// value in slot fout[i][x_F - c_i], the slot its own gather reads at t+1. The
// non-fluid node x_F - c_i never writes, and only x_F reads that slot, so there is
// no race and no second pass. This is the locality the paper argues for in its
// conclusions.
//
// BFL needs f*_ibar(x_FF, t) at x_FF = x_F + c_i, which another thread produces
// in the same step. The thread therefore writes ahead the part it knows,
// 2q g + (1-2q) ME. At t+1 the gather adds (1-2q) f*_ibar(x_FF, t), a value it
// has just loaded as its own population ibar. So BFL costs no extra load.
#pragma once

#include "lattice.cuh"

namespace lbm {

enum { BC_ELIBB_F = 0, BC_ELIBB_FQ = 1, BC_BFL = 2, BC_HWBB = 3, BC_ELIBB_U = 4, BC_ELIBB_UQ = 5 };

// ---------------------------------------------------------------- gather
// ---------------------------------------------------------------- population accesses
// The step kernels load and store population buffers through LD_POP / ST_POP. A build with LBM_DEBUG checks every
// index against [0, v.dbg_limit) first: the buffer's Q x padded nodes, or a
// smaller limit set by lbm_set_debug_limit. An index outside is not accessed (a
// load reads 0), and the first one is recorded in the device word *v.dbg as
// (source line << 40) | (index mod 2^40), which lbm_synchronize reports as
// LBM_ERR_BOUNDS. Without LBM_DEBUG the check compiles away.
__device__ __forceinline__ bool pop_index_ok(const View &v, long long idx, int line) {
#ifdef LBM_DEBUG
  if (idx >= 0 && idx < v.dbg_limit) return true;
  atomicCAS(v.dbg, 0ull, ((unsigned long long)line << 40) | ((unsigned long long)idx & ((1ull << 40) - 1ull)));
  return false;
#else
  (void)v;
  (void)idx;
  (void)line;
  return true;
#endif
}
template <typename T>
__device__ __forceinline__ T ld_pop(const View &v, const T *base, long long idx, int line) {
  return pop_index_ok(v, idx, line) ? __ldg(base + idx) : T{};
}
// a vector of two consecutive elements idx, idx + 1 (V: float2, __half2, ...)
template <typename V, typename T>
__device__ __forceinline__ V ld_pop2(const View &v, const T *base, long long idx, int line) {
  return pop_index_ok(v, idx, line) && pop_index_ok(v, idx + 1, line)
             ? __ldg(reinterpret_cast<const V *>(base + idx))
             : V{};
}
template <typename T>
__device__ __forceinline__ void st_pop(const View &v, T *base, long long idx, T val, int line) {
  if (pop_index_ok(v, idx, line)) base[idx] = val;
}
template <typename V, typename T>
__device__ __forceinline__ void st_pop2(const View &v, T *base, long long idx, V val, int line) {
  if (pop_index_ok(v, idx, line) && pop_index_ok(v, idx + 1, line)) *reinterpret_cast<V *>(base + idx) = val;
}
// The access is written as its pointer expression; base is the buffer's start.
#ifdef LBM_DEBUG
#define LD_POP(v, base, ptr) ld_pop((v), (base), (long long)((ptr) - (base)), __LINE__)
#define LD_POP2(V, v, base, ptr) ld_pop2<V>((v), (base), (long long)((ptr) - (base)), __LINE__)
#define ST_POP(v, base, ptr, ...) st_pop((v), (base), (long long)((ptr) - (base)), (__VA_ARGS__), __LINE__)
#define ST_POP2(v, base, ptr, ...) st_pop2((v), (base), (long long)((ptr) - (base)), (__VA_ARGS__), __LINE__)
#else  // the plain access, compiled exactly as written
#define LD_POP(v, base, ptr) __ldg(ptr)
#define LD_POP2(V, v, base, ptr) __ldg(reinterpret_cast<const V *>(ptr))
#define ST_POP(v, base, ptr, ...) (*(ptr) = (__VA_ARGS__))
#define ST_POP2(v, base, ptr, ...) (*reinterpret_cast<decltype(__VA_ARGS__) *>(ptr) = (__VA_ARGS__))
#endif

template <class L, typename S, typename M>
__device__ __forceinline__ void gather(const View &v, const S *__restrict__ fin, long long n,
                                       const Nbr &nb, M (&f)[L::Q]) {
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    f[i] = to_math<S, M>(LD_POP(v, fin, fin + (long long)i * v.np + n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))));
}

// BFL, q < 1/2: complete the written-ahead part with (1-2q) f*_ibar(x_FF, t),
// which the gather of direction ibar has just read from x_F - c_ibar = x_FF.
template <class L, typename M>
__device__ __forceinline__ void bfl_complete(const View &v, const Rec &r, M (&f)[L::Q]) {
  const M *lq = static_cast<const M *>(v.lq);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const uint32_t bit = 1u << i;
    if (r.cut & r.ffok & bit) {
      const M q = lq[r.link0 + __popc(r.cut & (bit - 1u))];
      if (q < M(0.5)) f[i] += (M(1) - M(2) * q) * f[opp<L>(i)];
    }
  }
}

// Inverse of bfl_complete: the slot of a BFL link with q < 1/2 holds the value minus
// (1-2q) f*_ibar(x_FF), so that the gather's completion restores it. Used when a
// state is written from outside (initialisation, set_populations).
template <class L, typename M>
__device__ __forceinline__ void bfl_encode(const View &v, const Rec &r, M (&f)[L::Q]) {
  const M *lq = static_cast<const M *>(v.lq);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const uint32_t bit = 1u << i;
    if (r.cut & r.ffok & bit) {
      const M q = lq[r.link0 + __popc(r.cut & (bit - 1u))];
      if (q < M(0.5)) f[i] -= (M(1) - M(2) * q) * f[opp<L>(i)];
    }
  }
}

// Record of a boundary node. bal is the warp ballot of the boundary flag, taken by
// a warp that covers 32 consecutive nodes of one row (one 32-node chunk).
__device__ __forceinline__ const Rec *record_of(const View &v, long long n, uint32_t bal) {
  const uint32_t lt = (1u << (threadIdx.x & 31)) - 1u;
  return v.rec + v.cbase[n >> 5] + __popc(bal & lt);
}

// Whether a non-fluid node's lattice lane stores into its slots: when the 32-byte
// sector of its slots holds a fluid node, so that the warp writes the sector
// whole, and unless it lies in a moving body's region. It then stores every
// plane that takes no written-ahead value (View::amask) and the values are
// never read. fluid_bal is the warp ballot of the fluid test, one bit per
// `per` consecutive nodes of each lane (a lane's nodes never straddle a sector).
template <typename S>
__device__ __forceinline__ bool fills_sector(uint8_t fl, uint32_t fluid_bal, int per) {
  constexpr int kNodes = 32 / (int)sizeof(S);  // nodes per 32-byte sector
  const int lanes = kNodes / per >= 32 ? 32 : kNodes / per;
  const int lane = threadIdx.x & 31;
  const uint32_t grp = lanes >= 32 ? 0xffffffffu : (((1u << lanes) - 1u) << (lane & ~(lanes - 1)));
  return (fl & 3) != K_FLUID && !(fl & F_KEEP) && (fluid_bal & grp) != 0;
}

// Explicitly rounded operations (Ex<M>: one rounding per multiply, add and fused
// multiply-add, in the order written). The moments, the relaxation and the
// boundary rule are written with them: the compiler is then free neither to fuse
// nor to split an operation, so every kernel that inlines them (the step
// variants, the batched step, the TMA-staged step) rounds exactly alike. The
// FP32 division is the hardware reciprocal times the dividend (__fdividef: at
// most 2 ulp from the rounded quotient for divisors of normal magnitude, which
// 1/rho and the boundary rule's q, 1-q and 2q^2 are), deterministic like the
// rest; FP64 divides with correct rounding.
template <typename M> struct Ex;
template <> struct Ex<float> {
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
};
template <> struct Ex<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
};

// ---------------------------------------------------------------- moments, equilibrium
template <class L, typename M>
struct Macro {
  M drho, rho, ux, uy, uz, usq;
};

// Density deviation and Guo-corrected velocity, summed over opposite pairs
// (f_i + f_ibar and f_i - f_ibar), with the rest population in the middle slot.
// U: f in the units of the stored values (Units<S>), with Par's stored-units rho0 and F.
template <class L, typename M, bool U = false>
__device__ __forceinline__ Macro<L, M> moments(const View &v, const M (&f)[L::Q]) {
  using X = Ex<M>;
  constexpr int R = L::Q / 2;
  M d = f[R], jx = M(0), jy = M(0), jz = M(0);
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int j = L::Q - 1 - i;
    const M sum = X::add(f[i], f[j]), dif = X::sub(f[i], f[j]);
    d = X::add(d, sum);
    if (L::cx(i) > 0) jx = X::add(jx, dif); else if (L::cx(i) < 0) jx = X::sub(jx, dif);
    if (L::cy(i) > 0) jy = X::add(jy, dif); else if (L::cy(i) < 0) jy = X::sub(jy, dif);
    if (L::cz(i) > 0) jz = X::add(jz, dif); else if (L::cz(i) < 0) jz = X::sub(jz, dif);
  }
  const Par<M> P(v, U);
  Macro<L, M> m;
  m.drho = d;
  m.rho = X::add(P.rho0, d);
  const M inv = X::div(M(1), m.rho);
  if (v.has_force) {  // Guo: u = (sum c f + F/2) / rho
    jx = X::fma(M(0.5), P.F[0], jx);
    jy = X::fma(M(0.5), P.F[1], jy);
    jz = X::fma(M(0.5), P.F[2], jz);
  }
  m.ux = X::mul(jx, inv);
  m.uy = X::mul(jy, inv);
  m.uz = X::mul(jz, inv);
  m.usq = X::fma(m.uz, m.uz, X::fma(m.uy, m.uy, X::mul(m.ux, m.ux)));
  return m;
}

// c_i . a for a compile-time direction i: a signed sum of the components, each
// added or subtracted in the order x, y, z (the selection itself is exact)
template <class L, typename M>
__device__ __forceinline__ M cdot_c(int i, M ax, M ay, M az) {
  using X = Ex<M>;
  M r = M(0);
  bool any = false;
  if (L::cx(i) != 0) { r = L::cx(i) > 0 ? ax : -ax; any = true; }
  if (L::cy(i) != 0) { r = any ? (L::cy(i) > 0 ? X::add(r, ay) : X::sub(r, ay)) : (L::cy(i) > 0 ? ay : -ay); any = true; }
  if (L::cz(i) != 0) { r = any ? (L::cz(i) > 0 ? X::add(r, az) : X::sub(r, az)) : (L::cz(i) > 0 ? az : -az); }
  return r;
}

// shifted equilibrium f^eq_i(rho, u) - w_i rho0 = w_i [drho + rho (3 cu + 9/2 cu^2 - 3/2 u^2)]
template <class L, typename M>
__device__ __forceinline__ M feq_s(int i, M drho, M rho, M ux, M uy, M uz, M usq) {
  const M cu = M(L::cx(i)) * ux + M(L::cy(i)) * uy + M(L::cz(i)) * uz;
  return M(weight<L>(i)) * (drho + rho * (M(3) * cu + M(4.5) * cu * cu - M(1.5) * usq));
}

// Compile-time physics of a step kernel: bit 0 adds the Guo body force, bit 1
// selects the TRT collision instead of BGK.
enum : int { PH_FORCE = 1, PH_TRT = 2 };

// Bulk relaxation, by opposite pairs (i, ibar). The shifted equilibrium splits into
// an even part e+ = w [drho - 3/2 rho u^2 + 9/2 rho (c.u)^2], shared by the pair,
// and an odd part e- = 3 w rho (c.u), which flips sign. The Guo source splits the
// same way: S+ = w (9 (c.u)(c.F) - 3 u.F), S- = 3 w (c.F).
//  - BGK (Eq. LB-BGK): f*_i = (1 - omega) f_i + omega (e+ + e-) + k (S+ + S-),
//    k = 1 - omega/2.
//  - TRT (Sec. II.A): with f+ = (f_i + f_ibar)/2 and f- = (f_i - f_ibar)/2,
//    f*_i = f_i + omega+ (e+ - f+) + omega- (e- - f-) + k+ S+ + k- S-, where
//    k+- = 1 - omega+-/2, omega+ = 1/tau and omega- follows from the magic
//    parameter (Eq. magic-parameter).
// The relaxed value of direction i goes to put(i, value); collide_store writes it
// to the output planes, post_all to registers. Every operation is explicitly
// rounded (Ex<M>), so that all kernels relax a node bit for bit alike.
template <class L, typename M, int PHYS, bool U, class Put>
__device__ __forceinline__ void relax(const View &v, const M (&f)[L::Q], const Macro<L, M> &m, Put &&put) {
  using X = Ex<M>;
  constexpr bool FORCE = (PHYS & PH_FORCE) != 0, TRT = (PHYS & PH_TRT) != 0;
  constexpr int R = L::Q / 2;
  const Par<M> P(v, U);
  const M om = P.omega, omr = X::sub(M(1), om);
  M Fx = M(0), Fy = M(0), Fz = M(0), kf = M(0), km = M(0), uF3 = M(0);
  if constexpr (FORCE) {
    Fx = P.F[0]; Fy = P.F[1]; Fz = P.F[2];
    kf = X::fma(M(-0.5), om, M(1));
    if constexpr (TRT) km = X::fma(M(-0.5), P.omega_m, M(1));
    uF3 = X::mul(M(-3), X::fma(m.uz, Fz, X::fma(m.uy, Fy, X::mul(m.ux, Fx))));  // -3 u.F
  }
  if constexpr (TRT) {
    const M omm = P.omega_m;
    const M d0 = X::fma(X::mul(M(-1.5), m.rho), m.usq, m.drho);
    const M rho45 = X::mul(M(4.5), m.rho);
    {
      const M w = M(weight<L>(R));
      M r = X::fma(om, X::sub(X::mul(w, d0), f[R]), f[R]);
      if constexpr (FORCE) r = X::fma(X::mul(w, kf), uF3, r);
      put(R, r);
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int j = L::Q - 1 - i;
      const M w = M(weight<L>(i)), w3 = M(3.0 * weight<L>(i));
      const M cu = cdot_c<L, M>(i, m.ux, m.uy, m.uz);
      const M ep = X::mul(w, X::fma(X::mul(rho45, cu), cu, d0)), em = X::mul(X::mul(w3, m.rho), cu);
      M dp = X::mul(om, X::fma(M(-0.5), X::add(f[i], f[j]), ep));
      M dm = X::mul(omm, X::fma(M(-0.5), X::sub(f[i], f[j]), em));
      if constexpr (FORCE) {
        const M cF = cdot_c<L, M>(i, Fx, Fy, Fz);
        dp = X::fma(X::mul(kf, w), X::fma(X::mul(M(9), cu), cF, uF3), dp);
        dm = X::fma(X::mul(km, w3), cF, dm);
      }
      put(i, X::add(f[i], X::add(dp, dm)));
      put(j, X::add(f[j], X::sub(dp, dm)));
    }
  } else {
    const M wr = X::mul(om, m.rho);
    const M b0 = X::mul(om, X::fma(X::mul(M(-1.5), m.rho), m.usq, m.drho));
    const M wr45 = X::mul(M(4.5), wr);
    {
      const M w = M(weight<L>(R));
      M eq = X::mul(w, b0);
      if constexpr (FORCE) eq = X::fma(X::mul(w, kf), uF3, eq);
      put(R, X::fma(omr, f[R], eq));
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int j = L::Q - 1 - i;
      const M w = M(weight<L>(i)), w3 = M(3.0 * weight<L>(i));
      const M cu = cdot_c<L, M>(i, m.ux, m.uy, m.uz);
      M sym = X::mul(w, X::fma(X::mul(wr45, cu), cu, b0));
      M asym = X::mul(X::mul(w3, wr), cu);
      if constexpr (FORCE) {
        const M cF = cdot_c<L, M>(i, Fx, Fy, Fz);
        sym = X::fma(X::mul(kf, w), X::fma(X::mul(M(9), cu), cF, uF3), sym);
        asym = X::fma(X::mul(kf, w3), cF, asym);
      }
      put(i, X::fma(omr, f[i], X::add(sym, asym)));
      put(j, X::fma(omr, f[j], X::sub(sym, asym)));
    }
  }
}

// The lattice tiles' relaxation, in the units of the stored values (Units<S>).
// skip: planes not to store (bit i); 0 for fluid nodes.
template <class L, typename S, typename M, int PHYS>
__device__ __forceinline__ void collide_store(const View &v, const M (&f)[L::Q], const Macro<L, M> &m,
                                              S *__restrict__ fout, int n, int np, uint32_t skip) {
  relax<L, M, PHYS, Units<S>::kStored>(v, f, m, [&](int i, M val) {
    if (!((skip >> i) & 1u)) ST_POP(v, fout, fout + n + i * np, Units<S>::template store<M>(val));
  });
}

// The same, storing node n's planes at the view's precomputed plane offsets.
template <class L, typename S, typename M, int PHYS>
__device__ __forceinline__ void collide_store_at(const View &v, const M (&f)[L::Q], const Macro<L, M> &m,
                                                 S *__restrict__ fout, int n, uint32_t skip) {
  relax<L, M, PHYS, Units<S>::kStored>(v, f, m, [&](int i, M val) {
    if (!((skip >> i) & 1u)) ST_POP(v, fout, &fout[v.soff[i] + n], Units<S>::template store<M>(val));
  });
}

template <class L, typename M, int PHYS, bool U>
__device__ __forceinline__ void post_all(const View &v, const M (&f)[L::Q], const Macro<L, M> &m,
                                         M (&out)[L::Q]) {
  relax<L, M, PHYS, U>(v, f, m, [&](int i, M val) { out[i] = val; });
}

// ---------------------------------------------------------------- boundary rule
// Unknown incoming population f_i(x_F, t+1) (shifted) of every wall or open link.
// Points on the link, by the s coordinate of Eq. x_to_s_helper:
//   f0 = f~_i^{t+1}(x_W) = f^eq_i(rho_F, u_w(t+1)) + f^neq_ibar(x_F)            s = 0
//   g  = f*_ibar(x_F) + ME, ME = 2 w_i rho_F c_i.u_w / c_s^2 (Eq. ME-solid-to-fluid)  s = 1-q
//   f1 = f~*_i(x_W) = f^eq_i(rho_F, u_w(t)) + (1 - omega) f^neq_ibar(x_F)          s = 1
//   h  = f*_i(x_F)                                                                 s = 1+q
// Weights: Lagrange weights (Eq. poli_coeff) at s_ref = q, in closed form:
//   ELIBB-F  (Eq. linear_broken_method): f0, g for q < 1/2; g, f1 for q >= 1/2;
//   ELIBB-FQ (Eq. quadratic_fragmented_method): f0, g, f1 for q < 1/2 (ELIBB-F
//            below q_cut); g, f1, h for q >= 1/2;
//   ELIBB-U  (Eq. unified_space_coordinates): (1 - q) f0 + q f1;
//   ELIBB-UQ (Eq. elibbqu): f0, g, f1 for every q, which is
//            (1 - 2q) f0 + g + (2q - 1) f1; ELIBB-U where 1 - q < q_cut, where
//            the points s = 0 and s = 1 - q meet.
// At q = 1/2 every rule but ELIBB-U reduces exactly to g (half-way bounce-back).
// Under TRT the post-collision wall value f1 keeps the factor (1 - omega+): the
// wall non-equilibrium is even in c at first order.
// The loop runs over the set bits of the link masks with a run-time direction
// index, which keeps the code small. The node's populations sit in shared memory
// (fs[i*stride]), and the direction constants come from packed words.

// c_i . a for a run-time direction
template <class L, typename M>
__device__ __forceinline__ M cdot_r(int i, M ax, M ay, M az) {
  using X = Ex<M>;
  return X::fma(M(dcz<L>(i)), az, X::fma(M(dcy<L>(i)), ay, X::mul(M(dcx<L>(i)), ax)));
}

// shifted equilibrium w_i [drho + rho (3 cu + 9/2 cu^2 - 3/2 u^2)] for a run-time direction
template <class L, typename M>
__device__ __forceinline__ M feq_r(int i, M drho, M rho, M ux, M uy, M uz, M usq) {
  using X = Ex<M>;
  const M cu = cdot_r<L, M>(i, ux, uy, uz);
  const M t = X::fma(X::mul(M(4.5), cu), cu, X::fma(M(3), cu, X::mul(M(-1.5), usq)));
  return X::mul(dweight<L, M>(i), X::fma(rho, t, drho));
}

// post-collision value (with the Guo source) of direction i, whose opposite
// population is fo, for a run-time direction; BGK or TRT as in relax
template <class L, typename M, bool BGK = false>
__device__ __forceinline__ M post_r(const View &v, const Par<M> &P, int i, M fi, M fo, const Macro<L, M> &m) {
  using X = Ex<M>;
  const M w = dweight<L, M>(i);
  const M cu = cdot_r<L, M>(i, m.ux, m.uy, m.uz);
  M r;
  if (!BGK && v.trt) {
    const M e2 = X::fma(X::mul(M(4.5), cu), cu, X::mul(M(-1.5), m.usq));
    const M ep = X::mul(w, X::fma(m.rho, e2, m.drho));
    const M em = X::mul(X::mul(M(3), w), X::mul(m.rho, cu));
    const M fp = X::mul(M(0.5), X::add(fi, fo)), fm = X::mul(M(0.5), X::sub(fi, fo));
    r = X::fma(P.omega_m, X::sub(em, fm), X::fma(P.omega, X::sub(ep, fp), fi));
  } else {
    r = X::fma(P.omega, X::sub(feq_r<L, M>(i, m.drho, m.rho, m.ux, m.uy, m.uz, m.usq), fi), fi);
  }
  if (v.has_force) {
    const M cF = cdot_r<L, M>(i, P.F[0], P.F[1], P.F[2]);
    const M uF = X::fma(m.uz, P.F[2], X::fma(m.uy, P.F[1], X::mul(m.ux, P.F[0])));
    const M kp = X::fma(M(-0.5), P.omega, M(1));
    const M km = X::fma(M(-0.5), !BGK && v.trt ? P.omega_m : P.omega, M(1));
    const M sp = X::fma(X::mul(M(9), cu), cF, X::mul(M(-3), uF));
    r = X::fma(w, X::fma(kp, sp, X::mul(X::mul(M(3), km), cF)), r);
  }
  return r;
}

// element offset of node (x, y, z) - c, with the periodic and sheared wraps
__device__ __forceinline__ int upstream_offset(const View &v, int x, int y, int z, int cx, int cy, int cz) {
  int X = x - cx, Y = y - cy, Z = z - cz;
  if (X < 0) { X += v.nx; Y += v.xshift; }
  else if (X >= v.nx) { X -= v.nx; Y -= v.xshift; }
  if (v.xshift != 0) { Y %= v.ny; if (Y < 0) Y += v.ny; }
  else { Y = Y < 0 ? Y + v.ny : (Y >= v.ny ? Y - v.ny : Y); }
  Z = Z < 0 ? Z + v.nz : (Z >= v.nz ? Z - v.nz : Z);
  return ((Z - z) * v.ny + (Y - y)) * v.nxp + (X - x);
}

// Non-equilibrium stress of a node, Pi_ab = sum_j c_ja c_jb (f_j - f^eq_j), from
// its shifted populations: Pi = sum_j c_j c_j f~_j - drho c_s^2 I - rho u u (in
// the lattice's own dimensions).
// Components xx, yy, zz, xy, xz, yz.
template <class L, typename M>
__device__ __forceinline__ void neq_stress(const M (&f)[L::Q], const Macro<L, M> &m, M (&pi)[6]) {
  using X = Ex<M>;
  M s[6] = {M(0), M(0), M(0), M(0), M(0), M(0)};
#pragma unroll
  for (int j = 0; j < L::Q; ++j) {
    const int cx = L::cx(j), cy = L::cy(j), cz = L::cz(j);
    if (cx) s[0] = X::add(s[0], f[j]);
    if (cy) s[1] = X::add(s[1], f[j]);
    if (cz) s[2] = X::add(s[2], f[j]);
    if (cx * cy) s[3] = cx * cy > 0 ? X::add(s[3], f[j]) : X::sub(s[3], f[j]);
    if (cx * cz) s[4] = cx * cz > 0 ? X::add(s[4], f[j]) : X::sub(s[4], f[j]);
    if (cy * cz) s[5] = cy * cz > 0 ? X::add(s[5], f[j]) : X::sub(s[5], f[j]);
  }
  const M d = X::mul(m.drho, M(1.0 / 3.0));
  const M ru[3] = {X::mul(m.rho, m.ux), X::mul(m.rho, m.uy), X::mul(m.rho, m.uz)};
  pi[0] = X::sub(X::sub(s[0], d), X::mul(ru[0], m.ux));
  pi[1] = X::sub(X::sub(s[1], d), X::mul(ru[1], m.uy));
  // a 2-D lattice has no z velocities: its equilibrium has no zz moment either
  pi[2] = L::D == 2 ? M(0) : X::sub(X::sub(s[2], d), X::mul(ru[2], m.uz));
  pi[3] = X::sub(s[3], X::mul(ru[0], m.uy));
  pi[4] = X::sub(s[4], X::mul(ru[0], m.uz));
  pi[5] = X::sub(s[5], X::mul(ru[1], m.uz));
}

// Regularized estimate of the non-equilibrium part of wall population i (the
// appendix's Eq. fi_neq, third-order truncation): with a2 = Pi and, by Eq.
// malaspinas, a3_abc = u_c Pi_ab + u_b Pi_ac + u_a Pi_bc (u the wall velocity),
//   f1_i = w_i [H2_i : a2 / (2 c_s^4) + H3_i : a3 / (6 c_s^6)]
//        = w_i [9/2 (c.Pi.c) - 3/2 tr Pi + 27/2 (c.u)(c.Pi.c) - 9/2 (2 c.Pi.u + (c.u) tr Pi)].
template <class L, typename M>
__device__ __forceinline__ M neq_regularized(int i, const M (&pi)[6], M ux, M uy, M uz) {
  using X = Ex<M>;
  const M cx = M(dcx<L>(i)), cy = M(dcy<L>(i)), cz = M(dcz<L>(i));
  const M pcx = X::fma(cz, pi[4], X::fma(cy, pi[3], X::mul(cx, pi[0])));  // (Pi c)_x
  const M pcy = X::fma(cz, pi[5], X::fma(cy, pi[1], X::mul(cx, pi[3])));  // (Pi c)_y
  const M pcz = X::fma(cz, pi[2], X::fma(cy, pi[5], X::mul(cx, pi[4])));  // (Pi c)_z
  const M cpc = X::fma(cz, pcz, X::fma(cy, pcy, X::mul(cx, pcx)));
  const M cpu = X::fma(uz, pcz, X::fma(uy, pcy, X::mul(ux, pcx)));
  const M tr = X::add(X::add(pi[0], pi[1]), pi[2]);
  const M cu = cdot_r<L, M>(i, ux, uy, uz);
  const M t2 = X::fma(M(4.5), cpc, X::mul(M(-1.5), tr));
  const M t3 = X::fma(X::mul(M(13.5), cu), cpc, X::mul(M(-4.5), X::fma(M(2), cpu, X::mul(cu, tr))));
  return X::mul(dweight<L, M>(i), X::add(t2, t3));
}

// RULE >= 0: the rule is BC_ELIBB_F or BC_ELIBB_FQ under BGK with the bounce-back
// wall non-equilibrium, known at compile time, so that the link loop carries no
// run-time choice of rule; a static wall (u_w = 0) then also skips the
// wall-velocity terms, f^eq_i(rho, 0) = w_i drho and no moving-wall term, which
// the general form computes with zeros. RULE < 0: every rule, chosen at run time.
// A node whose neighbours need no wrap finds its written-ahead slots at the
// host's per-direction offsets (View::loff).
template <class L, typename S, typename M, int RULE>
__device__ __forceinline__ void boundary_rule(const View &v, const RecSet &rs, const Rec &r, const M *fs,
                                              int stride, const Macro<L, M> &m, const M (&pi)[6], long long n,
                                              int x, int y, int z, S *__restrict__ fout) {
  using X = Ex<M>;
  constexpr bool SPEC = RULE >= 0;
  const int bc = SPEC ? RULE : v.bc;
  const M *lq = static_cast<const M *>(rs.lq);
  const M *luw = static_cast<const M *>(rs.luw);
  const M *luw1 = static_cast<const M *>(rs.luw1);
  const Par<M> P(v);
  const uint32_t open = r.open & ~REC_MOVING;
  const bool moving = luw != nullptr && (r.open & REC_MOVING);
  const bool interior = x > 0 && x < v.nx - 1 && y > 0 && y < v.ny - 1 && (L::D == 2 || (z > 0 && z < v.nz - 1));
  uint32_t links = r.cut | open;
#pragma unroll 1
  while (links) {
    const int i = __ffs(links) - 1;
    const uint32_t bit = 1u << i;
    links &= links - 1u;
    const int ib = opp<L>(i);
    const M fib = fs[ib * stride];
    M val;
    if (open & bit) {
      // single-node pressure outlet: f^eq_i(rho0, u_F) + f^neq_ibar(x_F)
      const M fneq_ib = X::sub(fib, feq_r<L, M>(ib, m.drho, m.rho, m.ux, m.uy, m.uz, m.usq));
      val = X::add(feq_r<L, M>(i, M(0), P.rho0, m.ux, m.uy, m.uz, m.usq), fneq_ib);
    } else {
      const uint32_t li = r.link0 + __popc(r.cut & (bit - 1u));
      const M q = lq[li];
      const M w = dweight<L, M>(i);
      const M fi = fs[i * stride];
      const M q2 = X::mul(M(2), q);               // 2q (exact)
      const M a = X::sub(q2, M(1)), oma = X::sub(M(1), q2);  // 2q - 1, 1 - 2q
      const M omq = X::sub(M(1), q);              // 1 - q
      if constexpr (SPEC) {
        const M fneq_ib = X::sub(fib, feq_r<L, M>(ib, m.drho, m.rho, m.ux, m.uy, m.uz, m.usq));
        M g = post_r<L, M, true>(v, P, ib, fib, fi, m), f0, f1;
        if (moving) {
          const M wx = luw[3 * li], wy = luw[3 * li + 1], wz = luw[3 * li + 2];
          const M vx = luw1[3 * li], vy = luw1[3 * li + 1], vz = luw1[3 * li + 2];
          g = X::add(g, X::mul(X::mul(X::mul(M(6), w), m.rho), cdot_r<L, M>(i, wx, wy, wz)));
          const M u0sq = X::fma(wz, wz, X::fma(wy, wy, X::mul(wx, wx)));
          const M u1sq = X::fma(vz, vz, X::fma(vy, vy, X::mul(vx, vx)));
          f1 = X::fma(X::sub(M(1), P.omega), fneq_ib, feq_r<L, M>(i, m.drho, m.rho, wx, wy, wz, u0sq));
          f0 = X::add(feq_r<L, M>(i, m.drho, m.rho, vx, vy, vz, u1sq), fneq_ib);
        } else {
          const M weq = X::mul(w, m.drho);  // f^eq_i(rho, 0), shifted
          f1 = X::fma(X::sub(M(1), P.omega), fneq_ib, weq);
          f0 = X::add(weq, fneq_ib);
        }
        if (q == M(0.5)) {
          val = g;
        } else if (q < M(0.5)) {
          if (RULE == BC_ELIBB_FQ && q >= P.qcut)
            val = X::fma(a, f1, X::fma(oma, f0, g));                  // (1-2q) f0 + g + (2q-1) f1
          else
            val = X::div(X::fma(q, g, X::mul(oma, f0)), omq);         // ((1-2q) f0 + q g) / (1-q)
        } else if (RULE == BC_ELIBB_FQ) {
          const M h = post_r<L, M, true>(v, P, i, fi, fib, m);
          val = X::div(X::fma(X::mul(a, X::sub(q, M(1))), h, X::fma(X::mul(M(2), a), f1, X::mul(omq, g))),
                       X::mul(q2, q));
        } else {
          val = X::div(X::fma(a, f1, X::mul(omq, g)), q);              // ((1-q) g + (2q-1) f1) / q
        }
      } else {
        M wx = M(0), wy = M(0), wz = M(0), vx = M(0), vy = M(0), vz = M(0);
        if (moving) {
          wx = luw[3 * li]; wy = luw[3 * li + 1]; wz = luw[3 * li + 2];
          vx = luw1[3 * li]; vy = luw1[3 * li + 1]; vz = luw1[3 * li + 2];
        }
        const M me = X::mul(X::mul(X::mul(M(6), w), m.rho), cdot_r<L, M>(i, wx, wy, wz));
        const M g = X::add(post_r<L, M>(v, P, ib, fib, fi, m), me);
        if (bc == BC_HWBB || (q == M(0.5) && bc != BC_ELIBB_U)) {
          val = g;
        } else if (bc == BC_BFL) {
          if (q < M(0.5)) {
            val = (r.ffok & bit) ? X::fma(q2, g, X::mul(oma, me)) : g;
          } else {
            const M h = post_r<L, M>(v, P, i, fi, fib, m);
            val = X::div(X::fma(a, h, g), q2);
          }
        } else {
          // wall non-equilibrium: f^neq_ibar(x_F) (Eq. neqbb-s), or the regularized
          // estimate with the wall velocity of each wall point's time (Eq. fi_neq)
          const M fneq_ib = X::sub(fib, feq_r<L, M>(ib, m.drho, m.rho, m.ux, m.uy, m.uz, m.usq));
          const bool reg = v.wall_neq != 0;
          const M fn1 = reg ? neq_regularized<L, M>(i, pi, wx, wy, wz) : fneq_ib;
          const M fn0 = reg ? neq_regularized<L, M>(i, pi, vx, vy, vz) : fneq_ib;
          const M u0sq = X::fma(wz, wz, X::fma(wy, wy, X::mul(wx, wx)));
          const M f1 = X::fma(X::sub(M(1), P.omega), fn1, feq_r<L, M>(i, m.drho, m.rho, wx, wy, wz, u0sq));
          const bool unified_lin = bc == BC_ELIBB_U || (bc == BC_ELIBB_UQ && omq < P.qcut);
          if (unified_lin || q < M(0.5) || bc == BC_ELIBB_UQ) {
            const M u1sq = X::fma(vz, vz, X::fma(vy, vy, X::mul(vx, vx)));
            const M f0 = X::add(feq_r<L, M>(i, m.drho, m.rho, vx, vy, vz, u1sq), fn0);
            if (unified_lin)  // ELIBB-U: the wall points s = 0 and s = 1 only
              val = X::fma(q, f1, X::mul(omq, f0));
            else if ((bc == BC_ELIBB_FQ && q >= P.qcut) || bc == BC_ELIBB_UQ)
              val = X::fma(a, f1, X::fma(oma, f0, g));                  // (1-2q) f0 + g + (2q-1) f1
            else
              val = X::div(X::fma(q, g, X::mul(oma, f0)), omq);         // ((1-2q) f0 + q g) / (1-q)
          } else if (bc == BC_ELIBB_FQ) {
            // ((1-q) g + 2 (2q-1) f1 + (2q-1)(q-1) h) / (2 q^2)
            const M h = post_r<L, M>(v, P, i, fi, fib, m);
            val = X::div(X::fma(X::mul(a, X::sub(q, M(1))), h, X::fma(X::mul(M(2), a), f1, X::mul(omq, g))),
                         X::mul(q2, q));
          } else {
            val = X::div(X::fma(a, f1, X::mul(omq, g)), q);              // ((1-q) g + (2q-1) f1) / q
          }
        }
      }
    }
    const long long slot = interior ? (long long)v.loff[i] + n
                                    : (long long)i * v.np + n + upstream_offset(v, x, y, z, dcx<L>(i), dcy<L>(i), dcz<L>(i));
    ST_POP(v, fout, &fout[slot], to_store<S, M>(val));
  }
}

// The general rule (TRT, the regularized wall estimate, BFL, HWBB, ELIBB-U/UQ) is a
// call of its own: its registers then do not count against a step kernel's budget,
// which the lattice tiles and the specialised rules set, and a kernel compiled for
// 40 or 48 registers spills only around this call, on the general path. The step
// kernels take their view as a grid constant, so that passing it by reference
// makes no per-thread copy.
template <class L, typename S, typename M>
__device__ __noinline__ void boundary_general(const View &v, const RecSet &rs, const Rec &r, const M *fs,
                                              int stride, const Macro<L, M> &m, const M (&pi)[6], long long n,
                                              int x, int y, int z, S *__restrict__ fout) {
  boundary_rule<L, S, M, -1>(v, rs, r, fs, stride, m, pi, n, x, y, z, fout);
}

template <class L, typename S, typename M>
__device__ void boundary(const View &v, const RecSet &rs, const Rec &r, const M *fs, int stride,
                         const Macro<L, M> &m, const M (&pi)[6], long long n, int x, int y, int z,
                         S *__restrict__ fout) {
  const bool bgk_bb = !v.trt && !v.wall_neq;
  if (bgk_bb && v.bc == BC_ELIBB_F)
    boundary_rule<L, S, M, BC_ELIBB_F>(v, rs, r, fs, stride, m, pi, n, x, y, z, fout);
  else if (bgk_bb && v.bc == BC_ELIBB_FQ)
    boundary_rule<L, S, M, BC_ELIBB_FQ>(v, rs, r, fs, stride, m, pi, n, x, y, z, fout);
  else
    boundary_general<L, S, M>(v, rs, r, fs, stride, m, pi, n, x, y, z, fout);
}

// non-binding request to bring the line holding p into L1
__device__ __forceinline__ void prefetch_l1(const void *p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// The boundary work of one boundary node: the node's own pre-collision
// populations (gathered from fin, which is unchanged during the step, and
// BFL-completed), its moments, and the written-ahead unknowns of its wall and
// open links. fs is this thread's column of the block's shared staging array.
template <class L, typename S, typename M>
__device__ __forceinline__ void boundary_node(const View &v, const RecSet &rs, const Rec r,
                                              const S *__restrict__ fin, S *__restrict__ fout, long long n,
                                              int x, int y, int z, M *fs, int stride) {
  // The link loop reads q (and the wall velocities) one link after another. Ask
  // for the record's contiguous link data now, so that it is in L1 by then and
  // the loop does not wait on memory once per link.
  if (r.cut) {
    const uint32_t l0 = r.link0, l1 = r.link0 + __popc(r.cut) - 1u;
    prefetch_l1(static_cast<const M *>(rs.lq) + l0);
    prefetch_l1(static_cast<const M *>(rs.lq) + l1);
    if (rs.luw != nullptr && (r.open & REC_MOVING)) {
      prefetch_l1(static_cast<const M *>(rs.luw) + 3 * l0);
      prefetch_l1(static_cast<const M *>(rs.luw) + 3 * l1 + 2);
      prefetch_l1(static_cast<const M *>(rs.luw1) + 3 * l0);
      prefetch_l1(static_cast<const M *>(rs.luw1) + 3 * l1 + 2);
    }
  }
  M f[L::Q];
  if (x > 0 && x < v.nx - 1 && y > 0 && y < v.ny - 1 && (L::D == 2 || (z > 0 && z < v.nz - 1))) {
#pragma unroll
    for (int i = 0; i < L::Q; ++i) f[i] = to_math<S, M>(LD_POP(v, fin, fin + (v.loff[i] + n)));
  } else {
    Nbr nb;
    nb.init(v, x, y, z);
    gather<L, S, M>(v, fin, n, nb, f);
  }
  if (v.bc == BC_BFL) bfl_complete<L, M>(v, r, f);
  const Macro<L, M> m = moments<L, M>(v, f);
  M pi[6] = {M(0), M(0), M(0), M(0), M(0), M(0)};
  if (v.wall_neq) neq_stress<L, M>(f, m, pi);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) fs[i * stride] = f[i];
  if (r.shell) {
    // A node with links across a thin shell is relaxed here, not by its lattice
    // tile. Its post-collision population i streams to n + c_i. When link ibar
    // crosses the shell, n + c_i is the fluid node on the other side, whose
    // boundary rule writes that slot ahead: this node stores nothing there.
    const Par<M> P(v);
#pragma unroll 1
    for (int i = 0; i < L::Q; ++i) {
      const int ib = opp<L>(i);
      if ((r.shell >> ib) & 1u) continue;
      ST_POP(v, fout, &fout[v.soff[i] + n], to_store<S, M>(post_r<L, M>(v, P, i, fs[i * stride], fs[ib * stride], m)));
    }
  }
  boundary<L, S, M>(v, rs, r, fs, stride, m, pi, n, x, y, z, fout);
}

// Quotients by divisors fixed for a run (the tiles per row gx, the padded row
// nxp, the plane nxp ny): t / d by one wide multiply and a shift (division by an
// invariant integer, Granlund and Montgomery). With l = floor(log2 d) the host
// sets m = ceil(2^(32+l) / d) < 2^32 and s = 32 + l, or m = 2^31 and s = 31 + l
// when d is a power of two. The error of the product is below
// t / 2^(32+l) < 1 / (2 d) for t < 2^31, so the quotient is exact.
__device__ __forceinline__ int div_by(int t, uint32_t m, uint32_t s) {
  return (int)(((unsigned long long)(unsigned)t * m) >> s);
}

// column and row of lattice tile t in its plane
__device__ __forceinline__ int2 tile_coords(const View &v, int t) {
  const int ty = div_by(t, v.gx_m, v.gx_s);
  return make_int2(t - ty * v.gx, ty);
}

// x, y, z of padded node n (n < 2^31), with the same multiply-and-shift quotients
// by nxp and nxp ny
__device__ __forceinline__ int3 node_coords(const View &v, int n) {
  const int z = div_by(n, v.pl_m, v.pl_s);
  const int r = n - z * v.nxp * v.ny;
  const int y = div_by(r, v.nxp_m, v.nxp_s);
  return make_int3(r - y * v.nxp, y, z);
}

// ---------------------------------------------------------------- the fused step
// One launch does the whole update t -> t+1. Each block takes one entry of the
// tile table v.tiles:
//  - lattice tile {z, t}: a bx-by-by block of plane z (bx a multiple of 32 that
//    divides nxp, so a warp covers one 32-node chunk of a row). Every fluid
//    node, boundary nodes included, is gathered, relaxed and stored;
//  - boundary tile {-1 - count, first}: records first .. first+count-1, one
//    thread per boundary node. Each evaluates the boundary rule of its node
//    and writes the unknowns ahead into the non-fluid slots that only this
//    node reads.
// The table lists plane z's boundary tiles right after its lattice tiles. The
// boundary threads' gathers then hit the lines the plane's lattice threads have
// just brought into L2, and their written-ahead values complete the same
// sectors in L2. The two kinds touch disjoint output slots and only read fin,
// so they need no ordering. Dense boundary tiles keep the rule off the lattice
// warps, where wall rows would otherwise diverge into it for every lane.
// MINB is the minimum number of resident 256-thread blocks per SM that the
// register allocation must allow (1: unconstrained); the autotuner picks it.
// PHYS selects the body-force path and the collision (PH_FORCE, PH_TRT) at
// compile time. Element offsets are 32-bit,
// since the library keeps Q x padded nodes below 2^31 per simulation.
// Lattice tile {z, t} of the table: gather, relax and store every fluid node (in
// the units of the stored values, Units<S>). A non-fluid node whose 32-byte sector
// holds a fluid node stores the relaxation of zeros into the planes that take no
// written-ahead value, values that nothing reads, so that the warp writes every
// sector it touches whole.
template <class L, typename S, typename M, int PHYS>
__device__ __forceinline__ void lattice_tile(const View &v, const S *__restrict__ fin,
                                             S *__restrict__ fout, int2 tile) {
  const int2 tc = tile_coords(v, tile.y);
  const int x = tc.x * blockDim.x + threadIdx.x;
  const int y = tc.y * blockDim.y + threadIdx.y;
  const int z = tile.x;
  if (y >= v.ny) return;  // uniform across the warp
  const int n = (z * v.ny + y) * v.nxp + x;
  const uint8_t fl = v.flags[n];
  const uint32_t fbal = __ballot_sync(0xffffffffu, (fl & 3) == K_FLUID);
  if (!fbal) return;  // the whole warp is idle
  uint32_t bal = 0;
  if (v.bc == BC_BFL) bal = __ballot_sync(0xffffffffu, fl & F_BOUNDARY);
  const bool here = (fl & K_LATTICE_MASK) == K_FLUID;  // fluid, and not relaxed by its boundary tile
  const bool fill = fills_sector<S>(fl, fbal, 1);      // a non-fluid node completing a sector
  const bool masked = __any_sync(0xffffffffu, fill);   // the warp's stores need the per-plane masks
  if (!here && !fill) return;
  const int np = (int)v.np;
  M f[L::Q];
  uint32_t skip = 0;
  if (here) {
    const bool interior = x > 0 && x < v.nx - 1 && y > 0 && y < v.ny - 1 &&
                          (L::D == 2 || (z > 0 && z < v.nz - 1));
    if (interior) {
      // no wrap: the source of population i is n - c_i, at an offset that is the
      // same for every thread and precomputed on the host (loff)
#pragma unroll
      for (int i = 0; i < L::Q; ++i) f[i] = Units<S>::template load<M>(LD_POP(v, fin, fin + (v.loff[i] + n)));
    } else {
      Nbr nb;
      nb.init(v, x, y, z);
      const S *__restrict__ src = fin + n;
#pragma unroll
      for (int i = 0; i < L::Q; ++i)
        f[i] = Units<S>::template load<M>(LD_POP(v, fin, src + (i * np + nb.at(-L::cx(i), -L::cy(i), -L::cz(i)))));
    }
    if (v.bc == BC_BFL && (fl & F_BOUNDARY)) bfl_complete<L, M>(v, *record_of(v, n, bal), f);
  } else {
    skip = v.amask[n];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) f[i] = M(0);
  }
  const Macro<L, M> m = moments<L, M, Units<S>::kStored>(v, f);
  if (masked) collide_store_at<L, S, M, PHYS>(v, f, m, fout, n, skip);
  else collide_store_at<L, S, M, PHYS>(v, f, m, fout, n, 0u);
}

// ---------------------------------------------------------------- two nodes per thread
// Lattice tile {z, t} with bx threads covering 2 bx nodes of a row: thread tx owns
// the aligned pair (x, x+1), x = x0 + 2 tx. One vector load per plane fetches the
// pair at x of the plane's source row (y - c_iy, z - c_iz). A plane with c_ix = +1
// needs (x-1, x), and x-1 is the upper element of the previous lane's pair. A plane
// with c_ix = -1 needs (x+1, x+2), and x+2 is the lower element of the next lane's
// pair. Lanes at the ends of the warp, and nodes whose source leaves [0, nx) (the
// x wrap, with its shear), take one scalar load per such plane instead. All loads
// are issued before any value is used, since a shuffle waits for its load. Both
// nodes are then relaxed as in lattice_tile. A pair whose two nodes are fluid is
// stored with one vector store per plane. A non-fluid node next to a fluid one
// stores into the planes whose slot takes no written-ahead value (View::amask),
// so that the sector is written whole; with such a value in the pair, the pair
// is stored node by node and plane by plane. Not used with BFL, whose record
// lookup assumes one node per lane.
template <typename S> struct Vec2;
template <> struct Vec2<float> {
  using T = float2;
  __device__ static float lo(T v) { return v.x; }
  __device__ static float hi(T v) { return v.y; }
  __device__ static T make(float a, float b) { return make_float2(a, b); }
};
template <> struct Vec2<__half> {  // in the units of the stored values (Units<__half>)
  using T = __half2;
  __device__ static float lo(T v) { return __low2float(v); }
  __device__ static float hi(T v) { return __high2float(v); }
  __device__ static T make(float a, float b) { return __floats2half2_rn(a, b); }
};
template <> struct Vec2<__nv_bfloat16> {
  using T = __nv_bfloat162;
  __device__ static float lo(T v) { return __low2float(v); }
  __device__ static float hi(T v) { return __high2float(v); }
  __device__ static T make(float a, float b) { return __floats2bfloat162_rn(a, b); }
};

template <class L, typename S, typename M, int PHYS>
__device__ __forceinline__ void lattice_tile_pair(const View &v, const S *__restrict__ fin,
                                                  S *__restrict__ fout, int2 tile) {
  using V = Vec2<S>;
  using T = typename V::T;
  const int lane = threadIdx.x & 31;
  const int2 tc = tile_coords(v, tile.y);
  const int x = tc.x * (2 * blockDim.x) + 2 * threadIdx.x;
  const int y = tc.y * blockDim.y + threadIdx.y;
  const int z = tile.x;
  if (y >= v.ny) return;  // uniform across the warp
  const int n = (z * v.ny + y) * v.nxp + x;
  const uint16_t fl2 = *reinterpret_cast<const uint16_t *>(v.flags + n);
  const uint8_t fla = (uint8_t)(fl2 & 0xff), flb = (uint8_t)(fl2 >> 8);
  const bool fa = (fla & K_LATTICE_MASK) == K_FLUID, fb = (flb & K_LATTICE_MASK) == K_FLUID;
  const uint32_t fbal = __ballot_sync(0xffffffffu, (fla & 3) == K_FLUID || (flb & 3) == K_FLUID);
  if (!fbal) return;  // the whole warp is idle
  // stores: the nodes relaxed here, and non-fluid nodes that complete a sector
  // with a fluid node (every plane that takes no written-ahead value)
  const bool ga = fills_sector<S>(fla, fbal, 2), gb = fills_sector<S>(flb, fbal, 2);
  const bool sa = fa || ga, sb = fb || gb;
  // offsets of the 9 (dy, dz) source rows, without the x wrap
  const int plane = v.nxp * v.ny;
  int ro[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      int yy = y + b - 1, zz = z + c - 1;
      yy = yy < 0 ? yy + v.ny : (yy >= v.ny ? yy - v.ny : yy);
      zz = zz < 0 ? zz + v.nz : (zz >= v.nz ? zz - v.nz : zz);
      ro[b][c] = (zz - z) * plane + (yy - y) * v.nxp;
    }
  const int np = (int)v.np;
  T p[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    p[i] = LD_POP2(T, v, fin, fin + (v.soff[i] + n + ro[1 - L::cy(i)][1 - L::cz(i)]));
  // the element per x-shifted plane that the neighbouring lanes cannot supply:
  // c_ix = +1: x-1 at lane 0 (wrapping when x = 0); c_ix = -1: x+1 when it leaves
  // the row (node x+1 is then padding), else x+2 at lane 31 or when it wraps
  // Away from the row ends that element sits in the pair's own source row, one
  // before or two after the pair; only a warp holding a row end takes the
  // periodic (and sheared) wrap.
  const bool wa = x + 1 >= v.nx;
  const bool need_up = lane == 0, need_dn = wa || lane == 31 || x + 2 >= v.nx;
  M e[L::Q];
  if (__any_sync(0xffffffffu, x == 0 || x + 2 >= v.nx)) {
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const int cx = L::cx(i);
      e[i] = M(0);
      if (cx > 0 && need_up)
        e[i] = Units<S>::template load<M>(
            LD_POP(v, fin, fin + (long long)i * np + n + upstream_offset(v, x, y, z, cx, L::cy(i), L::cz(i))));
      if (cx < 0 && need_dn) {
        const int off = wa ? upstream_offset(v, x, y, z, cx, L::cy(i), L::cz(i))
                           : 1 + upstream_offset(v, x + 1, y, z, cx, L::cy(i), L::cz(i));
        e[i] = Units<S>::template load<M>(LD_POP(v, fin, fin + (long long)i * np + n + off));
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const int cx = L::cx(i);
      const S *row = fin + (v.soff[i] + n + ro[1 - L::cy(i)][1 - L::cz(i)]);
      e[i] = M(0);
      if (cx > 0 && need_up) e[i] = Units<S>::template load<M>(LD_POP(v, fin, row - 1));
      if (cx < 0 && need_dn) e[i] = Units<S>::template load<M>(LD_POP(v, fin, row + 2));
    }
  }
  M f0[L::Q], f1[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int cx = L::cx(i);
    if (cx == 0) {
      f0[i] = V::lo(p[i]);
      f1[i] = V::hi(p[i]);
    } else if (cx > 0) {  // sources x-1, x
      const M prev = __shfl_up_sync(0xffffffffu, V::hi(p[i]), 1);
      f0[i] = need_up ? e[i] : prev;
      f1[i] = V::lo(p[i]);
    } else {  // sources x+1, x+2
      const M next = __shfl_down_sync(0xffffffffu, V::lo(p[i]), 1);
      f0[i] = wa ? e[i] : V::hi(p[i]);
      f1[i] = need_dn && !wa ? e[i] : next;
    }
  }
  // every lane relaxes both nodes (a non-fluid node's values are never read), so
  // that only the stores of pairs with a non-fluid node diverge
  constexpr bool U = Units<S>::kStored;
  const Macro<L, M> ma = moments<L, M, U>(v, f0), mb = moments<L, M, U>(v, f1);
  M pa[L::Q], pb[L::Q];
  post_all<L, M, PHYS, U>(v, f0, ma, pa);
  post_all<L, M, PHYS, U>(v, f1, mb, pb);
  if (fa && fb) {
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      ST_POP2(v, fout, fout + (v.soff[i] + n), V::make(pa[i], pb[i]));
  } else if (sa || sb) {
    const uint32_t ka = ga ? v.amask[n] : (fa ? 0u : ~0u), kb = gb ? v.amask[n + 1] : (fb ? 0u : ~0u);
    if (!(ka | kb)) {
#pragma unroll
      for (int i = 0; i < L::Q; ++i)
        ST_POP2(v, fout, fout + (v.soff[i] + n), V::make(pa[i], pb[i]));
    } else {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        if (!((ka >> i) & 1u)) ST_POP(v, fout, &fout[(long long)i * np + n], Units<S>::template store<M>(pa[i]));
        if (!((kb >> i) & 1u)) ST_POP(v, fout, &fout[(long long)i * np + n + 1], Units<S>::template store<M>(pb[i]));
      }
    }
  }
}

// Boundary tile: one thread per boundary record. {-1 - count, first} takes static
// records first .. first+count-1. {DYN_TILE, first} takes the moving body's
// records first .. first+blocksize-1 that exist in this step (their number is
// in device memory).
constexpr int DYN_TILE = -(1 << 20);
template <class L, typename S, typename M>
__device__ __forceinline__ void boundary_tile(const View &v, const S *__restrict__ fin,
                                              S *__restrict__ fout, int2 tile, M *stage) {
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const bool dyn = tile.x == DYN_TILE;
  // signed arithmetic throughout: tiles past the moving body's record count get a
  // negative count and do nothing
  const int tpb = (int)(blockDim.x * blockDim.y);
  const int count = dyn ? min(tpb, *v.dyn_count - tile.y) : -1 - tile.x;
  if (t >= count) return;
  const RecSet rs = dyn ? v.dyn : v.stat();
  const int rid = tile.y + t;
  const Rec r = rs.rec[rid];
  const int n = (int)rs.rnode[rid];
  const int3 c = node_coords(v, n);
  boundary_node<L, S, M>(v, rs, r, fin, fout, n, c.x, c.y, c.z, stage + t, stage_threads<L, M>());
}

// Block b takes table entries b*T .. b*T+T-1 (T = v.tpb_tiles <= 4), whose
// descriptors it loads together up front. MAXT: the largest block the register
// budget is set for (MINB resident blocks of MAXT threads).
template <class L, typename S, typename M, int MINB, int PHYS, bool PAIR = false, int MAXT = 256>
__global__ void __launch_bounds__(MAXT, MINB) k_step(const __grid_constant__ View v, const S *__restrict__ fin,
                                                     S *__restrict__ fout) {
  __shared__ M stage[L::Q * stage_threads<L, M>()];  // boundary tiles: populations, [direction][thread]
  const int T = v.tpb_tiles;
  const int first = blockIdx.x * T;
  int2 tl[4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (k < T && first + k < v.ntiles) tl[k] = v.tiles[first + k];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k >= T || first + k >= v.ntiles) break;
    if (tl[k].x < 0) boundary_tile<L, S, M>(v, fin, fout, tl[k], stage);
    else if constexpr (PAIR) lattice_tile_pair<L, S, M, PHYS>(v, fin, fout, tl[k]);
    else lattice_tile<L, S, M, PHYS>(v, fin, fout, tl[k]);
  }
}

// ---------------------------------------------------------------- split step
// The same step as two kernels that run side by side (launch variants 9 and 10):
// k_lattice takes the lattice tiles of the table v.tiles (no boundary entries),
// k_boundary the boundary tiles of v.btiles, one entry per block. Both only read
// fin and write disjoint slots of fout, so they need no ordering within a step;
// the host forks the boundary kernel onto a second stream and joins it before
// the next step. The point is the register budget: the boundary tiles' link
// loop needs about 64 registers a thread, the lattice tiles alone 40 (no body
// force) or 48 (with one) without spilling, so the lattice kernel keeps 48 or
// 40 warps per SM resident instead of the combined kernel's 32.
template <class L, typename S, typename M, int MINB, int PHYS>
__global__ void __launch_bounds__(256, MINB) k_lattice(const __grid_constant__ View v, const S *__restrict__ fin,
                                                       S *__restrict__ fout) {
  const int T = v.tpb_tiles;
  const int first = blockIdx.x * T;
  int2 tl[4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (k < T && first + k < v.ntiles) tl[k] = v.tiles[first + k];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k >= T || first + k >= v.ntiles) break;
    lattice_tile<L, S, M, PHYS>(v, fin, fout, tl[k]);
  }
}

template <class L, typename S, typename M>
__global__ void __launch_bounds__(256, 4) k_boundary(const __grid_constant__ View v, const S *__restrict__ fin,
                                                     S *__restrict__ fout) {
  __shared__ M stage[L::Q * stage_threads<L, M>()];  // populations, [direction][thread]
  boundary_tile<L, S, M>(v, fin, fout, v.btiles[blockIdx.x], stage);
}

// ---------------------------------------------------------------- TMA-staged step
// A persistent variant of k_step for FP32/FP16/BF16 storage. Each block walks
// the tile table with a grid stride. For a lattice tile, one producer thread
// copies every source row the tile needs into a shared-memory stage with bulk
// asynchronous copies (cp.async.bulk, completion counted on an mbarrier):
//  - for each population plane i and tile row h, the row y0 + h - c_iy of plane
//    z - c_iz (rows wrap in y and z), over x0 - HALO .. x0 + W + HALO, where
//    HALO is one 16-byte chunk, clipped to the padded row;
//  - the tile's flag rows.
// The producer runs nstage - 1 entries ahead (nstage <= 16: the stage parities
// are kept in one word), so the loads in flight are bounded by shared memory, not
// by registers. Consumers read f_i(x) = stage[i][row][x - c_ix]
// and take a direct (wrapped) load only when x - c_ix leaves [0, nx). Boundary
// tiles run as in k_step, staging in the entry's shared slot. Every mbarrier
// wait is bounded: if it runs out, the block sets bit 0 of *v.err, waits (again
// bounded) for its copies in flight, and leaves.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

constexpr long long kWaitLimit = 1LL << 24;  // try_wait polls before a wait counts as hung

// Bounded wait on one mbarrier phase: at most `limit` polls. Returns false if the
// limit ran out (limit 0 returns false at once).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
  for (long long k = 0; k < limit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <typename S>
struct TmaLayout {
  static constexpr int HALO = 16 / (int)sizeof(S);  // elements in one 16-byte chunk
  int W, H, rowlen;                                 // rowlen = W + 2 HALO
  __device__ __forceinline__ TmaLayout(int w, int h) : W(w), H(h), rowlen(w + 2 * HALO) {}
  template <class L>
  __device__ __forceinline__ int pops_bytes() const { return L::Q * H * rowlen * (int)sizeof(S); }
};

// Producer: copies of lattice tile `tile` into stage buffer `base`, armed on `bar`.
// Called by all 32 lanes of warp 0: lane 0 arms the barrier with the byte count,
// then the lanes share the row copies (rows of the Q planes, then the flag rows).
template <class L, typename S>
__device__ void tma_issue(const View &v, const S *__restrict__ fin, int2 tile, unsigned char *base,
                          uint64_t *bar, const TmaLayout<S> &lay, int lane) {
  constexpr int HALO = TmaLayout<S>::HALO;
  const int W = lay.W, H = lay.H;
  const int2 tc = tile_coords(v, tile.y);
  const int z = tile.x, x0 = tc.x * W, y0 = tc.y * H;
  const int xa = max(x0 - HALO, 0), xb = min(x0 + W + HALO, v.nxp);
  const int rows = min(H, v.ny - y0);
  const uint32_t rowbytes = (uint32_t)((xb - xa) * (int)sizeof(S));
  if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)L::Q * rows * rowbytes + (uint32_t)rows * W);
  __syncwarp();
  S *pops = reinterpret_cast<S *>(base);
  unsigned char *fl = base + lay.template pops_bytes<L>();
  const long long plane = (long long)v.nxp * v.ny;
  const int ncopy = (L::Q + 1) * rows;
  for (int c = lane; c < ncopy; c += 32) {
    const int i = c / rows, h = c - i * rows;
    if (i == L::Q) {
      bulk_g2s(fl + h * W, v.flags + (z * (long long)v.ny + y0 + h) * v.nxp + x0, (uint32_t)W, bar);
    } else {
      int zs = z - dcz<L>(i);
      zs = zs < 0 ? zs + v.nz : (zs >= v.nz ? zs - v.nz : zs);
      int ys = y0 + h - dcy<L>(i);
      ys = ys < 0 ? ys + v.ny : (ys >= v.ny ? ys - v.ny : ys);
      long long first = (long long)i * v.np + zs * plane + (long long)ys * v.nxp + xa;
      // a range outside the buffer is recorded, and the copy then reads the
      // buffer's start instead, so that the stage's byte count still completes
      if (!pop_index_ok(v, first, __LINE__) ||
          !pop_index_ok(v, first + rowbytes / (uint32_t)sizeof(S) - 1, __LINE__))
        first = 0;
      const S *src = fin + first;
      S *dst = pops + ((long long)i * H + h) * lay.rowlen + (xa - (x0 - HALO));
      bulk_g2s(dst, src, rowbytes, bar);
    }
  }
}

// Consumer: one node per thread from the stage.
template <class L, typename S, typename M, int PHYS>
__device__ __forceinline__ void tma_lattice(const View &v, const S *__restrict__ fin, S *__restrict__ fout,
                                            int2 tile, const unsigned char *base, const TmaLayout<S> &lay) {
  constexpr int HALO = TmaLayout<S>::HALO;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int2 tc = tile_coords(v, tile.y);
  const int x = tc.x * lay.W + tx;
  const int y = tc.y * lay.H + ty;
  const int z = tile.x;
  if (y >= v.ny) return;  // uniform across the warp
  const int n = (z * v.ny + y) * v.nxp + x;
  const uint8_t fl = base[lay.template pops_bytes<L>() + ty * lay.W + tx];
  const uint32_t fbal = __ballot_sync(0xffffffffu, (fl & 3) == K_FLUID);
  if (!fbal) return;
  uint32_t bal = 0;
  if (v.bc == BC_BFL) bal = __ballot_sync(0xffffffffu, fl & F_BOUNDARY);
  const bool here = (fl & K_LATTICE_MASK) == K_FLUID;
  const bool fill = fills_sector<S>(fl, fbal, 1);  // as in lattice_tile
  const bool masked = __any_sync(0xffffffffu, fill);
  if (!here && !fill) return;
  const S *pops = reinterpret_cast<const S *>(base);
  const bool xedge = x == 0 || x >= v.nx - 1;
  const int np = (int)v.np;
  M f[L::Q];
  uint32_t skip = 0;
  if (!here) {
    skip = v.amask[n];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) f[i] = M(0);
  } else if (!xedge) {
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      f[i] = Units<S>::template load<M>(pops[(i * lay.H + ty) * lay.rowlen + tx + HALO - L::cx(i)]);
  } else {
    Nbr nb;
    nb.init(v, x, y, z);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      f[i] = L::cx(i) == 0 ? Units<S>::template load<M>(pops[(i * lay.H + ty) * lay.rowlen + tx + HALO])
                           : Units<S>::template load<M>(LD_POP(v, fin, fin + (long long)i * v.np + n +
                                                                  nb.at(-L::cx(i), -L::cy(i), -L::cz(i))));
  }
  if (here && v.bc == BC_BFL && (fl & F_BOUNDARY)) bfl_complete<L, M>(v, *record_of(v, n, bal), f);
  const Macro<L, M> m = moments<L, M, Units<S>::kStored>(v, f);
  if (masked) collide_store<L, S, M, PHYS>(v, f, m, fout, n, np, skip);
  else collide_store<L, S, M, PHYS>(v, f, m, fout, n, np, 0u);
}

template <class L, typename S, typename M, int PHYS>
__global__ void __launch_bounds__(256, 2) k_step_tma(const __grid_constant__ View v, const S *__restrict__ fin,
                                                     S *__restrict__ fout, int nstage, int stage_bytes) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  unsigned char *stages = smem + 128;
  const TmaLayout<S> lay(blockDim.x, blockDim.y);
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int G = gridDim.x;
  if (t == 0) {
    for (int k = 0; k < nstage; ++k) mbar_init(&bars[k], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t armed = 0;  // (warp 0) bit k: stage k has copies in flight that nobody has waited for
  if (t < 32)
    for (int j = 0; j < nstage - 1; ++j) {
      const int e = blockIdx.x + j * G;
      if (e >= v.ntiles) break;
      const int2 tl = v.tiles[e];
      if (tl.x >= 0) {
        tma_issue<L, S>(v, fin, tl, stages + j * stage_bytes, &bars[j], lay, t);
        armed |= 1u << j;
      }
    }
  uint32_t parity = 0;  // bit k: parity of the next wait on stage k
  for (int j = 0;; ++j) {
    const int e = blockIdx.x + j * G;
    if (e >= v.ntiles) break;  // uniform across the block
    const int k = j % nstage;
    if (t < 32) {
      const int en = e + (nstage - 1) * G;
      const int kn = (j + nstage - 1) % nstage;
      if (en < v.ntiles) {
        const int2 tl = v.tiles[en];
        if (tl.x >= 0) {
          fence_proxy_async_smem();  // order earlier generic accesses of the stage before the copies
          tma_issue<L, S>(v, fin, tl, stages + kn * stage_bytes, &bars[kn], lay, t);
          armed |= 1u << kn;
        }
      }
    }
    const int2 tile = v.tiles[e];
    if (tile.x < 0) {
      boundary_tile<L, S, M>(v, fin, fout, tile, reinterpret_cast<M *>(stages + k * stage_bytes));
    } else {
      const bool ok = mbar_wait_bounded(&bars[k], (parity >> k) & 1u, v.wait_limit);
      if (__syncthreads_or(!ok)) {  // the whole block leaves together
        if (t == 0) {
          atomicOr(v.err, 1);
          // drain: the copies this block issued and nobody waited for complete
          // before it leaves (they target its shared memory); only armed stages
          // are waited on, each with the full limit
          for (int q = 0; q < nstage; ++q)
            if ((armed >> q) & 1u) mbar_wait_bounded(&bars[q], (parity >> q) & 1u, kWaitLimit);
        }
        return;
      }
      parity ^= 1u << k;
      armed &= ~(1u << k);
      tma_lattice<L, S, M, PHYS>(v, fin, fout, tile, stages + k * stage_bytes, lay);
    }
    __syncthreads();  // the stage is free for the producer
  }
}

// ---------------------------------------------------------------- batched step
// Many independent simulations advance in one launch. Entry k holds the view
// and the two population buffers of simulation k. The tile table lists
// {sim, z, t, 0} lattice tiles and {sim, -1, first, count} boundary tiles, one
// simulation after another, each plane-interleaved as in k_step. parity picks
// which buffer of each entry is read in this step. A block copies the entry of
// its tile into shared memory. The table is grouped by physics class (body
// force, collision operator), and one launch covers one class, compiled for it
// (PHYS) as k_step is. The per-node code is the same as k_step's, so a batched
// simulation gives exactly the results it gives when stepped alone.
struct alignas(16) BatchEntry {
  View v;
  const void *f0;  // read on even batch steps
  void *f1;        // read on odd batch steps
};

template <class L, typename S, typename M, int MINB, int PHYS>
__global__ void __launch_bounds__(256, MINB) k_step_batch(const BatchEntry *__restrict__ entries,
                                                          const int4 *__restrict__ tiles, int ntiles,
                                                          int T, int parity) {
  __shared__ M stage[L::Q * stage_threads<L, M>()];
  __shared__ BatchEntry se;
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  int held = -1;  // the entry in se; a block's tiles mostly belong to one simulation
  for (int k = 0; k < T; ++k) {
    const int idx = blockIdx.x * T + k;
    if (idx >= ntiles) break;  // uniform across the block
    const int4 tile = tiles[idx];
    if (tile.x != held) {  // uniform across the block
      __syncthreads();  // the previous tile is done with se
      {  // the first warp copies the entry in 16-byte pieces
        constexpr int kPieces = (int)(sizeof(BatchEntry) / 16);
        const int4 *src = reinterpret_cast<const int4 *>(entries + tile.x);
        int4 *dst = reinterpret_cast<int4 *>(&se);
        if (t < 32)
          for (int k = t; k < kPieces; k += 32) dst[k] = __ldg(src + k);
      }
      __syncthreads();
      held = tile.x;
    }
    const S *fin = static_cast<const S *>(parity ? se.f1 : se.f0);
    S *fout = static_cast<S *>(parity ? const_cast<void *>(se.f0) : se.f1);
    // each simulation takes the same compiled path as when it steps alone: the
    // launch covers the simulations of one physics class (PHYS) only
    if (tile.y < 0) boundary_tile<L, S, M>(se.v, fin, fout, make_int2(-1 - tile.w, tile.z), stage);
    else lattice_tile<L, S, M, PHYS>(se.v, fin, fout, make_int2(tile.y, tile.z));
  }
}

// ---------------------------------------------------------------- state set-up and read-out
// f_i(x) = f^eq_i(rho, u) on every fluid node, written to the slot its gather reads.
template <class L, typename S, typename M>
__global__ void k_init(const View v, S *__restrict__ fout, double rho, double ux, double uy,
                       double uz) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (y >= v.ny) return;
  const long long n = ((long long)z * v.ny + y) * v.nxp + x;
  const uint8_t fl = v.flags[n];
  const uint32_t bal = __ballot_sync(0xffffffffu, fl & F_BOUNDARY);
  if ((fl & 3) != K_FLUID) return;
  Nbr nb;
  nb.init(v, x, y, z);
  const M usq = M(ux * ux + uy * uy + uz * uz);
  M f[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) f[i] = feq_s<L, M>(i, M(rho - v.rho0), M(rho), M(ux), M(uy), M(uz), usq);
  if ((fl & F_BOUNDARY) && v.bc == BC_BFL) bfl_encode<L, M>(v, *record_of(v, n, bal), f);
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    ST_POP(v, fout, &fout[(long long)i * v.np + n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))], to_store<S, M>(f[i]));
}

// Host-layout FP64 populations fh[(x + nx*(y + ny*z))*Q + i] -> slots (unshifted in, shifted stored).
template <class L, typename S, typename M>
__global__ void k_set_pop(const View v, S *__restrict__ fout, const double *__restrict__ fh) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (y >= v.ny) return;
  const long long n = ((long long)z * v.ny + y) * v.nxp + x;
  const uint8_t fl = v.flags[n];
  const uint32_t bal = __ballot_sync(0xffffffffu, fl & F_BOUNDARY);
  if ((fl & 3) != K_FLUID) return;  // also every padding node (x >= nx)
  const long long hn = ((long long)z * v.ny + y) * v.nx + x;
  Nbr nb;
  nb.init(v, x, y, z);
  M f[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) f[i] = M(fh[hn * L::Q + i] - weight<L>(i) * v.rho0);
  if ((fl & F_BOUNDARY) && v.bc == BC_BFL) bfl_encode<L, M>(v, *record_of(v, n, bal), f);
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    ST_POP(v, fout, &fout[(long long)i * v.np + n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))], to_store<S, M>(f[i]));
}

// Pre-collision populations (gathered, BFL-completed), macroscopic fields, and the
// per-block FP64 partial of the mass. Any output pointer may be null.
template <class L, typename S, typename M>
__global__ void __launch_bounds__(256) k_read(const View v, const S *__restrict__ fin,
                                              double *__restrict__ fh, double *__restrict__ rho_out,
                                              double *__restrict__ u_out, double *__restrict__ mass_part) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  double mloc = 0.0;
  if (y < v.ny) {
    const long long n = ((long long)z * v.ny + y) * v.nxp + x;
    const uint8_t fl = v.flags[n];
    const uint32_t bal = __ballot_sync(0xffffffffu, fl & F_BOUNDARY);
    const long long hn = ((long long)z * v.ny + y) * v.nx + x;
    if ((fl & 3) == K_FLUID) {
      Nbr nb;
      nb.init(v, x, y, z);
      M f[L::Q];
      gather<L, S, M>(v, fin, n, nb, f);
      if ((fl & F_BOUNDARY) && v.bc == BC_BFL) bfl_complete<L, M>(v, *record_of(v, n, bal), f);
      double d = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const double fi = (double)f[i];
        d += fi;
        jx += L::cx(i) * fi;
        jy += L::cy(i) * fi;
        jz += L::cz(i) * fi;
        if (fh) fh[hn * L::Q + i] = fi + weight<L>(i) * v.rho0;
      }
      const double r = v.rho0 + d;
      mloc = r;
      if (rho_out) rho_out[hn] = r;
      if (u_out) {
        const double hx = v.has_force ? 0.5 * v.F[0] : 0.0, hy = v.has_force ? 0.5 * v.F[1] : 0.0,
                     hz = v.has_force ? 0.5 * v.F[2] : 0.0;
        u_out[hn * 3 + 0] = (jx + hx) / r;
        u_out[hn * 3 + 1] = (jy + hy) / r;
        u_out[hn * 3 + 2] = (jz + hz) / r;
      }
    } else if (x < v.nx) {
      if (fh)
        for (int i = 0; i < L::Q; ++i) fh[hn * L::Q + i] = 0.0;
      if (rho_out) rho_out[hn] = 0.0;
      if (u_out) u_out[hn * 3] = u_out[hn * 3 + 1] = u_out[hn * 3 + 2] = 0.0;
    }
  }
  if (mass_part) {
    // fixed-order block sum: warp shuffles, then warp 0 over the warp sums
    __shared__ double sm[32];
    for (int o = 16; o > 0; o >>= 1) mloc += __shfl_down_sync(0xffffffffu, mloc, o);
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y) >> 5;
    if ((t & 31) == 0) sm[t >> 5] = mloc;
    __syncthreads();
    if (t < 32) {
      double s = t < nw ? sm[t] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (t == 0)
        mass_part[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
    }
  }
}

// Momentum-exchange force (Sec. II.F, Eq. force-boundary-node) of the last step,
// one thread per boundary record of the set rs (nrec records, or *nrec_dev when
// that is not null), links of one tag (tag < 0: all). It reads the buffer just
// written: f*_ibar(x_F, t) from the node's own slot and f_i(x_F, t+1) from the
// written-ahead slot (BFL-completed). Writes a per-block FP64 partial (3 doubles).
// Links on the inner side of a thin shell (tag TAG_INNER) carry no force. On its
// outer side the node's own slot ibar holds the value written ahead from the
// other side, so f*_ibar(x_F, t) is computed again from the state at t, prev.
// With tpart non-null the kernel also writes the per-block partial of the torque
// about (cx, cy, cz), sum (x_W - c) x F_link with x_W = x_F - q c_i the link's wall
// point (3 doubles).
template <class L, typename S, typename M>
__global__ void __launch_bounds__(256) k_force(const View v, const S *__restrict__ cur,
                                               const S *__restrict__ prev, RecSet rs,
                                               long long nrec, const int *nrec_dev, int tag,
                                               double *__restrict__ part, double *__restrict__ tpart,
                                               double cx, double cy, double cz) {
  const long long rid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (nrec_dev) nrec = *nrec_dev;
  double fx = 0.0, fy = 0.0, fz = 0.0, tx = 0.0, ty = 0.0, tz = 0.0;
  if (rid < nrec) {
    const Rec r = rs.rec[rid];
    const long long n = rs.rnode[rid];
    const int x = (int)(n % v.nxp);
    const int y = (int)((n / v.nxp) % v.ny);
    const int z = (int)(n / ((long long)v.nxp * v.ny));
    Nbr nb;
    nb.init(v, x, y, z);
    const M *lq = static_cast<const M *>(rs.lq);
    const M *luw = static_cast<const M *>(rs.luw);
    M fp[L::Q];
    Macro<L, M> mp = {};
    if (r.shell && prev) {
      gather<L, S, M>(v, prev, n, nb, fp);
      if (v.bc == BC_BFL) bfl_complete<L, M>(v, r, fp);
      mp = moments<L, M>(v, fp);
    }
    const Par<M> P(v);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const uint32_t bit = 1u << i;
      if (!(r.cut & bit)) continue;
      const uint32_t li = r.link0 + __popc(r.cut & (bit - 1u));
      const uint8_t lt = rs.ltag[li];
      if (lt == TAG_INNER || (tag >= 0 && lt != tag)) continue;
      const int ib = opp<L>(i);
      const double w = weight<L>(i);
      const M fpost_m = (r.shell & bit) ? (prev ? post_r<L, M>(v, P, ib, fp[ib], fp[i], mp) : M(0))
                                        : to_math<S, M>(LD_POP(v, cur, &cur[(long long)ib * v.np + n]));
      const double fpost_ib = (double)fpost_m + w * v.rho0;
      double fnew = (double)to_math<S, M>(LD_POP(v, cur, &cur[(long long)i * v.np + n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))]));
      if (v.bc == BC_BFL && (r.ffok & bit)) {
        const M q = lq[li];
        if (q < M(0.5))
          fnew += (double)((M(1) - M(2) * q) *
                           to_math<S, M>(cur[(long long)ib * v.np + n + nb.at(L::cx(i), L::cy(i), L::cz(i))]));
      }
      fnew += w * v.rho0;
      double wx = 0.0, wy = 0.0, wz = 0.0;
      if (luw) { wx = (double)luw[3 * li]; wy = (double)luw[3 * li + 1]; wz = (double)luw[3 * li + 2]; }
      const double gx = (-L::cx(i) - wx) * fpost_ib - (L::cx(i) - wx) * fnew;
      const double gy = (-L::cy(i) - wy) * fpost_ib - (L::cy(i) - wy) * fnew;
      const double gz = (-L::cz(i) - wz) * fpost_ib - (L::cz(i) - wz) * fnew;
      fx += gx;
      fy += gy;
      fz += gz;
      if (tpart) {
        const double q = (double)lq[li];
        const double rx = x - q * L::cx(i) - cx, ry = y - q * L::cy(i) - cy,
                     rz = L::D == 3 ? z - q * L::cz(i) - cz : 0.0;
        tx += ry * gz - rz * gy;
        ty += rz * gx - rx * gz;
        tz += rx * gy - ry * gx;
      }
    }
  }
  __shared__ double sm[6][8];
  for (int o = 16; o > 0; o >>= 1) {
    fx += __shfl_down_sync(0xffffffffu, fx, o);
    fy += __shfl_down_sync(0xffffffffu, fy, o);
    fz += __shfl_down_sync(0xffffffffu, fz, o);
    tx += __shfl_down_sync(0xffffffffu, tx, o);
    ty += __shfl_down_sync(0xffffffffu, ty, o);
    tz += __shfl_down_sync(0xffffffffu, tz, o);
  }
  const int t = threadIdx.x;
  if ((t & 31) == 0) {
    sm[0][t >> 5] = fx; sm[1][t >> 5] = fy; sm[2][t >> 5] = fz;
    sm[3][t >> 5] = tx; sm[4][t >> 5] = ty; sm[5][t >> 5] = tz;
  }
  __syncthreads();
  if (t < 6) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sm[t][k];
    if (t < 3) part[(long long)blockIdx.x * 3 + t] = s;
    else if (tpart) tpart[(long long)blockIdx.x * 3 + t - 3] = s;
  }
}

// Fixed-order sum of per-block partials: out[c] = sum_b part[b*ncomp + c]. One block.
__global__ void k_reduce_final(const double *__restrict__ part, long long nblocks, int ncomp,
                               double *__restrict__ out);

}  // namespace lbm
