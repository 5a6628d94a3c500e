// Floating-point V-cycle kernels (sm_103a): the smoothing sweep (weighted
// Jacobi, or a red-black Gauss-Seidel half-sweep) and the restriction of the
// compact cycle in IEEE binary32 (float) or binary64 (double) arithmetic, inside
// the exact iterative refinement (the precision split of Table 1: the cycle needs
// only progressive(+m, b4) precision, the fmgResidual progressive(+p+m+1, b3)).
// The binary64 instantiation is the plain FP64 form of the same cycle.
//
// Every operation of the cycle rounds to nearest in its type, in one fixed
// order, with no fused multiply-add (explicit round-to-nearest intrinsics):
//   F   = fl(y + z) with z = P_l w_(l-1) = fl(fl(w_a + w_b) / 2) (or a copy)
//   S   = fl(fl(...fl(fl((2d) F_p) - F_-x) - F_+x ... - F_+z) * h^(d-2))
//   y'  = fl(y + fl(c fl(rc - S)))        (stored as RNE into the BFP section)
//   w_l = fl(y'_stored + z)               (temporary of the cycle's type for level l + 1)
//   d   = fl(rc - S)                      (restriction input; R_l d is exact)
// The stored sections (y~, rc, u~) keep their BFP format; the correction of u~
// and u^_l = u~_l + P_l u^_(l-1) stay exact (int64), as in the exact kernels.
// Rounding never produces bits below the grid of its inputs, so the
// restriction's integer scatter of d on the exact path's grid stays exact.
//
// The tile, prefetch and ring machinery is that of cmg_stencil.cu with
// floating-point operands.
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "cmg_device.cuh"
#include "cmg_kernels.h"
#include "cmg_stencil_common.cuh"

namespace cmg {
namespace {

#ifndef CMG_SWEEP_F32_MINB
#define CMG_SWEEP_F32_MINB 3
#endif

// BFP value as binary32: exact unless the value is a nonzero subnormal (flagged,
// as the oracle does)
__device__ __forceinline__ float raw_f32(const Raw &r, int boff, int W, bool &bad) {
  if (r.e == -128) return 0.0f;
  const float q = (float)raw_code(r, boff, W);
  const int k = r.e - W + 1;
  float v;
  if (k >= -126) {
    v = __fmul_rn(q, __int_as_float((k + 127) << 23));
  } else {  // two exact power-of-two steps; the second rounds only into subnormals
    v = __fmul_rn(__fmul_rn(q, __int_as_float((k + 64 + 127) << 23)), __int_as_float((-64 + 127) << 23));
  }
  if (v != 0.0f && fabsf(v) < FLT_MIN) bad = true;
  return v;
}

// rounded BFP value q 2^(e - W + 1) as binary32 (|q| < 2^23, exact when normal)
__device__ __forceinline__ float code_f32(int q, int e, int W, bool &bad) {
  if (e == -128) return 0.0f;
  const float qq = (float)q;
  const int k = e - W + 1;
  float v = k >= -126 ? __fmul_rn(qq, __int_as_float((k + 127) << 23))
                      : __fmul_rn(__fmul_rn(qq, __int_as_float((k + 191) << 23)), __int_as_float(63 << 23));
  if (v != 0.0f && fabsf(v) < FLT_MIN) bad = true;
  return v;
}

// Warp-collective: the binary32 values x of one block as integers v on one grid
// G, chosen 38 bits below the last bit of the largest value; values more than
// 38 bits below it lose bits under 2^G, far below the rounding position of any
// width <= 24, so the block's RNE codes are those of the exact values.
__device__ __forceinline__ long long f32_block_to_grid(float x, int &G, bool &bad) {
  const int bits = __float_as_int(x);
  const int ef = (bits >> 23) & 0xff;
  const int emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)ef);
  if (emax == 255) bad = true;  // infinity or NaN
  G = imax(emax, 1) - 188;      // the largest |x| < 2^(G + 62)
  const long long m = ef ? (long long)((bits & 0x7fffff) | 0x800000) : (long long)(bits & 0x7fffff);
  const int sh = imax(ef, 1) - 150 - G;
  const long long v = sh >= 0 ? (m << (sh & 63)) : (m >> imin(-sh, 63));
  return bits < 0 ? -v : v;
}

// binary32 x exactly as an integer on grid G (x is a multiple of 2^G and
// |x| < 2^(G + 58), else *bad)
__device__ __forceinline__ long long f32_on_grid(float x, int G, bool &bad) {
  const int bits = __float_as_int(x);
  const int ef = (bits >> 23) & 0xff;
  if (x == 0.0f) return 0;
  if (ef == 255) {
    bad = true;
    return 0;
  }
  const long long m = ef ? (long long)((bits & 0x7fffff) | 0x800000) : (long long)(bits & 0x7fffff);
  const int sh = imax(ef, 1) - 150 - G;
  long long v;
  if (sh >= 0) {
    if (sh > 34) bad = true;  // |x| may reach 2^(G + 58)
    v = m << (sh & 63);
  } else {
    const int r = imin(-sh, 63);
    if (m & ((1ll << r) - 1)) bad = true;  // x not on grid G
    v = m >> r;
  }
  return bits < 0 ? -v : v;
}

// 2^k as binary64 (k in the normal range)
__device__ __forceinline__ double pow2_f64(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// binary64 x exactly as an integer on grid G (x is a multiple of 2^G and
// |x| < 2^(G + 58), else *bad)
__device__ __forceinline__ long long f64_on_grid(double x, int G, bool &bad) {
  if (x == 0.0) return 0;
  const long long bits = __double_as_longlong(x);
  const int ef = (int)((bits >> 52) & 0x7ff);
  if (ef == 0x7ff) {
    bad = true;
    return 0;
  }
  const long long m = ef ? ((bits & 0xfffffffffffffll) | (1ll << 52)) : (bits & 0xfffffffffffffll);
  const int sh = imax(ef, 1) - 1075 - G;  // x = m 2^(max(ef, 1) - 1075)
  long long v;
  if (sh >= 0) {
    if (sh > 5) bad = true;  // m < 2^53: |x| may reach 2^(G + 58)
    v = m << imin(sh, 63);
  } else {
    const int r = imin(-sh, 63);
    if (m & ((1ll << r) - 1)) bad = true;  // x not on grid G
    v = m >> r;
  }
  return bits < 0 ? -v : v;
}

// The arithmetic of one cycle type: round-to-nearest operations, BFP values,
// the warp-collective BFP rounding of one block (code q, block exponent e, and
// the rounded value yr on grid Gy) and the exact conversion onto a grid.
template <class R>
struct RT;

template <>
struct RT<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
  static __device__ __forceinline__ float pow2(int k) { return __int_as_float((k + 127) << 23); }
  static __device__ __forceinline__ float raw(const Raw &r, int boff, int W, bool &bad) {
    return raw_f32(r, boff, W, bad);
  }
  static __device__ __forceinline__ float code(int q, int e, int W, bool &bad) { return code_f32(q, e, W, bad); }
  static __device__ __forceinline__ int encode(float x, int W, int &e, long long &yr, int &Gy, bool &bad,
                                               int *err) {
    const long long v = f32_block_to_grid(x, Gy, bad);
    int sh;
    const int q = encode_block(v, Gy, W, e, sh, err);
    yr = rounded_value(v, q, sh);
    return q;
  }
  static __device__ __forceinline__ long long on_grid(float x, int G, bool &bad) { return f32_on_grid(x, G, bad); }
};

template <>
struct RT<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
  static __device__ __forceinline__ double pow2(int k) { return pow2_f64(k); }
  // every BFP value (a code of at most 32 bits, a block exponent in [-127, 127]) is exact
  static __device__ __forceinline__ double raw(const Raw &r, int boff, int W, bool &) {
    if (r.e == -128) return 0.0;
    return __dmul_rn((double)raw_code(r, boff, W), pow2_f64(r.e - W + 1));
  }
  static __device__ __forceinline__ double code(int q, int e, int W, bool &) {
    return e == -128 ? 0.0 : __dmul_rn((double)q, pow2_f64(e - W + 1));
  }
  // RNE of the binary64 values of one block, as the oracle rounds doubles; the
  // rounded value is the code itself on the block grid e - W + 1
  static __device__ __forceinline__ int encode(double x, int W, int &e, long long &yr, int &Gy, bool &,
                                               int *err) {
    const int q = encode_block_f64(x, W, e, err);
    yr = q;
    Gy = e == -128 ? GRID_NONE : e - W + 1;
    return q;
  }
  static __device__ __forceinline__ long long on_grid(double x, int G, bool &bad) { return f64_on_grid(x, G, bad); }
};

template <class R>
struct SmemR {
  R Fs[2][PLANE];            // in-plane operand, double-buffered
  R ring[4 * CRX];           // coarse ring of w_(l-1) (the cycle's type)
  long long ringu[4 * CRX];  // coarse ring of u^_(l-1) (exact, grid G1u)
};

// one ring entry per thread of a floating-point coarse temporary
template <class R>
struct StagerR {
  bool on, ok;
  int cj, ci;
  R v;
};

template <class R>
__device__ __forceinline__ StagerR<R> make_stager_r(const Geo &gc, const Tile &T, int tid) {
  StagerR<R> s;
  s.on = tid < CRX;
  const int r = tid / CX, x = tid - (tid / CX) * CX;
  const int cj = T.cr0 + r, ci = T.cx0 + x;
  s.ok = s.on && (unsigned)ci < (unsigned)gc.n && (unsigned)cj < (unsigned)gc.n;
  s.cj = s.ok ? cj : 0;
  s.ci = s.ok ? ci : 0;
  s.v = (R)0;
  return s;
}

template <class R>
__device__ __forceinline__ void stage_load_r(StagerR<R> &s, const R *w, const Geo &gc, int c) {
  s.v = (R)0;
  if (s.ok && (unsigned)c < (unsigned)gc.nz) s.v = __ldg(w + (long long)(c * gc.n + s.cj) * gc.R + s.ci);
}

template <class R>
__device__ __forceinline__ void stage_store_r(const StagerR<R> &s, R *ring, int c, int tid) {
  if (s.on) ring[(c & 3) * CRX + tid] = s.v;
}

// z = P_l w at a slot: the copy for a single parent, else fl(fl(a + b) / 2)
template <class R>
__device__ __forceinline__ R ring_pr(const R *ring, const Slot &s, int za, int zb) {
  const R a = ring[(za & 3) * CRX + s.oa];
  if (s.oa == s.ob && za == zb) return a;
  return RT<R>::mul(RT<R>::add(a, ring[(zb & 3) * CRX + s.ob]), (R)0.5);
}

template <class R>
struct MarchR {
  Sec s;        // y~ (if has_s)
  bool has_s;
  const R *w;   // w_(l-1) (if has_z)
  bool has_z;
  Tmp u;        // u^_(l-1) ring (if has_u)
  bool has_u;
  int G1u;
  R c2d, hscale;  // 2d and h^(d-2)
  R cjac;         // Poisson: the Jacobi factor c_l
  // diffusion: nodal binary32 k on the finest grid (boundary included, kN^dim),
  // read at stride 2^(Lmax - l); the Jacobi factor is omega / D_p per node
  const float *kfield;
  int kN, kstride;
  R omega;
};

// The floating-point z-march: as march() in cmg_stencil.cu, with
// body.out(k, S, y, F, z, Pu, c) at every plane k (S, y, F, z of type R at the
// thread's node; Pu = (P_l u^)(node) exact on grid G1u - 1; c the Jacobi
// factor at the node).  COEF selects the diffusion operator: for the
// neighbours -x, +x, -y, +y, -z, +z, kf = fl(fl(k_q + k_p) * 0.5),
// acc = fl(acc + fl(kf fl(F_p - F_q))), dsum = fl(dsum + kf); S = fl(acc h^(d-2)),
// D = fl(dsum h^(d-2)), c = fl(omega / D) (nodes outside the level get S = c = 0).
template <class R, int DIM, bool COEF, class Body>
__device__ __forceinline__ void march_fp(const Geo &g, const Geo &gc, const Tile &T, const MarchR<R> &in,
                                         SmemR<R> &sm, Body &body, bool &bad) {
  using O = RT<R>;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const int Ws = in.has_s ? in.s.W : 1;
  const Slot own = make_slot(g, Ws, T.x0 + lane, T.j0 + ty, ty + 1, lane + 1, T);
  const bool has_h = tid < NHALO;
  Slot hal;
  {
    int i, j, r, x;
    if (tid < 32) {
      i = T.x0 + tid, j = T.j0 - 1, r = 0, x = tid + 1;
    } else if (tid < 64) {
      i = T.x0 + tid - 32, j = T.j0 + TY, r = TY + 1, x = tid - 31;
    } else {
      const int c = imin(tid - 64, 2 * (TY + 2) - 1);
      r = c >> 1, j = T.j0 - 1 + r;
      x = (c & 1) ? 33 : 0;
      i = (c & 1) ? T.x0 + 32 : T.x0 - 1;
    }
    hal = make_slot(g, Ws, i, j, r, x, T);
  }
  const int pb = g.n * g.nbx;
  const bool rings = in.has_z || in.has_u;
  StagerR<R> stw = make_stager_r<R>(gc, T, tid);
  Stager stu = make_stager(gc, T, tid);
  auto raw_at = [&](const Slot &sl, int kf) -> Raw {
    return raw_load(in.s, kf * pb + sl.bip, sl.cp, in.has_s && sl.ok && (unsigned)kf < (unsigned)g.nz);
  };
  // operand at a slot: F = fl(y + z) (y alone without z); y and z returned too
  auto F_at = [&](const Slot &sl, const Raw &r, int kf, R &y, R &z) -> R {
    y = in.has_s ? O::raw(r, sl.cp.boff, Ws, bad) : (R)0;
    z = (R)0;
    if (!in.has_z) return y;
    int za, zb;
    zparents<DIM>(kf, za, zb);
    z = ring_pr(sm.ring, sl, za, zb);
    return in.has_s ? O::add(y, z) : z;
  };
  auto pu_at = [&](int kf) -> long long {
    if (!in.has_u) return 0;
    int za, zb;
    zparents<DIM>(kf, za, zb);
    return ring_p(sm.ringu, own, za, zb);
  };
  auto kat = [&](int I, int J, int K) -> R {
    return (R)__ldg(in.kfield + ((long long)(DIM == 3 ? K * in.kstride : 0) * in.kN + J * in.kstride) * in.kN +
                 I * in.kstride);
  };
  auto stencil = [&](const R *P, R Fm, R F0, R Fp, int k, R &cp) -> R {
    if constexpr (COEF) {
      cp = (R)0;
      if (!own.ok) return (R)0;
      const int I = T.x0 + lane + 1, J = T.j0 + ty + 1, K = k + 1;
      const R kp = kat(I, J, K);
      const R nb[6] = {P[own.sm - 1], P[own.sm + 1], P[own.sm - PW], P[own.sm + PW], Fm, Fp};
      R acc = (R)0, dsum = (R)0;
#pragma unroll
      for (int e = 0; e < 2 * DIM; e++) {
        const int Iq = I + (e == 0 ? -1 : e == 1 ? 1 : 0), Jq = J + (e == 2 ? -1 : e == 3 ? 1 : 0);
        const int Kq = K + (e == 4 ? -1 : e == 5 ? 1 : 0);
        const R kf = O::mul(O::add(kat(Iq, Jq, Kq), kp), (R)0.5);
        acc = O::add(acc, O::mul(kf, O::sub(F0, nb[e])));
        dsum = O::add(dsum, kf);
      }
      cp = O::div(in.omega, O::mul(dsum, in.hscale));
      return O::mul(acc, in.hscale);
    }
    cp = in.cjac;
    R acc = O::mul(in.c2d, F0);
    acc = O::sub(acc, P[own.sm - 1]);
    acc = O::sub(acc, P[own.sm + 1]);
    acc = O::sub(acc, P[own.sm - PW]);
    acc = O::sub(acc, P[own.sm + PW]);
    if (DIM == 3) {
      acc = O::sub(acc, Fm);
      acc = O::sub(acc, Fp);
    }
    return O::mul(acc, in.hscale);
  };
  auto stage = [&](int c, bool load) {
    if (load) {
      if (in.has_z) stage_load_r(stw, in.w, gc, c);
      if (in.has_u) stage_load(stu, in.u, gc, c);
    } else {
      if (in.has_z) stage_store_r(stw, sm.ring, c, tid);
      if (in.has_u) stage_store(stu, sm.ringu, c, in.G1u, tid);
    }
  };

  if (DIM == 2) {
    if (rings) {
      stage(0, true);
      stage(0, false);
    }
    body.prefetch(0);
    const Raw r0 = raw_at(own, 0);
    Raw h0 = r0;
    if (has_h) h0 = raw_at(hal, 0);
    __syncthreads();
    R y0, z0, yh, zh;
    const R F0 = F_at(own, r0, 0, y0, z0);
    sm.Fs[0][own.sm] = F0;
    if (has_h) sm.Fs[0][hal.sm] = F_at(hal, h0, 0, yh, zh);
    __syncthreads();
    R cp;
    const R S = stencil(sm.Fs[0], (R)0, F0, (R)0, 0, cp);
    body.advance();
    body.out(0, S, y0, F0, z0, pu_at(0), cp);
    return;
  }

  int staged_hi = -2;
  if (rings) {
    for (int c = (T.k0 - 2) >> 1; c <= (T.k0 >> 1); c++) {
      stage(c, true);
      stage(c, false);
    }
    staged_hi = T.k0 >> 1;
  }
  const Raw rm = raw_at(own, T.k0 - 1);
  const Raw r0 = raw_at(own, T.k0);
  Raw h0 = rm, hn = rm;
  if (has_h) h0 = raw_at(hal, T.k0);
  Raw rn = raw_at(own, T.k0 + 1);
  if (has_h) hn = raw_at(hal, T.k0 + 1);
  body.prefetch(T.k0);
  __syncthreads();
  R yx, zx, y0, z0;
  R Fm = F_at(own, rm, T.k0 - 1, yx, zx);
  R F0 = F_at(own, r0, T.k0, y0, z0);
  sm.Fs[T.k0 & 1][own.sm] = F0;
  if (has_h) sm.Fs[T.k0 & 1][hal.sm] = F_at(hal, h0, T.k0, yx, zx);

  for (int k = T.k0; k < T.k1; k++) {
    const int cs = (k + 2) >> 1;
    const bool stg = rings && cs > staged_hi && cs <= gc.nz;
    if (stg) stage(cs, true);
    body.advance();
    if (k + 1 < T.k1) body.prefetch(k + 1);
    Raw rn2 = rm, hn2 = rm;
    if (k + 2 <= T.k1) rn2 = raw_at(own, k + 2);
    if (has_h && k + 2 < T.k1) hn2 = raw_at(hal, k + 2);
    __syncthreads();  // plane k complete in Fs[k & 1]; ring planes for k + 1 staged
    R yp, zp;
    const R Fp = F_at(own, rn, k + 1, yp, zp);
    if (k + 1 < T.k1) {
      R *nxt = sm.Fs[(k + 1) & 1];
      nxt[own.sm] = Fp;
      if (has_h) nxt[hal.sm] = F_at(hal, hn, k + 1, yx, zx);
    }
    R cp;
    const R S = stencil(sm.Fs[k & 1], Fm, F0, Fp, k, cp);
    body.out(k, S, y0, F0, z0, pu_at(k), cp);
    if (stg) {
      stage(cs, false);
      staged_hi = cs;
    }
    Fm = F0;
    F0 = Fp;
    y0 = yp;
    z0 = zp;
    rn = rn2;
    hn = hn2;
  }
}

// ------------------------------------------------------------------ sweep
enum SweepModeF {
  SF_GENERIC = 0,
  SF_DOWN,          // y~' = round(fl(y + c (rc - A y)))
  SF_UP,            // operand fl(y~ + z)
  SF_UP_CORR,       // last up-sweep on the finest level: u~ += y~'
  SF_UP_CORR_UH,    // ... and u^_l
  SF_UP_CORR_W_UH,  // below the finest level: u~ += y~', w_l, u^_l
  SF_UP0,           // first up-sweep from y~ = 0 (red half-sweep of V(0,1)): operand z
};

template <int M>
struct SfF {
  static constexpr bool fixed = M != SF_GENERIC;
  static constexpr bool y = M != SF_UP0;
  static constexpr bool z = M >= SF_UP;
  static constexpr bool wy = M == SF_DOWN || M == SF_UP || M == SF_UP0;
  static constexpr bool corr = M >= SF_UP_CORR && M <= SF_UP_CORR_W_UH;
  static constexpr bool uh = M == SF_UP_CORR_UH || M == SF_UP_CORR_W_UH;
  static constexpr bool w = M == SF_UP_CORR_W_UH;
};

template <class R, int DIM, int M>
struct SweepBodyR {
  using O = RT<R>;
  const SweepArgs &a;
  const Geo &g;
  R c_f;
  bool ring_u;
  int G1u, Mu;
  int bip, lane, i, j;
  bool rowok, pt;
  CodePos cprc, cpu;
  Raw rc_n, u_n, rc_c, u_c;
  bool ovf, bad;
  MetaAcc my, mu;
  uint32_t *pk;

  __device__ __forceinline__ bool HY() const { return SfF<M>::fixed ? SfF<M>::y : (bool)a.has_y; }
  __device__ __forceinline__ bool HZ() const { return SfF<M>::fixed ? SfF<M>::z : (bool)a.has_z; }
  __device__ __forceinline__ bool WY() const { return SfF<M>::fixed ? SfF<M>::wy : (bool)a.write_y; }
  __device__ __forceinline__ bool CORR() const { return SfF<M>::fixed ? SfF<M>::corr : (bool)a.corr; }
  __device__ __forceinline__ bool WW() const { return SfF<M>::fixed ? SfF<M>::w : (bool)a.write_w; }
  __device__ __forceinline__ bool WUH() const { return SfF<M>::fixed ? SfF<M>::uh : (bool)a.write_uh; }
  // red-black half-sweep: is node (i, j, k) updated?  red: 1-based I + J [+ K] even
  __device__ __forceinline__ bool upd(int k) const {
    return a.rb == 0 || (((i + j + (DIM == 3 ? k + 1 : 0)) ^ (a.rb - 1)) & 1) == 0;
  }

  __device__ __forceinline__ void prefetch(int k) {
    if (!rowok) return;
    const int blk = k * g.n * g.nbx + bip;
    rc_n = raw_load(a.rc, blk, cprc, true);
    if (CORR()) u_n = raw_load(a.u_in, blk, cpu, true);
  }
  __device__ __forceinline__ void advance() {
    rc_c = rc_n;
    u_c = u_n;
  }

  __device__ __forceinline__ void out(int k, R S, R y, R F0, R z, long long Pu, R cp) {
    if (!rowok) return;  // warp-uniform: one warp per row
    const int blk = k * g.n * g.nbx + bip;
    // y' = fl(y + fl(c fl(rc - S))); padding lanes carry 0; a node left out by a
    // half-sweep keeps y
    R ynew = (R)0;
    if (pt) {
      if (upd(k)) {
        const R rc = O::raw(rc_c, cprc.boff, a.rc.W, bad);
        ynew = O::add(y, O::mul(cp, O::sub(rc, S)));
      } else {
        ynew = y;
      }
    }
    int Gy, e;
    long long yr;
    const int q = O::encode(ynew, a.Wy, e, yr, Gy, bad, a.err);
    if (WY()) {
      pack_block(q, a.Wy, pk, a.y_out.words + (long long)blk * a.Wy);
      if (lane == 0) {
        a.y_out.exps[blk] = (int8_t)e;
        my.add(e);
      }
    }
    long long ur = 0;
    int Gu = Gy, eu = -128;
    if (CORR()) {  // exact: u~ <- round(u~ + y~'), as in the exact sweep
      // y~' on its own block grid e - W + 1 (exact: the rounding left only
      // multiples of it), not on the much finer conversion grid Gy
      const int gY = e == -128 ? Gy : imax(e - a.Wy + 1, Gy);
      const int eu0 = u_c.e;
      Gu = imin(blk_lsb(eu0, a.u_in.W), gY);
      if (e != -128 || eu0 != -128)
        if (imax(eu0 == -128 ? MAG_NONE : eu0, e) + 1 - Gu > 62) ovf = true;
      const long long usum = raw_val(u_c, cpu.boff, a.u_in.W, Gu) + regrid(regrid(yr, Gy, gY), gY, Gu);
      int su;
      const int qu = encode_block(usum, Gu, a.u_out.W, eu, su, a.err);
      ur = rounded_value(usum, qu, su);
      pack_block(qu, a.u_out.W, pk, a.u_out.words + (long long)blk * a.u_out.W);
      if (lane == 0) {
        a.u_out.exps[blk] = (int8_t)eu;
        mu.add(eu);
      }
    }
    const long long p = (long long)(k * g.n + j) * g.R + i;
    if (WW()) {  // w_l = fl(y~'_stored + z) in R; the stored value is q 2^(e - W + 1)
      const R ys = O::code(q, e, a.Wy, bad);
      if (pt) ((R *)a.w_out_r)[p] = O::add(ys, z);
    }
    if (WUH()) {  // u^_l = u~_l' + P u^_(l-1), exact
      if (ring_u || !a.has_uhc) {
        const int gU = eu == -128 ? GRID_NONE : imax(eu - a.u_out.W + 1, Gu);
        const int gP = a.has_uhc ? G1u - 1 : GRID_NONE;
        const int gu = imin(gU, gP);
        long long uh = 0;
        if (gu < GRID_NONE / 2) {
          const long long pu = (a.has_uhc && pt) ? Pu : 0;
          if (imax(eu == -128 ? MAG_NONE : eu, a.has_uhc ? Mu : MAG_NONE) + 1 - gu <= 62) {
            uh = regrid(ur, Gu, gu) + regrid(pu, gP, gu);
          } else {
            uh = (gu >= Gu ? regrid(ur, Gu, gu) : shl_ck(ur, Gu - gu, ovf)) +
                 (gu >= gP ? regrid(pu, gP, gu) : shl_ck(pu, gP - gu, ovf));
            ck62(uh, ovf);
          }
        }
        store_tmp_on(uh, gu, a.uh_out.v + p, a.uh_out.gb + blk, pt, ovf);
      } else {
        const int gu = pt ? prolong_grid<DIM>(a.uhc, a.gc, i + 1, j + 1, k + 1) : GRID_NONE;
        const int Guh = imin(Gu, __reduce_min_sync(0xffffffffu, gu));
        long long uh = shl_ck(ur, Gu - Guh, ovf);
        if (pt) uh += prolong_tmp<DIM>(a.uhc, a.gc, i + 1, j + 1, k + 1, Guh, ovf);
        ck62(uh, ovf);
        store_tmp_block(uh, Guh, a.uh_out.v + p, a.uh_out.gb + blk, pt, ovf);
      }
    }
  }
};

template <class R, int DIM, int M, bool COEF>
__global__ void __launch_bounds__(NT, CMG_SWEEP_F32_MINB) k_sweep_fp(SweepArgs a) {
  using F = SfF<M>;
  const bool has_y = F::fixed ? F::y : (bool)a.has_y, has_z = F::fixed ? F::z : (bool)a.has_z;
  const bool write_y = F::fixed ? F::wy : (bool)a.write_y, corr = F::fixed ? F::corr : (bool)a.corr;
  const bool write_uh = F::fixed ? F::uh : (bool)a.write_uh;
  __shared__ SmemR<R> sm;
  __shared__ uint32_t pk[TY][33];
  __shared__ int smy[2], smu[2], smb[6];
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const Tile T = make_tile(g);
  if (tid == 0) smy[0] = smy[1] = smu[0] = smu[1] = 0;
  const bool uring_wanted = write_uh && a.has_uhc;
  Bounds bs, bt, bu;
  footprint_bounds<DIM>(g, a.gc, T, a.y_in, false, a.uhc, false, a.uhc, uring_wanted, smb, bs, bt, bu);
  SweepBodyR<R, DIM, M> b{a, g};
  b.c_f = RT<R>::mul((R)a.c_num, RT<R>::pow2(a.c_exp));
  b.ring_u = uring_wanted && (bu.G >= GRID_NONE / 2 || bu.M - bu.G <= 61);
  b.G1u = bu.G < GRID_NONE / 2 ? bu.G : 0;
  b.Mu = bu.M;
  b.lane = lane;
  b.i = T.x0 + lane;
  b.j = T.j0 + ty;
  b.rowok = b.j < g.n;
  b.pt = b.rowok && b.i < g.n;
  b.bip = b.rowok ? b.j * g.nbx + T.bx : 0;
  b.cprc = code_pos(lane, a.rc.W);
  b.cpu = code_pos(lane, corr ? a.u_in.W : 1);
  b.ovf = false;
  b.bad = false;
  b.my.init();
  b.mu.init();
  b.pk = pk[ty];
  MarchR<R> in;
  in.s = a.y_in;
  in.has_s = has_y;
  in.w = (const R *)a.wc_r;
  in.has_z = has_z;
  in.u = a.uhc;
  in.has_u = b.ring_u;
  in.G1u = b.G1u;
  in.c2d = (R)(2 * DIM);
  in.hscale = RT<R>::pow2(-(DIM - 2) * g.l);
  in.cjac = b.c_f;
  in.kfield = a.kfield;
  in.kN = a.kN;
  in.kstride = a.kstride;
  in.omega = (R)a.omega;
  march_fp<R, DIM, COEF>(g, a.gc, T, in, sm, b, b.bad);
  ovf_flush(b.ovf, a.err, 111);
  ovf_flush(b.bad, a.err, 112);
  if (write_y) meta_flush(b.my, a.y_out.meta, smy);
  if (corr) meta_flush(b.mu, a.u_out.meta, smu);
}

// ------------------------------------------------------------------ restriction
template <class R, int DIM>
struct RestrictBodyR {
  using O = RT<R>;
  const RestrictArgs &a;
  const Geo &g;
  int Gd;
  int bip, i, j;
  bool rowok, pt;
  CodePos cprc;
  Raw rc_n, rc_c;
  bool ovf, bad;

  __device__ __forceinline__ void prefetch(int k) {
    if (!rowok) return;
    rc_n = raw_load(a.rc, k * g.n * g.nbx + bip, cprc, true);
  }
  __device__ __forceinline__ void advance() { rc_c = rc_n; }

  __device__ __forceinline__ void out(int k, R S, R, R, R, long long, R) {
    if (!rowok || !pt) return;
    const R d = O::sub(O::raw(rc_c, cprc.boff, a.rc.W, bad), S);
    const long long v = O::on_grid(d, Gd, bad);
    if (v) scatter_restrict<DIM>((unsigned long long *)a.acc.v, a.gc, i + 1, j + 1, k + 1, v);
  }
};

template <class R, int DIM>
__global__ void __launch_bounds__(NT, 2) k_restrict_fp(RestrictArgs a) {
  __shared__ SmemR<R> sm;
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const Tile T = make_tile(g);
  // the grid of every d = fl(rc - A y): that of the exact d (rounding keeps its
  // result on the grid of its inputs); the accumulator holds R d on Gd - 1
  const int sA = (DIM - 2) * g.l;
  const int Gd = imin(sec_lsb(a.rc), a.has_y ? sec_lsb(a.y) - sA : GRID_NONE);
  if (tid == 0 && first_cta()) a.acc.meta[0] = Gd - 1;
  RestrictBodyR<R, DIM> b{a, g};
  b.Gd = Gd;
  b.i = T.x0 + lane;
  b.j = T.j0 + ty;
  b.rowok = b.j < g.n;
  b.pt = b.rowok && b.i < g.n;
  b.bip = b.rowok ? b.j * g.nbx + T.bx : 0;
  b.cprc = code_pos(lane, a.rc.W);
  b.ovf = false;
  b.bad = false;
  MarchR<R> in;
  in.s = a.y;
  in.has_s = a.has_y;
  in.w = nullptr;
  in.has_z = false;
  in.u = a.acc;
  in.has_u = false;
  in.G1u = 0;
  in.c2d = (R)(2 * DIM);
  in.hscale = RT<R>::pow2(-(DIM - 2) * g.l);
  in.cjac = (R)0;
  in.kfield = nullptr;
  march_fp<R, DIM, false>(g, a.gc, T, in, sm, b, b.bad);
  ovf_flush(b.bad, a.err, 312);
}

// ------------------------------------------------------------------ diffusion restriction
// d = fl(rc - A y~) of the diffusion operator, stored in the cycle's type on level l
template <class R, int DIM>
struct DBodyR {
  const RestrictArgs &a;
  const Geo &g;
  int bip, i, j;
  bool rowok, pt;
  CodePos cprc;
  Raw rc_n, rc_c;
  bool bad;

  __device__ __forceinline__ void prefetch(int k) {
    if (!rowok) return;
    rc_n = raw_load(a.rc, k * g.n * g.nbx + bip, cprc, true);
  }
  __device__ __forceinline__ void advance() { rc_c = rc_n; }
  __device__ __forceinline__ void out(int k, R S, R, R, R, long long, R) {
    if (!rowok || !pt) return;
    ((R *)a.d_out)[(long long)(k * g.n + j) * g.R + i] = RT<R>::sub(RT<R>::raw(rc_c, cprc.boff, a.rc.W, bad), S);
  }
};

template <class R, int DIM>
__global__ void __launch_bounds__(NT, 3) k_dvec_diff(RestrictArgs a) {
  __shared__ SmemR<R> sm;
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y;
  const Tile T = make_tile(g);
  DBodyR<R, DIM> b{a, g};
  b.i = T.x0 + lane;
  b.j = T.j0 + ty;
  b.rowok = b.j < g.n;
  b.pt = b.rowok && b.i < g.n;
  b.bip = b.rowok ? b.j * g.nbx + T.bx : 0;
  b.cprc = code_pos(lane, a.rc.W);
  b.bad = false;
  MarchR<R> in;
  in.s = a.y;
  in.has_s = a.has_y;
  in.w = nullptr;
  in.has_z = false;
  in.u = a.acc;
  in.has_u = false;
  in.G1u = 0;
  in.c2d = (R)(2 * DIM);
  in.hscale = RT<R>::pow2(-(DIM - 2) * g.l);
  in.cjac = (R)0;
  in.kfield = a.kfield;
  in.kN = a.kN;
  in.kstride = a.kstride;
  in.omega = (R)1;
  march_fp<R, DIM, true>(g, a.gc, T, in, sm, b, b.bad);
  ovf_flush(b.bad, a.err, 313);
}

// rc_(l-1) = round(R_l d): per coarse node, in the cycle's type, the fine node 2J plus
// half the sum over the odd sets {x},{y},{x,y},{z},{x,z},{y,z},{x,y,z} of
// d(2J - e_S) then d(2J + e_S); one warp per coarse block row
template <class R, int DIM>
__global__ void __launch_bounds__(NT) k_gather_restrict_fp(GatherArgs a) {
  using O = RT<R>;
  __shared__ uint32_t pk[TY][33];
  __shared__ int smr[2];
  const Geo gc = a.gc, g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  if (tid == 0) smr[0] = smr[1] = 0;
  __syncthreads();
  bool bad = false;
  MetaAcc mr;
  mr.init();
  const long long blk = (long long)blockIdx.x * TY + ty;
  if (blk < gc.nblocks) {
    const long long row = blk / gc.nbx;
    const int bx = (int)(blk - row * gc.nbx);
    const int ci = bx * 32 + lane;
    const int cj = (int)(row % gc.n), ck = (int)(row / gc.n);
    R r = (R)0;
    if (ci < gc.n) {
      const int I = 2 * (ci + 1), J = 2 * (cj + 1), K = DIM == 3 ? 2 * (ck + 1) : 0;
      auto at = [&](int Ii, int Jj, int Kk) -> R {  // 1-based fine node, zero outside
        if (Ii < 1 || Ii > g.n || Jj < 1 || Jj > g.n) return (R)0;
        if (DIM == 3 && (Kk < 1 || Kk > g.nz)) return (R)0;
        const int kk = DIM == 3 ? Kk - 1 : 0;
        return __ldg((const R *)a.d + (long long)(kk * g.n + Jj - 1) * g.R + Ii - 1);
      };
      const int ns = DIM == 3 ? 7 : 3;
      const int ox[7] = {1, 0, 1, 0, 1, 0, 1}, oy[7] = {0, 1, 1, 0, 0, 1, 1}, oz[7] = {0, 0, 0, 1, 1, 1, 1};
      R sum = (R)0;
#pragma unroll
      for (int s = 0; s < ns; s++) {
        sum = O::add(sum, at(I - ox[s], J - oy[s], K - oz[s]));
        sum = O::add(sum, at(I + ox[s], J + oy[s], K + oz[s]));
      }
      r = O::add(at(I, J, K), O::mul(sum, (R)0.5));
    }
    int G, e;
    long long rr;
    const int q = O::encode(r, a.rc_out.W, e, rr, G, bad, a.err);
    pack_block(q, a.rc_out.W, pk[ty], a.rc_out.words + blk * a.rc_out.W);
    if (lane == 0) {
      a.rc_out.exps[blk] = (int8_t)e;
      mr.add(e);
    }
  }
  ovf_flush(bad, a.err, 314);
  meta_flush(mr, a.rc_out.meta, smr);
}

dim3 stencil_grid_f(const Geo &g) {
  return dim3((unsigned)g.nbx, (unsigned)((g.n + TY - 1) / TY), (unsigned)((g.nz + ZC - 1) / ZC));
}

template <class R, int DIM, bool COEF>
void launch_sweep_fp_dim(const SweepArgs &a, cudaStream_t st) {
  const dim3 grid = stencil_grid_f(a.g), b(32, TY);
  int m = SF_GENERIC;
  if (a.has_y) {
    if (!a.corr && a.write_y && !a.write_w && !a.write_uh) m = a.has_z ? SF_UP : SF_DOWN;
    else if (a.corr && a.has_z && !a.write_y && !a.write_w) m = a.write_uh ? SF_UP_CORR_UH : SF_UP_CORR;
    else if (a.corr && a.has_z && !a.write_y && a.write_w && a.write_uh) m = SF_UP_CORR_W_UH;
  } else if (!COEF && a.has_z && a.write_y && !a.corr && !a.write_w && !a.write_uh) {
    m = SF_UP0;  // red-black smoothing (Poisson only)
  }
  if constexpr (!COEF) {
    if (m == SF_UP0) {
      k_sweep_fp<R, DIM, SF_UP0, COEF><<<grid, b, 0, st>>>(a);
      return;
    }
  }
  switch (m) {
    case SF_DOWN: k_sweep_fp<R, DIM, SF_DOWN, COEF><<<grid, b, 0, st>>>(a); break;
    case SF_UP: k_sweep_fp<R, DIM, SF_UP, COEF><<<grid, b, 0, st>>>(a); break;
    case SF_UP_CORR: k_sweep_fp<R, DIM, SF_UP_CORR, COEF><<<grid, b, 0, st>>>(a); break;
    case SF_UP_CORR_UH: k_sweep_fp<R, DIM, SF_UP_CORR_UH, COEF><<<grid, b, 0, st>>>(a); break;
    case SF_UP_CORR_W_UH: k_sweep_fp<R, DIM, SF_UP_CORR_W_UH, COEF><<<grid, b, 0, st>>>(a); break;
    default: k_sweep_fp<R, DIM, SF_GENERIC, COEF><<<grid, b, 0, st>>>(a); break;
  }
}

template <class R>
void launch_sweep_r(int dim, const SweepArgs &a, cudaStream_t st) {
  if (a.kfield) {
    if (dim == 3) launch_sweep_fp_dim<R, 3, true>(a, st);
    else launch_sweep_fp_dim<R, 2, true>(a, st);
  } else {
    if (dim == 3) launch_sweep_fp_dim<R, 3, false>(a, st);
    else launch_sweep_fp_dim<R, 2, false>(a, st);
  }
}

}  // namespace

void launch_sweep_fp(int dim, bool f64, const SweepArgs &a, cudaStream_t st) {
  if (f64) launch_sweep_r<double>(dim, a, st);
  else launch_sweep_r<float>(dim, a, st);
}

void launch_dvec_diffusion(int dim, bool f64, const RestrictArgs &a, cudaStream_t st) {
  const dim3 grid = stencil_grid_f(a.g), b(32, TY);
  if (f64) {
    if (dim == 3) k_dvec_diff<double, 3><<<grid, b, 0, st>>>(a);
    else k_dvec_diff<double, 2><<<grid, b, 0, st>>>(a);
  } else {
    if (dim == 3) k_dvec_diff<float, 3><<<grid, b, 0, st>>>(a);
    else k_dvec_diff<float, 2><<<grid, b, 0, st>>>(a);
  }
}

void launch_gather_restrict_fp(int dim, bool f64, const GatherArgs &a, cudaStream_t st) {
  const dim3 b(32, TY);
  const unsigned nb = (unsigned)((a.gc.nblocks + TY - 1) / TY);
  if (f64) {
    if (dim == 3) k_gather_restrict_fp<double, 3><<<nb, b, 0, st>>>(a);
    else k_gather_restrict_fp<double, 2><<<nb, b, 0, st>>>(a);
  } else {
    if (dim == 3) k_gather_restrict_fp<float, 3><<<nb, b, 0, st>>>(a);
    else k_gather_restrict_fp<float, 2><<<nb, b, 0, st>>>(a);
  }
}

void launch_restrict_fp(int dim, bool f64, const RestrictArgs &a, cudaStream_t st) {
  const dim3 grid = stencil_grid_f(a.g), b(32, TY);
  if (f64) {
    if (dim == 3) k_restrict_fp<double, 3><<<grid, b, 0, st>>>(a);
    else k_restrict_fp<double, 2><<<grid, b, 0, st>>>(a);
  } else {
    if (dim == 3) k_restrict_fp<float, 3><<<grid, b, 0, st>>>(a);
    else k_restrict_fp<float, 2><<<grid, b, 0, st>>>(a);
  }
}

}  // namespace cmg
