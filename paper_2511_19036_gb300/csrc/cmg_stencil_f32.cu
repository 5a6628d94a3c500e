// FP32 V-cycle kernels (sm_103a): the smoothing sweep (weighted Jacobi, or a
// red-black Gauss-Seidel half-sweep) and the restriction of the compact cycle
// with binary32 arithmetic, inside the exact
// iterative refinement (the precision split of Table 1: the cycle needs only
// progressive(+m, b4) precision, the fmgResidual progressive(+p+m+1, b3)).
//
// Every operation of the cycle rounds to nearest binary32 in one fixed order,
// with no fused multiply-add (explicit __f*_rn intrinsics):
//   F   = fl(y + z) with z = P_l w_(l-1) = fl(fl(w_a + w_b) / 2) (or a copy)
//   S   = fl(fl(...fl(fl((2d) F_p) - F_-x) - F_+x ... - F_+z) * h^(d-2))
//   y'  = fl(y + fl(c fl(rc - S)))        (stored as RNE into the BFP section)
//   w_l = fl(y'_stored + z)               (binary32 temporary for level l + 1)
//   d   = fl(rc - S)                      (restriction input; R_l d is exact)
// The stored sections (y~, rc, u~) keep their BFP format; the correction of u~
// and u^_l = u~_l + P_l u^_(l-1) stay exact (int64), as in the exact kernels.
// Binary32 rounding never produces bits below the grid of its inputs, so the
// restriction's integer scatter of d on the exact path's grid stays exact.
//
// The tile, prefetch and ring machinery is that of cmg_stencil.cu with
// binary32 operands (half the registers and shared memory per value).
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

struct SmemF {
  float Fs[2][PLANE];        // in-plane operand, double-buffered
  float ring[4 * CRX];       // coarse ring of w_(l-1) (binary32)
  long long ringu[4 * CRX];  // coarse ring of u^_(l-1) (exact, grid G1u)
};

// one ring entry per thread of a binary32 coarse temporary
struct StagerF {
  bool on, ok;
  int cj, ci;
  float v;
};

__device__ __forceinline__ StagerF make_stager_f(const Geo &gc, const Tile &T, int tid) {
  StagerF s;
  s.on = tid < CRX;
  const int r = tid / CX, x = tid - (tid / CX) * CX;
  const int cj = T.cr0 + r, ci = T.cx0 + x;
  s.ok = s.on && (unsigned)ci < (unsigned)gc.n && (unsigned)cj < (unsigned)gc.n;
  s.cj = s.ok ? cj : 0;
  s.ci = s.ok ? ci : 0;
  s.v = 0.0f;
  return s;
}

__device__ __forceinline__ void stage_load_f(StagerF &s, const float *w, const Geo &gc, int c) {
  s.v = 0.0f;
  if (s.ok && (unsigned)c < (unsigned)gc.nz) s.v = __ldg(w + (long long)(c * gc.n + s.cj) * gc.R + s.ci);
}

__device__ __forceinline__ void stage_store_f(const StagerF &s, float *ring, int c, int tid) {
  if (s.on) ring[(c & 3) * CRX + tid] = s.v;
}

// z = P_l w at a slot: the copy for a single parent, else fl(fl(a + b) / 2)
__device__ __forceinline__ float ring_pf(const float *ring, const Slot &s, int za, int zb) {
  const float a = ring[(za & 3) * CRX + s.oa];
  if (s.oa == s.ob && za == zb) return a;
  return __fmul_rn(__fadd_rn(a, ring[(zb & 3) * CRX + s.ob]), 0.5f);
}

struct MarchF {
  Sec s;        // y~ (if has_s)
  bool has_s;
  const float *w;  // w_(l-1) (if has_z)
  bool has_z;
  Tmp u;        // u^_(l-1) ring (if has_u)
  bool has_u;
  int G1u;
  float c2d, hscale;  // 2d and h^(d-2)
  float cjac;         // Poisson: the Jacobi factor c_l
  // diffusion: nodal k on the finest grid (boundary included, kN^dim), read at
  // stride 2^(Lmax - l); the Jacobi factor is omega / D_p per node
  const float *kfield;
  int kN, kstride;
  float omega_f;
};

// The binary32 z-march: as march() in cmg_stencil.cu, with
// body.out(k, S, y, F, z, Pu, c) at every plane k (S, y, F, z binary32 at the
// thread's node; Pu = (P_l u^)(node) exact on grid G1u - 1; c the Jacobi
// factor at the node).  COEF selects the diffusion operator: for the
// neighbours -x, +x, -y, +y, -z, +z, kf = fl(fl(k_q + k_p) * 0.5),
// acc = fl(acc + fl(kf fl(F_p - F_q))), dsum = fl(dsum + kf); S = fl(acc h^(d-2)),
// D = fl(dsum h^(d-2)), c = fl(omega / D) (nodes outside the level get S = c = 0).
template <int DIM, bool COEF, class Body>
__device__ __forceinline__ void march_f32(const Geo &g, const Geo &gc, const Tile &T, const MarchF &in, SmemF &sm,
                                          Body &body, bool &bad) {
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
  StagerF stw = make_stager_f(gc, T, tid);
  Stager stu = make_stager(gc, T, tid);
  auto raw_at = [&](const Slot &sl, int kf) -> Raw {
    return raw_load(in.s, kf * pb + sl.bip, sl.cp, in.has_s && sl.ok && (unsigned)kf < (unsigned)g.nz);
  };
  // operand at a slot: F = fl(y + z) (y alone without z); y and z returned too
  auto F_at = [&](const Slot &sl, const Raw &r, int kf, float &y, float &z) -> float {
    y = in.has_s ? raw_f32(r, sl.cp.boff, Ws, bad) : 0.0f;
    z = 0.0f;
    if (!in.has_z) return y;
    int za, zb;
    zparents<DIM>(kf, za, zb);
    z = ring_pf(sm.ring, sl, za, zb);
    return in.has_s ? __fadd_rn(y, z) : z;
  };
  auto pu_at = [&](int kf) -> long long {
    if (!in.has_u) return 0;
    int za, zb;
    zparents<DIM>(kf, za, zb);
    return ring_p(sm.ringu, own, za, zb);
  };
  auto kat = [&](int I, int J, int K) -> float {
    return __ldg(in.kfield + ((long long)(DIM == 3 ? K * in.kstride : 0) * in.kN + J * in.kstride) * in.kN +
                 I * in.kstride);
  };
  auto stencil = [&](const float *P, float Fm, float F0, float Fp, int k, float &cp) -> float {
    if constexpr (COEF) {
      cp = 0.0f;
      if (!own.ok) return 0.0f;
      const int I = T.x0 + lane + 1, J = T.j0 + ty + 1, K = k + 1;
      const float kp = kat(I, J, K);
      const float nb[6] = {P[own.sm - 1], P[own.sm + 1], P[own.sm - PW], P[own.sm + PW], Fm, Fp};
      float acc = 0.0f, dsum = 0.0f;
#pragma unroll
      for (int e = 0; e < 2 * DIM; e++) {
        const int Iq = I + (e == 0 ? -1 : e == 1 ? 1 : 0), Jq = J + (e == 2 ? -1 : e == 3 ? 1 : 0);
        const int Kq = K + (e == 4 ? -1 : e == 5 ? 1 : 0);
        const float kf = __fmul_rn(__fadd_rn(kat(Iq, Jq, Kq), kp), 0.5f);
        acc = __fadd_rn(acc, __fmul_rn(kf, __fsub_rn(F0, nb[e])));
        dsum = __fadd_rn(dsum, kf);
      }
      cp = __fdiv_rn(in.omega_f, __fmul_rn(dsum, in.hscale));
      return __fmul_rn(acc, in.hscale);
    }
    cp = in.cjac;
    float acc = __fmul_rn(in.c2d, F0);
    acc = __fsub_rn(acc, P[own.sm - 1]);
    acc = __fsub_rn(acc, P[own.sm + 1]);
    acc = __fsub_rn(acc, P[own.sm - PW]);
    acc = __fsub_rn(acc, P[own.sm + PW]);
    if (DIM == 3) {
      acc = __fsub_rn(acc, Fm);
      acc = __fsub_rn(acc, Fp);
    }
    return __fmul_rn(acc, in.hscale);
  };
  auto stage = [&](int c, bool load) {
    if (load) {
      if (in.has_z) stage_load_f(stw, in.w, gc, c);
      if (in.has_u) stage_load(stu, in.u, gc, c);
    } else {
      if (in.has_z) stage_store_f(stw, sm.ring, c, tid);
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
    float y0, z0, yh, zh;
    const float F0 = F_at(own, r0, 0, y0, z0);
    sm.Fs[0][own.sm] = F0;
    if (has_h) sm.Fs[0][hal.sm] = F_at(hal, h0, 0, yh, zh);
    __syncthreads();
    float cp;
    const float S = stencil(sm.Fs[0], 0.0f, F0, 0.0f, 0, cp);
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
  float yx, zx, y0, z0;
  float Fm = F_at(own, rm, T.k0 - 1, yx, zx);
  float F0 = F_at(own, r0, T.k0, y0, z0);
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
    float yp, zp;
    const float Fp = F_at(own, rn, k + 1, yp, zp);
    if (k + 1 < T.k1) {
      float *nxt = sm.Fs[(k + 1) & 1];
      nxt[own.sm] = Fp;
      if (has_h) nxt[hal.sm] = F_at(hal, hn, k + 1, yx, zx);
    }
    float cp;
    const float S = stencil(sm.Fs[k & 1], Fm, F0, Fp, k, cp);
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

template <int DIM, int M>
struct SweepBodyF {
  const SweepArgs &a;
  const Geo &g;
  float c_f;
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

  __device__ __forceinline__ void out(int k, float S, float y, float F0, float z, long long Pu, float cp) {
    if (!rowok) return;  // warp-uniform: one warp per row
    const int blk = k * g.n * g.nbx + bip;
    // y' = fl(y + fl(c fl(rc - S))); padding lanes carry 0; a node left out by a
    // half-sweep keeps y
    float ynew = 0.0f;
    if (pt) {
      if (upd(k)) {
        const float rc = raw_f32(rc_c, cprc.boff, a.rc.W, bad);
        ynew = __fadd_rn(y, __fmul_rn(cp, __fsub_rn(rc, S)));
      } else {
        ynew = y;
      }
    }
    int Gy;
    const long long vy = f32_block_to_grid(ynew, Gy, bad);
    int e, sh;
    const int q = encode_block(vy, Gy, a.Wy, e, sh, a.err);
    const long long yr = rounded_value(vy, q, sh);
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
    if (WW()) {  // w_l = fl(y~'_stored + z), binary32; the stored value is q 2^(e - W + 1)
      const float ys = code_f32(q, e, a.Wy, bad);
      if (pt) a.w_out_f[p] = __fadd_rn(ys, z);
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

template <int DIM, int M, bool COEF>
__global__ void __launch_bounds__(NT, CMG_SWEEP_F32_MINB) k_sweep_f32(SweepArgs a) {
  using F = SfF<M>;
  const bool has_y = F::fixed ? F::y : (bool)a.has_y, has_z = F::fixed ? F::z : (bool)a.has_z;
  const bool write_y = F::fixed ? F::wy : (bool)a.write_y, corr = F::fixed ? F::corr : (bool)a.corr;
  const bool write_uh = F::fixed ? F::uh : (bool)a.write_uh;
  __shared__ SmemF sm;
  __shared__ uint32_t pk[TY][33];
  __shared__ int smy[2], smu[2], smb[6];
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const Tile T = make_tile(g);
  if (tid == 0) smy[0] = smy[1] = smu[0] = smu[1] = 0;
  const bool uring_wanted = write_uh && a.has_uhc;
  Bounds bs, bt, bu;
  footprint_bounds<DIM>(g, a.gc, T, a.y_in, false, a.uhc, false, a.uhc, uring_wanted, smb, bs, bt, bu);
  SweepBodyF<DIM, M> b{a, g};
  b.c_f = __fmul_rn((float)a.c_num, __int_as_float((a.c_exp + 127) << 23));
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
  MarchF in;
  in.s = a.y_in;
  in.has_s = has_y;
  in.w = a.wc_f;
  in.has_z = has_z;
  in.u = a.uhc;
  in.has_u = b.ring_u;
  in.G1u = b.G1u;
  in.c2d = (float)(2 * DIM);
  in.hscale = __int_as_float((127 - (DIM - 2) * g.l) << 23);
  in.cjac = b.c_f;
  in.kfield = a.kfield;
  in.kN = a.kN;
  in.kstride = a.kstride;
  in.omega_f = a.omega;
  march_f32<DIM, COEF>(g, a.gc, T, in, sm, b, b.bad);
  ovf_flush(b.ovf, a.err, 111);
  ovf_flush(b.bad, a.err, 112);
  if (write_y) meta_flush(b.my, a.y_out.meta, smy);
  if (corr) meta_flush(b.mu, a.u_out.meta, smu);
}

// ------------------------------------------------------------------ restriction
template <int DIM>
struct RestrictBodyF {
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

  __device__ __forceinline__ void out(int k, float S, float, float, float, long long, float) {
    if (!rowok || !pt) return;
    const float d = __fsub_rn(raw_f32(rc_c, cprc.boff, a.rc.W, bad), S);
    const long long v = f32_on_grid(d, Gd, bad);
    if (v) scatter_restrict<DIM>((unsigned long long *)a.acc.v, a.gc, i + 1, j + 1, k + 1, v);
  }
};

template <int DIM>
__global__ void __launch_bounds__(NT, 2) k_restrict_f32(RestrictArgs a) {
  __shared__ SmemF sm;
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const Tile T = make_tile(g);
  // the grid of every d = fl(rc - A y): that of the exact d (binary32 rounding
  // keeps its result on the grid of its inputs); the accumulator holds R d on Gd - 1
  const int sA = (DIM - 2) * g.l;
  const int Gd = imin(sec_lsb(a.rc), a.has_y ? sec_lsb(a.y) - sA : GRID_NONE);
  if (tid == 0 && first_cta()) a.acc.meta[0] = Gd - 1;
  RestrictBodyF<DIM> b{a, g};
  b.Gd = Gd;
  b.i = T.x0 + lane;
  b.j = T.j0 + ty;
  b.rowok = b.j < g.n;
  b.pt = b.rowok && b.i < g.n;
  b.bip = b.rowok ? b.j * g.nbx + T.bx : 0;
  b.cprc = code_pos(lane, a.rc.W);
  b.ovf = false;
  b.bad = false;
  MarchF in;
  in.s = a.y;
  in.has_s = a.has_y;
  in.w = nullptr;
  in.has_z = false;
  in.u = a.acc;
  in.has_u = false;
  in.G1u = 0;
  in.c2d = (float)(2 * DIM);
  in.hscale = __int_as_float((127 - (DIM - 2) * g.l) << 23);
  in.cjac = 0.0f;
  in.kfield = nullptr;
  march_f32<DIM, false>(g, a.gc, T, in, sm, b, b.bad);
  ovf_flush(b.bad, a.err, 312);
}

// ------------------------------------------------------------------ diffusion restriction
// d = fl(rc - A y~) of the diffusion operator, stored in binary32 on level l
template <int DIM>
struct DBodyF {
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
  __device__ __forceinline__ void out(int k, float S, float, float, float, long long, float) {
    if (!rowok || !pt) return;
    a.d_out[(long long)(k * g.n + j) * g.R + i] = __fsub_rn(raw_f32(rc_c, cprc.boff, a.rc.W, bad), S);
  }
};

template <int DIM>
__global__ void __launch_bounds__(NT, 3) k_dvec_diff(RestrictArgs a) {
  __shared__ SmemF sm;
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y;
  const Tile T = make_tile(g);
  DBodyF<DIM> b{a, g};
  b.i = T.x0 + lane;
  b.j = T.j0 + ty;
  b.rowok = b.j < g.n;
  b.pt = b.rowok && b.i < g.n;
  b.bip = b.rowok ? b.j * g.nbx + T.bx : 0;
  b.cprc = code_pos(lane, a.rc.W);
  b.bad = false;
  MarchF in;
  in.s = a.y;
  in.has_s = a.has_y;
  in.w = nullptr;
  in.has_z = false;
  in.u = a.acc;
  in.has_u = false;
  in.G1u = 0;
  in.c2d = (float)(2 * DIM);
  in.hscale = __int_as_float((127 - (DIM - 2) * g.l) << 23);
  in.cjac = 0.0f;
  in.kfield = a.kfield;
  in.kN = a.kN;
  in.kstride = a.kstride;
  in.omega_f = 1.0f;
  march_f32<DIM, true>(g, a.gc, T, in, sm, b, b.bad);
  ovf_flush(b.bad, a.err, 313);
}

// rc_(l-1) = round(R_l d): per coarse node, in binary32, the fine node 2J plus
// half the sum over the odd sets {x},{y},{x,y},{z},{x,z},{y,z},{x,y,z} of
// d(2J - e_S) then d(2J + e_S); one warp per coarse block row
template <int DIM>
__global__ void __launch_bounds__(NT) k_gather_restrict_f32(GatherArgs a) {
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
    float r = 0.0f;
    if (ci < gc.n) {
      const int I = 2 * (ci + 1), J = 2 * (cj + 1), K = DIM == 3 ? 2 * (ck + 1) : 0;
      auto at = [&](int Ii, int Jj, int Kk) -> float {  // 1-based fine node, zero outside
        if (Ii < 1 || Ii > g.n || Jj < 1 || Jj > g.n) return 0.0f;
        if (DIM == 3 && (Kk < 1 || Kk > g.nz)) return 0.0f;
        const int kk = DIM == 3 ? Kk - 1 : 0;
        return __ldg(a.d + (long long)(kk * g.n + Jj - 1) * g.R + Ii - 1);
      };
      const int ns = DIM == 3 ? 7 : 3;
      const int ox[7] = {1, 0, 1, 0, 1, 0, 1}, oy[7] = {0, 1, 1, 0, 0, 1, 1}, oz[7] = {0, 0, 0, 1, 1, 1, 1};
      float sum = 0.0f;
#pragma unroll
      for (int s = 0; s < ns; s++) {
        sum = __fadd_rn(sum, at(I - ox[s], J - oy[s], K - oz[s]));
        sum = __fadd_rn(sum, at(I + ox[s], J + oy[s], K + oz[s]));
      }
      r = __fadd_rn(at(I, J, K), __fmul_rn(sum, 0.5f));
    }
    int G;
    const long long v = f32_block_to_grid(r, G, bad);
    int e, sh;
    const int q = encode_block(v, G, a.rc_out.W, e, sh, a.err);
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

template <int DIM, bool COEF>
void launch_sweep_f32_dim(const SweepArgs &a, cudaStream_t st) {
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
      k_sweep_f32<DIM, SF_UP0, COEF><<<grid, b, 0, st>>>(a);
      return;
    }
  }
  switch (m) {
    case SF_DOWN: k_sweep_f32<DIM, SF_DOWN, COEF><<<grid, b, 0, st>>>(a); break;
    case SF_UP: k_sweep_f32<DIM, SF_UP, COEF><<<grid, b, 0, st>>>(a); break;
    case SF_UP_CORR: k_sweep_f32<DIM, SF_UP_CORR, COEF><<<grid, b, 0, st>>>(a); break;
    case SF_UP_CORR_UH: k_sweep_f32<DIM, SF_UP_CORR_UH, COEF><<<grid, b, 0, st>>>(a); break;
    case SF_UP_CORR_W_UH: k_sweep_f32<DIM, SF_UP_CORR_W_UH, COEF><<<grid, b, 0, st>>>(a); break;
    default: k_sweep_f32<DIM, SF_GENERIC, COEF><<<grid, b, 0, st>>>(a); break;
  }
}

}  // namespace

void launch_sweep_f32(int dim, const SweepArgs &a, cudaStream_t st) {
  if (a.kfield) {
    if (dim == 3) launch_sweep_f32_dim<3, true>(a, st);
    else launch_sweep_f32_dim<2, true>(a, st);
  } else {
    if (dim == 3) launch_sweep_f32_dim<3, false>(a, st);
    else launch_sweep_f32_dim<2, false>(a, st);
  }
}

void launch_dvec_diffusion(int dim, const RestrictArgs &a, cudaStream_t st) {
  const dim3 grid = stencil_grid_f(a.g), b(32, TY);
  if (dim == 3) k_dvec_diff<3><<<grid, b, 0, st>>>(a);
  else k_dvec_diff<2><<<grid, b, 0, st>>>(a);
}

void launch_gather_restrict_f32(int dim, const GatherArgs &a, cudaStream_t st) {
  const dim3 b(32, TY);
  const unsigned nb = (unsigned)((a.gc.nblocks + TY - 1) / TY);
  if (dim == 3) k_gather_restrict_f32<3><<<nb, b, 0, st>>>(a);
  else k_gather_restrict_f32<2><<<nb, b, 0, st>>>(a);
}

void launch_restrict_f32(int dim, const RestrictArgs &a, cudaStream_t st) {
  const dim3 grid = stencil_grid_f(a.g), b(32, TY);
  if (dim == 3) k_restrict_f32<3><<<grid, b, 0, st>>>(a);
  else k_restrict_f32<2><<<grid, b, 0, st>>>(a);
}

}  // namespace cmg
