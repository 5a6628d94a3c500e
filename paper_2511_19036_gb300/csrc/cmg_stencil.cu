// Stencil kernels of the compact FMG path for GB300 (sm_103a): the smoothing
// sweep (weighted Jacobi, or one colour's half of a red-black Gauss-Seidel
// sweep), the residual of Algorithm 2 and the restriction R_l = P_l^T.
//
// Tiling.  A CTA of TY warps owns a 32 x TY column tile of a level and marches
// it through up to ZC planes in z.  Thread (lane, ty) owns the column
// (x0 + lane, j0 + ty): it decodes the stencil operand F of that column once
// per plane and keeps the planes k-1, k, k+1 in registers, so only the
// in-plane neighbours go through shared memory (two plane buffers of
// (TY + 2) x 34 values; warps 0-2 also decode the halo).  One CTA barrier per
// plane separates writing plane k+1 from reading plane k.
//
// Latency.  The compact words and block exponents of plane k+2 (operand) and
// k+1 (per-kernel inputs such as r~c or u~) are loaded into registers one plane
// ahead of their use, so that decoding never waits on a global load that was
// issued in the same plane.
//
// Operand F = [BFP section s] + [P_l t] (t an int64 coarse temporary with one
// descriptor per block).  The coarse values P_l needs are staged once per CTA
// and coarse plane in a ring of four planes (7 x 19 values around the tile) on
// one grid, with all-zero planes at both ends of the level, so a fine value of
// P_l t is two shared-memory reads at offsets fixed per thread.  A second ring
// serves P_l u^_(l-1) for the fused u^_l = u~_l + P_l u^_(l-1) of the last
// up-sweep.
//
// Exactness (see cmg_device.cuh): F is converted to the finest grid found in
// the CTA's footprint; each warp picks the grid of its output block; per-value
// overflow checks run only for blocks whose static bounds do not fit.
#include <cuda_runtime.h>

#include <cstdint>

#include "cmg_device.cuh"
#include "cmg_kernels.h"
#include "cmg_stencil_common.cuh"

namespace cmg {
namespace {

constexpr int TMAXP = 8;  // right-hand-side terms with per-thread products in shared memory
// resident CTAs per SM the register allocation is fitted to, per kernel
#ifndef CMG_SWEEP_MINB
#define CMG_SWEEP_MINB 3
#endif
#ifndef CMG_RESID_MINB
#define CMG_RESID_MINB 3
#endif
#ifndef CMG_RESTRICT_MINB
#define CMG_RESTRICT_MINB 2
#endif

// ------------------------------------------------------------------ the z-march
// V: the integer type of the operand (int64, or int32 where the CTA's
// footprint bounds prove |2d F| + |neighbours| < 2^31 on the operand grid)
template <class V>
struct SmemT {
  V Fs[2][PLANE];           // in-plane operand, double-buffered
  V ring[4 * CRX];          // coarse ring of the operand's P_l t
  long long ringu[4 * CRX]; // coarse ring of P_l u^_(l-1)
  Two2 two;                 // staging of a two-level operand temporary
};
using SmemTile = SmemT<long long>;
union SmemAny {  // one shared buffer for either operand width
  SmemT<long long> w64;
  SmemT<int> w32;
};

// the 32-bit march is exact when |S| < 2^(MF + 4) fits: |F| < 2^MF on grid GF
__device__ __forceinline__ bool narrow_operand(int GF, int MF) { return GF < GRID_NONE / 2 && MF + 4 - GF <= 30; }

struct MarchIn {
  Sec s;         // operand section (if has_s)
  Tmp t;         // operand coarse temporary (if has_t)
  Tmp u;         // second ring (if has_u)
  bool has_s, has_t, has_u;
  int GF;        // operand grid
  int G1t, G1u;  // staging grids of the rings
  const Tmp2 *t2 = nullptr;  // the operand temporary held in two levels instead of t
  int *err = nullptr;        // flags of the two-level staging
};

// Calls, for every plane k of the tile in order, body.advance() (what
// body.prefetch(k) loaded becomes current), body.prefetch(k + 1) (loads for
// the next plane) and body.out(k, S, s0, F0, Pu): S = (2d) F - sum of the 2d
// neighbours at the thread's node (grid GF), s0 its section part, F0 its
// operand, Pu the value of P_l u at the node (grid G1u - 1).  Every thread of
// the CTA calls it.  A body with kRaw = true gets body.out_raw(k, Pc, Fm, F0,
// Fp, s0) instead: Pc points at the node in the plane buffer (neighbours
// Pc[-1], Pc[+1], Pc[-PW], Pc[+PW]), Fm / Fp are the z-neighbours.
template <int DIM, class V, class Body>
__device__ __forceinline__ void march(const Geo &g, const Geo &gc, const Tile &T, const MarchIn &in, SmemT<V> &sm,
                                      Body &body) {
  static_assert(sizeof(V) == 8 || !Body::kRaw, "raw bodies read 64-bit plane buffers");
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const int Ws = in.has_s ? in.s.W : 1;
  const Slot own = make_slot(g, Ws, T.x0 + lane, T.j0 + ty, ty + 1, lane + 1, T);
  // halo: warp 0 row j0-1, warp 1 row j0+TY, warp 2 the columns x0-1 and x0+32
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
  const int pb = g.n * g.nbx;  // blocks per plane (block indices fit in int)
  const bool rings = in.has_t || in.has_u;
  Stager st0 = make_stager(gc, T, tid), st1 = st0;
  bool sbad = false;  // two-level staging: an invalid code met
  auto load_t = [&](int c) {
    if (in.t2) two_step_issue(st0, *in.t2, gc, T, c, sm.two, tid);
    else stage_load(st0, in.t, gc, c);
  };
  auto store_t = [&](int c) {
    if (in.t2) two_step_store<DIM>(st0, *in.t2, gc, T, c, sm.two, sm.ring, in.G1t, tid, sbad);
    else stage_store(st0, sm.ring, c, in.G1t, tid);
  };
  auto staging_flush = [&]() {
    if (in.t2) {
      cp_async_wait_all();  // the step issued ahead past the tile's last plane
      corrupt_flush(sbad, in.err);
    }
  };
  const bool has_s = in.has_s;
  auto raw_at = [&](const Slot &sl, int kf) -> Raw {
    return raw_load(in.s, kf * pb + sl.bip, sl.cp, has_s && sl.ok && (unsigned)kf < (unsigned)g.nz);
  };
  auto F_at = [&](const Slot &sl, const Raw &r, int kf, V &sv) -> V {
    sv = has_s ? raw_val_as<V>(r, sl.cp.boff, Ws, in.GF) : 0;
    if (!in.has_t) return sv;
    int za, zb;
    zparents<DIM>(kf, za, zb);
    return sv + ring_p(sm.ring, sl, za, zb);
  };
  auto pu_at = [&](int kf) -> long long {
    if (!in.has_u) return 0;
    int za, zb;
    zparents<DIM>(kf, za, zb);
    return ring_p(sm.ringu, own, za, zb);
  };

  if (DIM == 2) {
    if (rings) {
      if (in.has_t && in.t2) two_prologue<DIM>(st0, *in.t2, gc, T, 0, 0, sm.two, sm.ring, in.G1t, tid, sbad);
      else if (in.has_t) load_t(0);
      if (in.has_u) stage_load(st1, in.u, gc, 0);
      if (in.has_t && !in.t2) store_t(0);
      if (in.has_u) stage_store(st1, sm.ringu, 0, in.G1u, tid);
    }
    body.prefetch(0);
    const Raw r0 = raw_at(own, 0);
    Raw h0 = r0;
    if (has_h) h0 = raw_at(hal, 0);
    __syncthreads();
    V s0, sh;
    const V F0 = F_at(own, r0, 0, s0);
    sm.Fs[0][own.sm] = F0;
    if (has_h) sm.Fs[0][hal.sm] = F_at(hal, h0, 0, sh);
    __syncthreads();
    const V *P = sm.Fs[0];
    body.advance();
    if constexpr (Body::kRaw) {
      body.out_raw(0, P + own.sm, 0, F0, 0, s0);
    } else {
      const V S = 4 * F0 - P[own.sm - 1] - P[own.sm + 1] - P[own.sm - PW] - P[own.sm + PW];
      body.out(0, (long long)S, (long long)s0, (long long)F0, pu_at(0));
    }
    staging_flush();
    return;
  }

  // 3-D: ring planes (k0 - 2)/2 .. k0/2 before the first decode
  int staged_hi = -2;
  if (rings) {
    if (in.has_t && in.t2)
      two_prologue<DIM>(st0, *in.t2, gc, T, (T.k0 - 2) >> 1, T.k0 >> 1, sm.two, sm.ring, in.G1t, tid, sbad);
    for (int c = (T.k0 - 2) >> 1; c <= (T.k0 >> 1); c++) {
      if (in.has_t && !in.t2) load_t(c);
      if (in.has_u) stage_load(st1, in.u, gc, c);
      if (in.has_t && !in.t2) store_t(c);
      if (in.has_u) stage_store(st1, sm.ringu, c, in.G1u, tid);
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
  V sx, s0, Fm, F0;
  Fm = F_at(own, rm, T.k0 - 1, sx);
  F0 = F_at(own, r0, T.k0, s0);
  sm.Fs[T.k0 & 1][own.sm] = F0;
  if (has_h) sm.Fs[T.k0 & 1][hal.sm] = F_at(hal, h0, T.k0, sx);

  for (int k = T.k0; k < T.k1; k++) {
    const int cs = (k + 2) >> 1;
    const bool stage = rings && cs > staged_hi && cs <= gc.nz;
    if (stage) {
      if (in.has_t) load_t(cs);
      if (in.has_u) stage_load(st1, in.u, gc, cs);
    }
    body.advance();
    if (k + 1 < T.k1) body.prefetch(k + 1);
    Raw rn2 = rm, hn2 = rm;
    if (k + 2 <= T.k1) rn2 = raw_at(own, k + 2);
    if (has_h && k + 2 < T.k1) hn2 = raw_at(hal, k + 2);
    __syncthreads();  // plane k complete in Fs[k & 1]; ring planes for k + 1 staged
    V sp;
    const V Fp = F_at(own, rn, k + 1, sp);
    if (k + 1 < T.k1) {
      V *nxt = sm.Fs[(k + 1) & 1];
      nxt[own.sm] = Fp;
      if (has_h) nxt[hal.sm] = F_at(hal, hn, k + 1, sx);
    }
    const V *P = sm.Fs[k & 1];
    if constexpr (Body::kRaw) {
      body.out_raw(k, P + own.sm, Fm, F0, Fp, s0);
    } else {
      const V S = 6 * F0 - Fm - Fp - P[own.sm - 1] - P[own.sm + 1] - P[own.sm - PW] - P[own.sm + PW];
      body.out(k, (long long)S, (long long)s0, (long long)F0, pu_at(k));
    }
    if (stage) {
      if (in.has_t) store_t(cs);
      if (in.has_u) stage_store(st1, sm.ringu, cs, in.G1u, tid);
      staged_hi = cs;
    }
    Fm = F0;
    F0 = Fp;
    s0 = sp;
    rn = rn2;
    hn = hn2;
  }
  staging_flush();
}

// March without an operand (F = 0): the body still sees every plane.
template <class Body>
__device__ __forceinline__ void march_none(const Tile &T, int nplanes_dim2, Body &body) {
  const int k1 = nplanes_dim2 ? 1 : T.k1;
  const int k0 = nplanes_dim2 ? 0 : T.k0;
  body.prefetch(k0);
  for (int k = k0; k < k1; k++) {
    body.advance();
    if (k + 1 < k1) body.prefetch(k + 1);
    body.out(k, 0, 0, 0, 0);
  }
}

// ------------------------------------------------------------------ sweep
// The sweep shapes the IR iteration launches, compiled separately so that each
// carries only its own work; SW_GENERIC takes every option at run time (step-wise API).
enum SweepMode {
  SW_GENERIC = 0,
  SW_DOWN,           // y~' = round(y~ + c (rc - A y~))
  SW_UP,             // operand y~ + P w_(l-1)
  SW_UP_CORR,        // last up-sweep on the finest level: u~ += y~' (y~' not stored)
  SW_UP_CORR_UH,     // ... and u^_l for the next FMG level
  SW_UP_CORR_W_UH,   // last up-sweep below the finest level: u~ += y~', w_l, u^_l
  SW_UP0,            // first up-sweep from y~ = 0 (red half-sweep of V(0,1)): operand P w_(l-1)
};

template <int M>
struct SwF {
  static constexpr bool fixed = M != SW_GENERIC;
  static constexpr bool y = M != SW_UP0;
  static constexpr bool z = M >= SW_UP;
  static constexpr bool wy = M == SW_DOWN || M == SW_UP || M == SW_UP0;
  static constexpr bool corr = M >= SW_UP_CORR && M <= SW_UP_CORR_W_UH;
  static constexpr bool uh = M == SW_UP_CORR_UH || M == SW_UP_CORR_W_UH;
  static constexpr bool w = M == SW_UP_CORR_W_UH;
};

template <int DIM, int M>
struct SweepBody {
  static constexpr bool kRaw = false;
  const SweepArgs &a;
  const Geo &g;
  int GF, MF, GA, MA, G1u;
  bool ring_u;          // P_l u^_(l-1) from the ring (else per value from global memory)
  int Mu;               // |P_l u^_(l-1)| < 2^Mu over the footprint
  int GPw, MPw;         // P_l w_(l-1) is exact on grid GPw, |P_l w_(l-1)| < 2^MPw
  int bip, lane, ty, i, j;
  bool rowok, pt;
  CodePos cprc, cpu;
  Raw rc_n, u_n;        // prefetched inputs of the next plane
  Raw rc_c, u_c;        // inputs of the current plane
  bool ovf;
  MetaAcc my, mu;
  uint32_t *pk;

  // options: compile-time for the fixed shapes (y~ present), run-time otherwise
  __device__ __forceinline__ bool HY() const { return SwF<M>::fixed ? SwF<M>::y : (bool)a.has_y; }
  __device__ __forceinline__ bool HZ() const { return SwF<M>::fixed ? SwF<M>::z : (bool)a.has_z; }
  __device__ __forceinline__ bool WY() const { return SwF<M>::fixed ? SwF<M>::wy : (bool)a.write_y; }
  __device__ __forceinline__ bool CORR() const { return SwF<M>::fixed ? SwF<M>::corr : (bool)a.corr; }
  __device__ __forceinline__ bool WW() const { return SwF<M>::fixed ? SwF<M>::w : (bool)a.write_w; }
  __device__ __forceinline__ bool WUH() const { return SwF<M>::fixed ? SwF<M>::uh : (bool)a.write_uh; }
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

  __device__ __forceinline__ void out(int k, long long S, long long own, long long F0, long long Pu) {
    if (!rowok) return;  // warp-uniform: one warp per row
    const Raw rc = rc_c, u = u_c;
    const int blk = k * g.n * g.nbx + bip;
    const int erc = rc.e;
    const int Gres = imin(blk_lsb(erc, a.rc.W), GA);
    const int Mres = imax(erc == -128 ? MAG_NONE : erc, MA) + 1;
    const int Gcr = Gres + a.c_exp;
    const int Gy = HY() ? imin(GF, Gcr) : Gcr;
    if (!pt) S = 0;
    const bool up = upd(k);  // a node left out by a half-sweep keeps y~
    long long ynew;
    // static range of this block (warp-uniform); else per-value checks
    if (Gres >= GRID_NONE / 2 || (Mres - Gres <= 62 - a.cbits && Mres + a.cbits + a.c_exp - Gy <= 61 &&
                                  (!HY() || MF - Gy <= 61))) {
      const long long res = raw_val(rc, cprc.boff, a.rc.W, Gres) - shl_fast(S, GA - Gres);
      ynew = up ? shl_fast(res * a.c_num, Gcr - Gy) : 0;
      if (HY()) ynew += shl_fast(own, GF - Gy);
    } else {
      if (erc != -128 && erc - Gres > 61) ovf = true;
      const long long res = raw_val(rc, cprc.boff, a.rc.W, Gres) - (up ? shl_ck(S, GA - Gres, ovf) : 0);
      ck62(res, ovf);
      ynew = up ? shl_ck(mul_ck(res, a.c_num, a.cbits, ovf), Gcr - Gy, ovf) : 0;
      if (HY()) ynew += shl_ck(own, GF - Gy, ovf);
      ck62(ynew, ovf);
    }
    int e, sh;
    const int q = encode_block(ynew, Gy, a.Wy, e, sh, a.err);
    const long long yr = rounded_value(ynew, q, sh);
    if (WY()) {
      pack_block(q, a.Wy, pk, a.y_out.words + (long long)blk * a.Wy);
      if (lane == 0) {
        a.y_out.exps[blk] = (int8_t)e;
        my.add(e);
      }
    }
    long long ur = 0;
    int Gu = Gy, eu = -128;
    if (CORR()) {
      const int eu0 = u.e;
      Gu = imin(blk_lsb(eu0, a.u_in.W), Gy);
      if (e != -128 || eu0 != -128)
        if (imax(eu0 == -128 ? MAG_NONE : eu0, e) + 1 - Gu > 62) ovf = true;
      const long long usum = raw_val(u, cpu.boff, a.u_in.W, Gu) + shl_fast(yr, Gy - Gu);
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
    if (WW()) {  // w_l = y~' + P w_(l-1); P w_(l-1) = F - y~ at this node
      // block grid: the coarser of the grids y~' and P w_(l-1) are exact on
      const int gY = e == -128 ? GRID_NONE : imax(e - a.Wy + 1, Gy);
      const int gw = imin(gY, HZ() ? GPw : GRID_NONE);
      long long w = 0;
      if (gw < GRID_NONE / 2) {
        const long long pw = (HZ() && pt) ? F0 - (HY() ? own : 0) : 0;
        if (imax(HZ() ? MPw : MAG_NONE, e == -128 ? MAG_NONE : e) + 1 - gw <= 62) {
          w = regrid(yr, Gy, gw) + regrid(pw, GF, gw);
        } else {
          w = regrid(yr, Gy, gw) + (gw >= GF ? regrid(pw, GF, gw) : shl_ck(pw, GF - gw, ovf));
          ck62(w, ovf);
        }
      }
      store_tmp_on(w, gw, a.w_out.v + p, a.w_out.gb + blk, pt, ovf);
    }
    if (WUH()) {  // u^_l = u~_l' + P u^_(l-1)
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

template <int DIM, int M>
__device__ __forceinline__ void sweep_tile(const SweepArgs &a, const Tile &T) {
  using F = SwF<M>;
  const bool has_y = F::fixed ? F::y : (bool)a.has_y, has_z = F::fixed ? F::z : (bool)a.has_z;
  const bool write_y = F::fixed ? F::wy : (bool)a.write_y, corr = F::fixed ? F::corr : (bool)a.corr;
  const bool write_uh = F::fixed ? F::uh : (bool)a.write_uh;
  __shared__ SmemAny sm;
  __shared__ uint32_t pk[TY][33];
  __shared__ int smy[2], smu[2], smb[6];
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  if (tid == 0) smy[0] = smy[1] = smu[0] = smu[1] = 0;
  const bool uring_wanted = write_uh && a.has_uhc;
  Bounds bs, bt, bu;
  footprint_bounds<DIM>(g, a.gc, T, a.y_in, has_y, a.wc, has_z, a.uhc, uring_wanted, smb, bs, bt, bu,
                        a.tl ? &a.wc2 : nullptr);
  const Bounds bF = operand_of(bs, bt);
  const int GF = bF.G, MF = bF.M;
  const int sA = (DIM - 2) * g.l;
  if (tid == 0 && GF < GRID_NONE / 2 && MF + 4 - GF > 62) flag_range(a.err, 101, MF + 4, GF);
  SweepBody<DIM, M> b{a, g};
  b.GF = GF;
  b.MF = MF;
  b.GA = GF - sA;
  b.MA = MF + 4 - sA;  // |A F| < 2^MA on grid GA
  // the u^ ring holds the footprint on one grid when its span fits
  b.ring_u = uring_wanted && (bu.G >= GRID_NONE / 2 || bu.M - bu.G <= 61);
  b.G1u = bu.G < GRID_NONE / 2 ? bu.G : 0;
  b.Mu = bu.M;
  b.GPw = bt.G < GRID_NONE / 2 ? bt.G - 1 : GRID_NONE;
  b.MPw = bt.M;
  b.lane = lane;
  b.ty = ty;
  b.i = T.x0 + lane;
  b.j = T.j0 + ty;
  b.rowok = b.j < g.n;
  b.pt = b.rowok && b.i < g.n;
  b.bip = b.rowok ? b.j * g.nbx + T.bx : 0;
  b.cprc = code_pos(lane, a.rc.W);
  b.cpu = code_pos(lane, corr ? a.u_in.W : 1);
  b.ovf = false;
  b.my.init();
  b.mu.init();
  b.pk = pk[ty];
  MarchIn in;
  in.s = a.y_in;
  in.t = a.wc;
  in.u = a.uhc;
  in.has_s = has_y;
  in.has_t = has_z;
  in.has_u = b.ring_u;
  in.GF = GF;
  in.G1t = GF + 1;
  in.G1u = b.G1u;
  if (a.tl) in.t2 = &a.wc2;
  in.err = a.err;
  if (in.has_s || in.has_t || in.has_u) {
    if (narrow_operand(GF, MF)) march<DIM>(g, a.gc, T, in, sm.w32, b);
    else march<DIM>(g, a.gc, T, in, sm.w64, b);
  } else {
    march_none(T, DIM == 2, b);
  }
  ovf_flush(b.ovf, a.err, 102);
  if (write_y) meta_flush(b.my, a.y_out.meta, smy);
  if (corr) meta_flush(b.mu, a.u_out.meta, smu);
}

// every tile of the level, or (list_mode) the fallback tiles the specialised
// kernel left, one after the other per CTA
template <int DIM, int M>
__global__ void __launch_bounds__(NT, CMG_SWEEP_MINB) k_sweep(SweepArgs a) {
  if (a.list_mode) {
    const int n = *a.ntiles;
    for (int idx = blockIdx.x; idx < n; idx += gridDim.x) {
      sweep_tile<DIM, M>(a, tile_of_code(a.g, a.tiles[idx]));
      __syncthreads();
    }
    return;
  }
  sweep_tile<DIM, M>(a, make_tile(a.g));
}

// ------------------------------------------------------------------ residual
__device__ __forceinline__ long long rne_shift128(__int128 v, int s) {
  if (s <= 0) return (long long)v;
  __int128 q = v >> s;
  __int128 rem = v - (q << s);
  __int128 half = (__int128)1 << (s - 1);
  if (rem > half || (rem == half && (q & 1))) q += 1;
  return (long long)q;
}

// F_q at level-l node (I, J, K): sum_t prod_a T[t][a][I_a * stride - 1], exact
// in 128 bits, rounded to nearest-even after dropping fsh bits (any number of
// terms; reads the tables from global memory).
template <int DIM>
__device__ __forceinline__ long long rhs_global(const ResidArgs &a, int I, int J, int K) {
  const int stride = 1 << (a.Lmax - a.g.l);
  const int n1 = a.n1max;
  __int128 F = 0;
  for (int t = 0; t < a.nterms; t++) {
    const int32_t *T = a.tables + (long long)t * DIM * n1;
    long long yz = (long long)__ldg(T + n1 + J * stride - 1);
    if (DIM == 3) yz *= (long long)__ldg(T + 2 * n1 + K * stride - 1);
    F += (__int128)__ldg(T + I * stride - 1) * (__int128)yz;
  }
  return rne_shift128(F, a.fsh);
}

struct RhsSmem {
  int2 pxy[TMAXP][NT];     // T_x(I) T_y(J) of each thread's column, per term, as
                           // lo + 2^32 hi with lo in [-2^31, 2^31)
  int tz[TMAXP][ZC];       // T_z(K) of the tile's planes
};

// round-to-nearest-even of (hi 2^32 + lo) / 2^fsh, lo in [0, 2^32)
__device__ __forceinline__ long long rne96(long long hi, unsigned lo, int fsh) {
  if (fsh >= 33) {
    const int s = fsh - 32;
    long long q = hi >> s;
    const unsigned long long rh = (unsigned long long)hi & ((1ull << s) - 1ull);
    const unsigned long long hh = 1ull << (s - 1);
    if (rh > hh || (rh == hh && (lo != 0u || (q & 1)))) q += 1;
    return q;
  }
  return rne_shift128(((__int128)hi << 32) + (__int128)lo, fsh);
}

// residual shapes: RS_FIRST (the IR iteration with pre-smoothing: r and the first
// sweep's y~, u^_(L-1) present) compiled apart from the run-time generic one
enum ResidMode { RS_GENERIC = 0, RS_FIRST };

template <int DIM, int M>
struct ResidBody {
  static constexpr bool kRaw = false;
  const ResidArgs &a;
  const Geo &g;
  const RhsSmem &rs;
  int GF, GA, Gt, Gcr, k0;
  int Gd;               // fused restriction: grid of R t^_L is Gd - 1
  bool fast, rhs_sm, dfast;
  int bip, lane, ty, i, j;
  bool rowok, pt;
  bool ovf;
  MetaAcc mr, my;
  uint32_t *pk;

  __device__ __forceinline__ bool FS() const { return M == RS_FIRST ? true : (bool)a.first_sweep; }
  __device__ __forceinline__ bool FR() const { return M == RS_FIRST ? false : (bool)a.fuse_restrict; }
  __device__ __forceinline__ void prefetch(int) {}
  __device__ __forceinline__ void advance() {}

  // F_q at this thread's node of plane k, exactly: each term (T_x T_y) T_z is
  // (lo + 2^32 hi) T_z with two 32 x 32-bit products; SA collects floor(term /
  // 2^32) (|SA| < 2^62 for a bound below 2^94), L the remainders (< 2^35)
  __device__ __forceinline__ long long rhs(int k) {
    if (!rhs_sm) return rhs_global<DIM>(a, i + 1, j + 1, k + 1);
    long long SA = 0, L = 0;
    const int tid = ty * 32 + lane;
    for (int t = 0; t < a.nterms; t++) {
      const int2 p = rs.pxy[t][tid];
      const int z = DIM == 3 ? rs.tz[t][k - k0] : 1;
      const long long b = (long long)p.x * z;  // |b| < 2^61
      SA += (long long)p.y * z + (b >> 32);
      L += b & 0xffffffffll;
    }
    return rne96(SA + (L >> 32), (unsigned)(L & 0xffffffffll), a.fsh);
  }

  __device__ __forceinline__ void out(int k, long long S, long long, long long, long long) {
    if (!rowok) return;
    long long t = 0;
    if (pt) {
      const long long fq = rhs(k);
      if (fast) {
        t = shl_fast(fq, a.Gf - Gt) - shl_fast(S, GA - Gt);
      } else {
        t = shl_ck(fq, a.Gf - Gt, ovf) - shl_ck(S, GA - Gt, ovf);
        ck62(t, ovf);
      }
    }
    int e, sh;
    const int q = encode_block(t, Gt, a.r_out.W, e, sh, a.err);
    const int blk = k * g.n * g.nbx + bip;
    pack_block(q, a.r_out.W, pk, a.r_out.words + (long long)blk * a.r_out.W);
    if (lane == 0) {
      a.r_out.exps[blk] = (int8_t)e;
      mr.add(e);
    }
    if (FS()) {  // y~ = round(c r): the first Jacobi sweep from y~ = 0
      const long long rr = rounded_value(t, q, sh);
      int ey, sy;
      const int qy = encode_block(fast ? rr * a.c_num : mul_ck(rr, a.c_num, a.cbits, ovf), Gcr, a.y_out.W, ey,
                                  sy, a.err);
      pack_block(qy, a.y_out.W, pk, a.y_out.words + (long long)blk * a.y_out.W);
      if (lane == 0) {
        a.y_out.exps[blk] = (int8_t)ey;
        my.add(ey);
      }
    }
    if (FR()) {  // t^_L at the width of Table 1 (Wt), restricted at once: R t^_L on Gd - 1
      int et, st;
      const int qt = encode_block(t, Gt, a.Wt, et, st, a.err);
      const long long th = rounded_value(t, qt, st);  // on grid Gt >= Gd
      long long d;
      if (dfast) {
        d = shl_fast(th, Gt - Gd);
      } else {
        d = shl_ck(th, Gt - Gd, ovf);
        ck58(d, ovf);
      }
      if (pt && d) scatter_restrict<DIM>((unsigned long long *)a.racc.v, a.gc, i + 1, j + 1, k + 1, d);
    }
  }
};

template <int DIM, int M>
__device__ __forceinline__ void residual_tile(const ResidArgs &a, const Tile &T) {
  const bool first_sweep = M == RS_FIRST ? true : (bool)a.first_sweep;
  const bool has_uhc = M == RS_FIRST ? true : (bool)a.has_uhc;
  __shared__ SmemAny sm;
  __shared__ RhsSmem rs;
  __shared__ uint32_t pk[TY][33];
  __shared__ int smr[2], smy[2], smb[6];
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  if (tid == 0) smr[0] = smr[1] = smy[0] = smy[1] = 0;
  // the tile's slice of the separable right-hand side tables (Sec. 7 problems):
  // exact products need |sum| < 2^94 for the split accumulation
  const bool rhs_sm = a.nterms <= TMAXP && a.rhs_bits <= 94;
  if (rhs_sm) {
    const int stride = 1 << (a.Lmax - g.l), n1 = a.n1max;
    const int ii = T.x0 + lane, jj = T.j0 + ty;
    for (int t = 0; t < a.nterms; t++) {
      const int32_t *Tt = a.tables + (long long)t * DIM * n1;
      const long long p = (ii < g.n && jj < g.n)
                              ? (long long)__ldg(Tt + (ii + 1) * stride - 1) * __ldg(Tt + n1 + (jj + 1) * stride - 1)
                              : 0;
      const int lo = (int)(unsigned)(unsigned long long)p;
      rs.pxy[t][tid] = make_int2(lo, (int)((p - lo) >> 32));
    }
    for (int idx = tid; idx < a.nterms * ZC; idx += NT) {
      const int t = idx / ZC, r = idx - t * ZC, kk = T.k0 + r;
      const int32_t *Tt = a.tables + (long long)t * DIM * n1;
      rs.tz[t][r] = (DIM == 3 && kk < g.nz) ? __ldg(Tt + 2 * n1 + (kk + 1) * stride - 1) : 1;
    }
  }
  Bounds bs, bt, bu;
  footprint_bounds<DIM>(g, a.gc, T, a.u, true, a.uhc, has_uhc, a.uhc, false, smb, bs, bt, bu,
                        a.tl ? &a.uhc2 : nullptr);
  const Bounds bF = operand_of(bs, bt);
  const int GF = bF.G, MF = bF.M;
  const int sA = (DIM - 2) * g.l;
  const int GA = GF - sA, MA = MF + 4 - sA;
  const int Gt = imin(a.Gf, GA), Mt = imax(a.Gf + 51, MA) + 1;
  if (tid == 0 && GF < GRID_NONE / 2 && MF + 4 - GF > 62) flag_range(a.err, 201, MF + 4, GF);
  ResidBody<DIM, M> b{a, g, rs};
  b.GF = GF;
  b.GA = GA;
  b.Gt = Gt;
  b.Gcr = Gt + a.c_exp;
  b.k0 = T.k0;
  // the bound |t| < 2^Mt is loose (t is a residual, far below |f| + |A F|): when
  // it does not fit, every value is checked instead
  b.fast = Mt - Gt <= 62 && (!first_sweep || Mt + 1 + a.cbits - Gt <= 62);
  b.Gd = 0;
  b.dfast = true;
  if (!first_sweep && a.fuse_restrict) {
    // every operand grid of the level is at least min over l of (grid of u~_l) - (L - l):
    // u^_l = u~_l + P u^_(l-1), and P halves the grid at most once per level
    int Glo = GRID_NONE;
    for (int l = 1; l <= g.l; l++) {
      Sec s{};
      s.meta = const_cast<int *>(a.umeta[l]);
      s.W = a.uW[l];
      const int G = sec_lsb(s);
      if (G < GRID_NONE / 2) Glo = imin(Glo, G - (g.l - l));
    }
    b.Gd = imin(a.Gf, Glo < GRID_NONE / 2 ? Glo - sA : GRID_NONE);
    if (tid == 0 && first_cta()) a.racc.meta[0] = b.Gd - 1;
    b.dfast = Mt - b.Gd <= 57;
  }
  b.rhs_sm = rhs_sm;
  b.lane = lane;
  b.ty = ty;
  b.i = T.x0 + lane;
  b.j = T.j0 + ty;
  b.rowok = b.j < g.n;
  b.pt = b.rowok && b.i < g.n;
  b.bip = b.rowok ? b.j * g.nbx + T.bx : 0;
  b.ovf = false;
  b.mr.init();
  b.my.init();
  b.pk = pk[ty];
  MarchIn in;
  in.s = a.u;
  in.t = a.uhc;
  in.u = a.uhc;
  in.has_s = true;
  in.has_t = has_uhc;
  in.has_u = false;
  in.GF = GF;
  in.G1t = GF + 1;
  in.G1u = 0;
  if (a.tl) in.t2 = &a.uhc2;
  in.err = a.err;
  if (narrow_operand(GF, MF)) march<DIM>(g, a.gc, T, in, sm.w32, b);
  else march<DIM>(g, a.gc, T, in, sm.w64, b);
  ovf_flush(b.ovf, a.err, 202);
  meta_flush(b.mr, a.r_out.meta, smr);
  if (first_sweep) meta_flush(b.my, a.y_out.meta, smy);
}

template <int DIM, int M>
__global__ void __launch_bounds__(NT, CMG_RESID_MINB) k_residual(ResidArgs a) {
  if (a.list_mode) {
    const int n = *a.ntiles;
    for (int idx = blockIdx.x; idx < n; idx += gridDim.x) {
      residual_tile<DIM, M>(a, tile_of_code(a.g, a.tiles[idx]));
      __syncthreads();
    }
    return;
  }
  residual_tile<DIM, M>(a, make_tile(a.g));
}

// ------------------------------------------------------------------ diffusion residual
// The outer residual of the variable-coefficient problem, t = f - A u^_L in FP64
// in the oracle's order: for the neighbours -x, +x, -y, +y, -z, +z,
// acc = acc + ((k_q + k_p) * 0.5) * (u_p - u_q), A u = acc h^(d-2), t = f - A u,
// rounded into r as the oracle rounds doubles.  u^_L comes exactly from the
// int64 march (u~_L + P u^_(L-1) on the CTA grid) and converts exactly to FP64
// while it spans at most 53 bits (else an error flag).
template <int DIM>
struct ResidDiffBody {
  static constexpr bool kRaw = true;
  const ResidArgs &a;
  const Geo &g;
  int GF;             // grid of the raw operand values
  double hs;          // h^(d-2)
  int kstride;
  int bip, lane, i, j;
  bool rowok, pt, bad;
  MetaAcc mr;
  uint32_t *pk;

  __device__ __forceinline__ void prefetch(int) {}
  __device__ __forceinline__ void advance() {}
  __device__ __forceinline__ int b_stride() const { return kstride; }
  __device__ __forceinline__ float kat(int I, int J, int K) const {
    return __ldg(a.kfield + ((long long)(DIM == 3 ? K * kstride : 0) * a.kN + J * kstride) * a.kN + I * kstride);
  }
  __device__ __forceinline__ void ck53(long long v) {  // u^ must be an exact binary64 value
    if (v >= (1ll << 53) || v <= -(1ll << 53)) bad = true;
  }
  __device__ __forceinline__ void out(int, long long, long long, long long, long long) {}

  __device__ __forceinline__ void out_raw(int k, const long long *Pc, long long Fm, long long F0, long long Fp,
                                          long long) {
    if (!rowok) return;
    double t = 0.0;
    if (pt) {
      const int I = i + 1, J = j + 1, K = k + 1;
      ck53(F0);
      const float kp = kat(I, J, K);
      const long long nv[6] = {Pc[-1], Pc[1], Pc[-PW], Pc[PW], Fm, Fp};
      double acc = 0.0;
      // the oracle's acc + ((k_q + k_p) 0.5)(u_p - u_q) in FP64: u_p, u_q are exact
      // doubles on one grid, so fl(u_p - u_q) is the RNE binary64 of the exact
      // integer difference, formed here with integer instructions; k_q + k_p of
      // two binary32 values is exact in binary64, and (s 0.5) d = s (d 0.5) is the
      // same real product, so the 0.5 goes into the difference's exponent
#pragma unroll
      for (int e = 0; e < 2 * DIM; e++) {
        const int Iq = I + (e == 0 ? -1 : e == 1 ? 1 : 0), Jq = J + (e == 2 ? -1 : e == 3 ? 1 : 0);
        const int Kq = K + (e == 4 ? -1 : e == 5 ? 1 : 0);
        ck53(nv[e]);
        const double s = f32_sum_f64(kat(Iq, Jq, Kq), kp, bad);
        acc = __dadd_rn(acc, __dmul_rn(s, i64_to_f64_rne(F0 - nv[e], GF - 1, bad)));
      }
      double f;
      if (a.grhs) {  // nodal right-hand side, injected: f_L = h_L^d 2^grhs_log2 g (exact scaling)
        const int s = b_stride(), n1 = a.n1max;
        const long long gi = DIM == 3 ? ((long long)(K * s - 1) * n1 + (J * s - 1)) * n1 + (I * s - 1)
                                      : (long long)(J * s - 1) * n1 + (I * s - 1);
        f = scalbn(__ldg(a.grhs + gi), a.grhs_log2 - DIM * g.l);
      } else {
        const long long fq = rhs_global<DIM>(a, I, J, K);  // below 2^52 after the rounding shift
        ck53(fq);
        f = i64_to_f64_rne(fq, a.Gf, bad);
      }
      t = __dsub_rn(f, __dmul_rn(acc, hs));
    }
    int e;
    const int q = encode_block_f64(t, a.r_out.W, e, a.err);
    const int blk = k * g.n * g.nbx + bip;
    pack_block(q, a.r_out.W, pk, a.r_out.words + (long long)blk * a.r_out.W);
    if (lane == 0) {
      a.r_out.exps[blk] = (int8_t)e;
      mr.add(e);
    }
  }
};

template <int DIM>
__global__ void __launch_bounds__(NT, 2) k_residual_diff(ResidArgs a) {
  __shared__ SmemTile sm;
  __shared__ uint32_t pk[TY][33];
  __shared__ int smr[2], smb[6];
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const Tile T = make_tile(g);
  if (tid == 0) smr[0] = smr[1] = 0;
  Bounds bs, bt, bu;
  footprint_bounds<DIM>(g, a.gc, T, a.u, true, a.uhc, a.has_uhc, a.uhc, false, smb, bs, bt, bu);
  const Bounds bF = operand_of(bs, bt);
  const int GF = bF.G, MF = bF.M;
  if (tid == 0 && GF < GRID_NONE / 2 && MF + 4 - GF > 62) flag_range(a.err, 204, MF + 4, GF);
  ResidDiffBody<DIM> b{a, g};
  // 2^GF as a double (GF is at least -1022 for every operand that fits here)
  b.GF = GF;
  b.hs = __longlong_as_double((long long)(1023 - (DIM - 2) * g.l) << 52);
  b.kstride = 1 << (a.Lmax - g.l);
  b.lane = lane;
  b.i = T.x0 + lane;
  b.j = T.j0 + ty;
  b.rowok = b.j < g.n;
  b.pt = b.rowok && b.i < g.n;
  b.bip = b.rowok ? b.j * g.nbx + T.bx : 0;
  b.bad = false;
  b.mr.init();
  b.pk = pk[ty];
  MarchIn in;
  in.s = a.u;
  in.t = a.uhc;
  in.u = a.uhc;
  in.has_s = true;
  in.has_t = a.has_uhc;
  in.has_u = false;
  in.GF = GF;
  in.G1t = GF + 1;
  in.G1u = 0;
  march<DIM>(g, a.gc, T, in, sm, b);
  ovf_flush(b.bad, a.err, 205);
  meta_flush(b.mr, a.r_out.meta, smr);
}

// ------------------------------------------------------------------ restriction
template <int DIM>
struct RestrictBody {
  static constexpr bool kRaw = false;
  const RestrictArgs &a;
  const Geo &g;
  int GA, Gd;
  bool fast;
  int bip, i, j;
  bool rowok, pt;
  CodePos cprc;
  Raw rc_n, rc_c;
  bool ovf;

  __device__ __forceinline__ void prefetch(int k) {
    if (!rowok) return;
    rc_n = raw_load(a.rc, k * g.n * g.nbx + bip, cprc, true);
  }
  __device__ __forceinline__ void advance() { rc_c = rc_n; }

  __device__ __forceinline__ void out(int k, long long S, long long, long long, long long) {
    if (!rowok) return;
    const Raw rc = rc_c;
    if (rc.e != -128 && rc.e - Gd > 57) ovf = true;
    long long d = raw_val(rc, cprc.boff, a.rc.W, Gd);
    if (a.has_y && pt) {
      if (fast) {
        d -= shl_fast(S, GA - Gd);
      } else {
        d -= shl_ck(S, GA - Gd, ovf);
        ck58(d, ovf);
      }
    }
    if (pt && d) scatter_restrict<DIM>((unsigned long long *)a.acc.v, a.gc, i + 1, j + 1, k + 1, d);
  }
};

template <int DIM>
__global__ void __launch_bounds__(NT, CMG_RESTRICT_MINB) k_restrict(RestrictArgs a) {
  __shared__ SmemAny sm;
  __shared__ int smb[6];
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const Tile T = make_tile(g);
  // one grid for every contribution to the accumulator, from the sections'
  // global finest grids: the accumulator holds R d on Gd - 1
  const int sA = (DIM - 2) * g.l;
  const int Gd = imin(sec_lsb(a.rc), a.has_y ? sec_lsb(a.y) - sA : GRID_NONE);
  if (tid == 0 && first_cta()) a.acc.meta[0] = Gd - 1;
  Bounds bs, bt, bu;
  footprint_bounds<DIM>(g, a.gc, T, a.y, a.has_y, a.acc, false, a.acc, false, smb, bs, bt, bu);
  const Bounds bF = operand_of(bs, bt);
  const int GF = bF.G, MF = bF.M;
  const int GA = GF - sA, MA = MF + 4 - sA;
  if (tid == 0 && a.has_y && GF < GRID_NONE / 2 && MF + 4 - GF > 62) flag_range(a.err, 301, MF + 4, GF);
  RestrictBody<DIM> b{a, g};
  b.GA = GA;
  b.Gd = Gd;
  b.fast = !a.has_y || GF >= GRID_NONE / 2 || MA - Gd <= 57;  // else every d is checked
  b.i = T.x0 + lane;
  b.j = T.j0 + ty;
  b.rowok = b.j < g.n;
  b.pt = b.rowok && b.i < g.n;
  b.bip = b.rowok ? b.j * g.nbx + T.bx : 0;
  b.cprc = code_pos(lane, a.rc.W);
  b.ovf = false;
  MarchIn in;
  in.s = a.y;
  in.t = a.acc;
  in.u = a.acc;
  in.has_s = a.has_y;
  in.has_t = false;
  in.has_u = false;
  in.GF = GF;
  in.G1t = 0;
  in.G1u = 0;
  if (!in.has_s) march_none(T, DIM == 2, b);
  else if (narrow_operand(GF, MF)) march<DIM>(g, a.gc, T, in, sm.w32, b);
  else march<DIM>(g, a.gc, T, in, sm.w64, b);
  ovf_flush(b.ovf, a.err, 302);
}

dim3 stencil_grid(const Geo &g) {
  return dim3((unsigned)g.nbx, (unsigned)((g.n + TY - 1) / TY), (unsigned)((g.nz + ZC - 1) / ZC));
}

}  // namespace

template <int DIM>
static void launch_sweep_dim(const SweepArgs &a, cudaStream_t st) {
  const dim3 grid = stencil_grid(a.g), b(32, TY);
  int m = SW_GENERIC;
  if (a.has_y) {
    if (!a.corr && a.write_y && !a.write_w && !a.write_uh) m = a.has_z ? SW_UP : SW_DOWN;
    else if (a.corr && a.has_z && !a.write_y && !a.write_w) m = a.write_uh ? SW_UP_CORR_UH : SW_UP_CORR;
    else if (a.corr && a.has_z && !a.write_y && a.write_w && a.write_uh) m = SW_UP_CORR_W_UH;
  } else if (a.has_z && a.write_y && !a.corr && !a.write_w && !a.write_uh) {
    m = SW_UP0;
  }
  switch (m) {
    case SW_DOWN: k_sweep<DIM, SW_DOWN><<<grid, b, 0, st>>>(a); break;
    case SW_UP: k_sweep<DIM, SW_UP><<<grid, b, 0, st>>>(a); break;
    case SW_UP_CORR: k_sweep<DIM, SW_UP_CORR><<<grid, b, 0, st>>>(a); break;
    case SW_UP_CORR_UH: k_sweep<DIM, SW_UP_CORR_UH><<<grid, b, 0, st>>>(a); break;
    case SW_UP_CORR_W_UH: k_sweep<DIM, SW_UP_CORR_W_UH><<<grid, b, 0, st>>>(a); break;
    case SW_UP0: k_sweep<DIM, SW_UP0><<<grid, b, 0, st>>>(a); break;
    default: k_sweep<DIM, SW_GENERIC><<<grid, b, 0, st>>>(a); break;
  }
}

void launch_sweep(int dim, const SweepArgs &a, cudaStream_t st) {
  if (dim == 3) launch_sweep_dim<3>(a, st);
  else launch_sweep_dim<2>(a, st);
}

// the fallback tiles of a specialised 3-D launch: a fixed grid of CTAs that
// each read the list length and run their share (usually none)
static unsigned list_grid(const Geo &g) {
  const long long tiles = (long long)stencil_grid(g).x * stencil_grid(g).y * stencil_grid(g).z;
  return (unsigned)(tiles < 456 ? tiles : 456);
}

void launch_sweep_list(int dim, const SweepArgs &a, cudaStream_t st) {
  SweepArgs b = a;
  b.list_mode = 1;
  const dim3 t(32, TY);
  int m = SW_GENERIC;
  if (!a.has_y && a.has_z && a.write_y && !a.corr && !a.write_w && !a.write_uh) m = SW_UP0;
  else if (a.has_y && a.corr && a.has_z && !a.write_y && !a.write_w && !a.write_uh) m = SW_UP_CORR;
  else if (a.has_y && a.corr && a.has_z && !a.write_y && a.write_w && a.write_uh) m = SW_UP_CORR_W_UH;
  else if (a.has_y && a.corr && a.has_z && !a.write_y && !a.write_w && a.write_uh) m = SW_UP_CORR_UH;
  if (dim != 3) return;
  if (m == SW_UP0) k_sweep<3, SW_UP0><<<list_grid(a.g), t, 0, st>>>(b);
  else if (m == SW_UP_CORR) k_sweep<3, SW_UP_CORR><<<list_grid(a.g), t, 0, st>>>(b);
  else if (m == SW_UP_CORR_W_UH) k_sweep<3, SW_UP_CORR_W_UH><<<list_grid(a.g), t, 0, st>>>(b);
  else if (m == SW_UP_CORR_UH) k_sweep<3, SW_UP_CORR_UH><<<list_grid(a.g), t, 0, st>>>(b);
  else k_sweep<3, SW_GENERIC><<<list_grid(a.g), t, 0, st>>>(b);
}

void launch_residual_list(int dim, const ResidArgs &a, cudaStream_t st) {
  ResidArgs b = a;
  b.list_mode = 1;
  if (dim == 3) k_residual<3, RS_GENERIC><<<list_grid(a.g), dim3(32, TY), 0, st>>>(b);
}

void launch_residual(int dim, const ResidArgs &a, cudaStream_t st) {
  dim3 b(32, TY);
  const bool first = a.first_sweep && !a.fuse_restrict && a.has_uhc;
  if (dim == 3) {
    if (first) k_residual<3, RS_FIRST><<<stencil_grid(a.g), b, 0, st>>>(a);
    else k_residual<3, RS_GENERIC><<<stencil_grid(a.g), b, 0, st>>>(a);
  } else {
    if (first) k_residual<2, RS_FIRST><<<stencil_grid(a.g), b, 0, st>>>(a);
    else k_residual<2, RS_GENERIC><<<stencil_grid(a.g), b, 0, st>>>(a);
  }
}

// dJ/dk_i = -(1/2) h^(d-2) sum over the neighbours q of i inside the closed grid
// (order -x,+x,-y,+y,-z,+z) of (u_i - u_q)(lam_i - lam_q), u = lam = 0 on the
// boundary; one thread per node of the closed grid.  dg = h^d lam.
__global__ void __launch_bounds__(256) k_gradient(GradArgs a) {
  const long long N = a.kN, total = a.dim == 3 ? N * N * N : N * N;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int I = (int)(t % N), J = (int)((t / N) % N), K = a.dim == 3 ? (int)(t / (N * N)) : 0;
  const int n = (int)N - 2;
  auto at = [&](const double *x, int Ii, int Jj, int Kk) -> double {  // zero on the boundary
    if (Ii < 1 || Ii > n || Jj < 1 || Jj > n) return 0.0;
    if (a.dim == 3 && (Kk < 1 || Kk > n)) return 0.0;
    const long long p = a.dim == 3 ? ((long long)(Kk - 1) * n + (Jj - 1)) * n + (Ii - 1)
                                   : (long long)(Jj - 1) * n + (Ii - 1);
    return __ldg(x + p);
  };
  const double ui = at(a.u, I, J, K), li = at(a.lam, I, J, K);
  double acc = 0.0;
  for (int e = 0; e < 2 * a.dim; e++) {
    const int Iq = I + (e == 0 ? -1 : e == 1 ? 1 : 0), Jq = J + (e == 2 ? -1 : e == 3 ? 1 : 0);
    const int Kq = K + (e == 4 ? -1 : e == 5 ? 1 : 0);
    if (Iq < 0 || Iq >= N || Jq < 0 || Jq >= N || (a.dim == 3 && (Kq < 0 || Kq >= N))) continue;
    acc = __dadd_rn(acc, __dmul_rn(__dsub_rn(ui, at(a.u, Iq, Jq, Kq)), __dsub_rn(li, at(a.lam, Iq, Jq, Kq))));
  }
  const double hs = __longlong_as_double((long long)(1023 - (a.dim - 2) * a.L) << 52);
  a.dk[t] = -__dmul_rn(__dmul_rn(acc, 0.5), hs);
  if (a.dg && I >= 1 && I <= n && J >= 1 && J <= n && (a.dim == 2 || (K >= 1 && K <= n))) {
    const long long p = a.dim == 3 ? ((long long)(K - 1) * n + (J - 1)) * n + (I - 1) : (long long)(J - 1) * n + (I - 1);
    a.dg[p] = __dmul_rn(li, __longlong_as_double((long long)(1023 - a.dim * a.L) << 52));
  }
}

void launch_gradient(const GradArgs &a, cudaStream_t st) {
  const long long N = a.kN, total = a.dim == 3 ? N * N * N : N * N;
  k_gradient<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a);
}

void launch_residual_diffusion(int dim, const ResidArgs &a, cudaStream_t st) {
  dim3 b(32, TY);
  if (dim == 3) k_residual_diff<3><<<stencil_grid(a.g), b, 0, st>>>(a);
  else k_residual_diff<2><<<stencil_grid(a.g), b, 0, st>>>(a);
}

void launch_restrict(int dim, const RestrictArgs &a, cudaStream_t st) {
  dim3 b(32, TY);
  if (dim == 3) k_restrict<3><<<stencil_grid(a.g), b, 0, st>>>(a);
  else k_restrict<2><<<stencil_grid(a.g), b, 0, st>>>(a);
}

}  // namespace cmg
