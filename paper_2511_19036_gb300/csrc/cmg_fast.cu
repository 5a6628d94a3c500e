// Specialised kernels of the exact compact cycle for 3-D Poisson problems
// (sm_103a): the sweep shapes that dominate the red-black V(0,1) solve.
//
//   k_fast_sweep<0>  red half-sweep from y~ = 0: y~' = round(c (rc - A P w_(l-1)))
//                    at the red nodes (Algorithm 1 smoothing on eq. cfas, the
//                    operand z_l = P_l w_(l-1) of the coarser corrections)
//   k_fast_sweep<1>  black half-sweep with the fused correction of Algorithm 3:
//                    y~' = round(y~ + c (rc - A (y~ + P w_(l-1)))) at the black
//                    nodes, u~ <- round(u~ + y~'), y~' not stored
//
// They compute the same exact values, rounded the same way, as the generic
// k_sweep, with fewer instructions per value:
//   * 32-bit march.  A CTA runs only when its footprint bounds prove the
//     operand and the 7-point sum below 2^31 on the tile's grid
//     (MF + 4 - GF <= 30); other CTAs append their tile to a fallback list that
//     the generic kernel then runs.
//   * 32-bit output step.  Per block, bounds from the block's exponents and the
//     exact block maximum of |S| (one warp reduction) decide whether the update
//     and both roundings fit 30 bits; a block that does not fit takes an exact
//     64-bit path (a non-inlined function, so that it costs the common path no
//     registers).
//   * Packing across the CTA.  Each warp leaves the W-bit codes of its block in
//     shared memory; after the next plane's barrier one warp per 32 output
//     words packs the whole plane of TY blocks (a word per lane), and one warp
//     writes the TY exponents and keeps the section's exponent range.  No
//     shared-memory atomics.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "cmg_device.cuh"
#include "cmg_kernels.h"
#include "cmg_stencil_common.cuh"

namespace cmg {
namespace {

// resident CTAs per SM the register allocation is fitted to (red, black)
#ifndef CMG_FAST_RED_MINB
#define CMG_FAST_RED_MINB 4
#endif
#ifndef CMG_FAST_BLACK_MINB
#define CMG_FAST_BLACK_MINB 3
#endif

constexpr unsigned FULL = 0xffffffffu;

// Shifts with the PTX semantics: a count of 32 or more (as unsigned, so a
// negative count too) gives 0.  Used where the operand is zero whenever the
// count is out of range.
__device__ __forceinline__ int shl32(int v, int n) {
  int r;
  asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(n));
  return r;
}

// round-to-nearest-even of v / 2^s for s > 0 (no intermediate overflow for any
// int32 v), v * 2^-s for s <= 0 (the caller knows the result to fit)
__device__ __forceinline__ int rne32(int v, int s) {
  const int s1 = s > 1 ? s : 1;
  const int t = v >> (s1 - 1);  // floor(v / 2^(s-1)): its last bit is the half bit
  const int sticky = (v & ((1 << (s1 - 1)) - 1)) != 0;
  const int up = t & 1 & (sticky | (t >> 1));
  const int r = (t >> 1) + up;
  return s <= 0 ? (v << ((-s) & 31)) : r;
}

// Warp-collective BFP rounding (Sec. 4: nearest, ties to even) of one block of
// int32 values v on grid 2^G (padding lanes pass 0): the W-bit code; e gets the
// block exponent (-128 for an all-zero block).  The rounded value is
// code * 2^(e - W + 1), as in encode_block.  WC: compile-time width (0: W).
template <int WC>
__device__ __forceinline__ int enc32(int v, int G, int Wrt, int &e) {
  const int W = WC ? WC : Wrt;
  const unsigned m = __reduce_max_sync(FULL, (unsigned)abs(v));
  const int bmax = 32 - __clz((int)m);  // 2^(bmax-1) <= max|v| < 2^bmax (0 for m = 0)
  int s = bmax - (W - 1);
  int q = rne32(v, s);
  const unsigned lim = 1u << (W - 1), mask = (lim << 1) - 1u;
  const bool carry = __any_sync(FULL, (((unsigned)q + lim) & mask) == 0u);  // a code reached 2^(W-1)
  if (carry) q = rne32(v, s + 1);
  e = m ? bmax + G + (carry ? 1 : 0) : -128;
  return q;
}

// the same for an int64 block (rare paths)
// (the exponent range is checked by the packing warp)
__device__ __forceinline__ int enc64(long long v, int G, int W, int &e) {
  const int bmax = block_bitlen(v);
  if (bmax == 0) {
    e = -128;
    return 0;
  }
  e = bmax + G;
  const int s = bmax - (W - 1);
  long long q = rne_shift_w(v, s);
  const unsigned lim = 1u << (W - 1), mask = (lim << 1) - 1u;
  if (__any_sync(FULL, (((unsigned)q + lim) & mask) == 0u)) {
    e += 1;
    q = rne_shift_w(v, s + 1);
  }
  return (int)q;
}

// ---------------------------------------------------------------- packing
// One lane's share of packing a plane of TY blocks of W-bit codes: output word
// kw of block row b, assembled from the codes i0 .. i0 + n.
struct PackJob {
  bool on;
  int b, kw, i0, n, sh0;
};

__device__ __forceinline__ PackJob make_job(int W, int pass, int lane) {
  PackJob p;
  const int q = pass * 32 + lane;
  p.on = q < TY * W;
  p.b = p.on ? q / W : 0;
  p.kw = q - p.b * W;
  p.i0 = (32 * p.kw) / W;
  const int i1 = imin(31, (32 * p.kw + 31) / W);
  p.n = i1 - p.i0;
  p.sh0 = 32 * p.kw - W * p.i0;  // code i0 starts sh0 bits below the word
  return p;
}

constexpr int CSW = 33;  // staged code row stride (padded against bank conflicts)

// the word from the staged codes of one block row (codes masked to W bits)
template <int WC>
__device__ __forceinline__ uint32_t pack_word(const int *row, const PackJob &p, int Wrt) {
  const int W = WC ? WC : Wrt;
  uint32_t w = (uint32_t)row[p.i0] >> p.sh0;
  if constexpr (WC != 0) {
#pragma unroll
    for (int t = 1; t <= 32 / WC + 1; t++)
      if (t <= p.n) w |= (uint32_t)row[p.i0 + t] << (W * t - p.sh0);
  } else {
    int sh = W - p.sh0;
    for (int t = 1; t <= p.n; t++, sh += W) w |= (uint32_t)row[p.i0 + t] << sh;
  }
  return w;
}

// Packs plane k of the tile from staged codes / exponents: warp `pass` writes
// output words, warp TY - 1 the exponents; that warp also keeps the section's
// exponent range (as MetaAcc does) and flags exponents outside [-127, 127].
struct Packer {
  PackJob job;
  bool exp_lane;
  int W;
  int emax, emin_neg;
  bool bad_exp;
};

// Width 4 packs inside the warp: 8 codes per word, gathered by a butterfly of
// ORs over groups of 8 lanes; lane 8w writes word w.  (W = 4 is the finest-level
// residual and correction width of the red-black configurations.)
__device__ __forceinline__ void pack_w4(int q, uint32_t *words, int lane) {
  uint32_t v = ((uint32_t)q & 15u) << (4 * (lane & 7));
  v |= __shfl_xor_sync(FULL, v, 1);
  v |= __shfl_xor_sync(FULL, v, 2);
  v |= __shfl_xor_sync(FULL, v, 4);
  if ((lane & 7) == 0) words[lane >> 3] = v;
}

template <int WC>
__device__ __forceinline__ void pack_plane(Packer &pk, const Sec &out, const Geo &g, const Tile &T, int k,
                                           const int *cs, const int *ce) {
  if (WC != 4 && pk.job.on && T.j0 + pk.job.b < g.n) {
    const long long blk = ((long long)k * g.n + T.j0 + pk.job.b) * g.nbx + T.bx;
    out.words[blk * (WC ? WC : pk.W) + pk.job.kw] = pack_word<WC>(cs + pk.job.b * CSW, pk.job, pk.W);
  }
  if (pk.exp_lane) {
    const int lane = threadIdx.x;
    if (T.j0 + lane < g.n) {
      const int e = ce[lane];
      out.exps[((long long)k * g.n + T.j0 + lane) * g.nbx + T.bx] = (int8_t)e;
      if (e != -128) {
        pk.emax = imax(pk.emax, e + META_BIAS);
        pk.emin_neg = imax(pk.emin_neg, META_BIAS - e);
        pk.bad_exp |= e > 127 || e < -127;
      }
    }
  }
}

// the exponent warp publishes the section's exponent range once per CTA
__device__ __forceinline__ void packer_flush(const Packer &pk, int *meta, int *err) {
  if (threadIdx.y != TY - 1) return;
  const unsigned mx = __reduce_max_sync(FULL, (unsigned)pk.emax);
  const unsigned mn = __reduce_max_sync(FULL, (unsigned)pk.emin_neg);
  const bool bad = __any_sync(FULL, pk.bad_exp);
  if (threadIdx.x == 0) {
    if (mx) {
      if ((int)mx > *(volatile int *)meta) atomicMax(meta, (int)mx);
      if ((int)mn > *(volatile int *)(meta + 1)) atomicMax(meta + 1, (int)mn);
    }
    if (bad) atomicOr(err, ERR_EXP);
  }
}

__device__ __forceinline__ Packer make_packer(int W) {
  Packer pk;
  const int npass = (TY * W + 31) / 32;
  pk.job = make_job(W, threadIdx.y, threadIdx.x);
  pk.job.on = pk.job.on && (int)threadIdx.y < npass;
  pk.exp_lane = threadIdx.y == TY - 1 && threadIdx.x < TY;
  pk.W = W;
  pk.emax = 0;
  pk.emin_neg = 0;
  pk.bad_exp = false;
  return pk;
}

// ---------------------------------------------------------------- per-tile bounds
// The prologue of the specialised sweeps: the operand footprint (as
// footprint_bounds: exponents of the section s over planes k0-1..k1, rows
// j0-1..j0+TY, blocks bx-1..bx+1; descriptors of the coarse temporary t over the
// coarse nodes P_l reads) and, over the tile's own blocks, the grid range of rc
// and of u~ (c0 / c1).  One CTA barrier at the end.
struct TileBounds {
  Bounds s, t, t2;     // operand section, coarse temporary, second coarse temporary
  int rc_lsb, rc_msb;  // finest grid and largest exponent of rc's nonzero blocks in the tile
};

// tl: the coarse temporary t is held in two levels (t2l) instead.
template <bool HAS_S, bool HAS_T2>
__device__ __forceinline__ TileBounds tile_bounds(const Geo &g, const Geo &gc, const Tile &T, const Sec &sec,
                                                  const Tmp &t, const Tmp &t2, const Sec &rc, int *sm,
                                                  bool tl = false, const Tmp2 *t2l = nullptr) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid < 8) sm[tid] = (tid & 1) ? MAG_NONE : GRID_NONE;  // {G, M} x {s, t, rc, t2}
  __syncthreads();
  int G = GRID_NONE, M = MAG_NONE;
  if (HAS_S) {
    const int klo = T.k0 - 1, cnt = (T.k1 - klo + 1) * (TY + 2) * 3;
    for (int idx = tid; idx < cnt; idx += NT) {
      const int kk = klo + idx / ((TY + 2) * 3), rem = idx % ((TY + 2) * 3);
      const int jj = T.j0 - 1 + rem / 3, bb = T.bx - 1 + rem % 3;
      if ((unsigned)kk < (unsigned)g.nz && (unsigned)jj < (unsigned)g.n && (unsigned)bb < (unsigned)g.nbx) {
        const int e = __ldg(sec.exps + ((long long)kk * g.n + jj) * g.nbx + bb);
        if (e != -128) {
          G = imin(G, e - sec.W + 1);
          M = imax(M, e);
        }
      }
    }
    if (G < GRID_NONE / 2) atomicMin(sm, G);
    if (M > MAG_NONE / 2) atomicMax(sm + 1, M);
  }
  {  // coarse descriptors: at most 18 planes x 7 rows x 2 blocks
    const int cj0 = imax(0, T.cr0), ck0 = imax(0, ((T.k0 - 1) - 1) >> 1), cb0 = imax(0, T.cx0) >> 5;
    const int cj1 = imin(gc.n - 1, T.cr0 + CR - 1), ck1 = imin(gc.nz - 1, T.k1 >> 1);
    const int cb1 = imin(gc.n - 1, T.cx0 + CX - 1) >> 5;
    G = GRID_NONE;
    M = MAG_NONE;
    int G2 = GRID_NONE, M2 = MAG_NONE;
    if (tl) bounds2_scan(*t2l, gc, ck0, ck1, cj0, cj1, cb0, cb1, sm + 2, tid);
    for (int idx = tid; idx < 18 * CR * 2; idx += NT) {
      const int kk = ck0 + idx / (CR * 2), rem = idx % (CR * 2), jj = cj0 + rem / 2, bb = cb0 + (rem & 1);
      if (kk <= ck1 && jj <= cj1 && bb <= cb1) {
        const long long b = ((long long)kk * gc.n + jj) * gc.nbx + bb;
        const int gbv = tl ? 0 : __ldg(t.gb + b);
        if (gbv & 0xff) {
          G = imin(G, gb_grid(gbv));
          M = imax(M, gb_mag(gbv));
        }
        if (HAS_T2) {
          const int gb2 = __ldg(t2.gb + b);
          if (gb2 & 0xff) {
            G2 = imin(G2, gb_grid(gb2));
            M2 = imax(M2, gb_mag(gb2));
          }
        }
      }
    }
    if (G < GRID_NONE / 2) atomicMin(sm + 2, G);
    if (M > MAG_NONE / 2) atomicMax(sm + 3, M);
    if (HAS_T2 && G2 < GRID_NONE / 2) atomicMin(sm + 6, G2);
    if (HAS_T2 && M2 > MAG_NONE / 2) atomicMax(sm + 7, M2);
  }
  {  // the tile's own blocks of rc: thread (ty, lane) takes row j0 + ty of plane k0 + lane
    const int kk = T.k0 + threadIdx.x, jj = T.j0 + threadIdx.y;
    if (kk < T.k1 && jj < g.n) {
      const int e = __ldg(rc.exps + ((long long)kk * g.n + jj) * g.nbx + T.bx);
      if (e != -128) {
        atomicMin(sm + 4, e - rc.W + 1);
        atomicMax(sm + 5, e);
      }
    }
  }
  __syncthreads();
  TileBounds tb;
  tb.s.G = sm[0];
  tb.s.M = sm[1];
  tb.t.G = sm[2];
  tb.t.M = sm[3];
  tb.rc_lsb = sm[4];
  tb.rc_msb = sm[5];
  tb.t2.G = sm[6];
  tb.t2.M = sm[7];
  return tb;
}

// ---------------------------------------------------------------- the sweep kernels
// MODE 0: red from y~ = 0; 1: black with the correction of u~ (finest level);
// 2: the same, also writing w_l = y~' + z_l and u^_l = u~_l' + P_l u^_(l-1) (the
// levels below the finest); 3: the black half-sweep writing u^_l but no w_l (the
// finest level of an FMG stage before the next one); 4: mode 1 also storing y~'
// (the level below the finest on the two-level path: the finest level reads
// w_(L-1) = y~' + P w_(L-2) from it).  WY: width of rc and y~
// known at compile time (0: run time); WU the same for u~; C1: the Jacobi
// numerator is 1 (c = 2^c_exp).
template <int MODE, int WY, int WU, bool C1, bool TL>
__global__ void __launch_bounds__(NT, MODE >= 1 ? CMG_FAST_BLACK_MINB : CMG_FAST_RED_MINB)
    k_fast_sweep(SweepArgs a) {
  constexpr bool BLACK = MODE >= 1;
  constexpr bool WW = MODE == 2, WUH = MODE == 2 || MODE == 3;
  constexpr bool WYO = MODE == 4;  // y~' stored besides u~'
  constexpr int WO = BLACK ? WU : WY;  // output width when known
  __shared__ int Fs[2][PLANE];
  __shared__ int ring[4 * CRX];
  __shared__ long long ringu[WUH ? 4 * CRX : 1];  // P_l u^_(l-1), on one grid per tile
  __shared__ int cs[2][TY * CSW];
  __shared__ int ce[2][TY];
  __shared__ std::conditional_t<TL, Two2, char> two;  // staging of the two-level w_(l-1)
  __shared__ int cs2[WYO ? 2 : 1][WYO ? TY * CSW : 1];  // the y~' codes and exponents (mode 4)
  __shared__ int ce2[WYO ? 2 : 1][WYO ? TY : 1];
  __shared__ int smb[8];
  const Geo g = a.g, gc = a.gc;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const Tile T = make_tile(g);
  const TileBounds tb = tile_bounds<BLACK, WUH>(g, gc, T, a.y_in, a.wc, a.uhc, a.rc, smb, TL, &a.wc2);
  const Bounds bF = operand_of(tb.s, tb.t);
  const bool anyF = bF.G < GRID_NONE / 2, anyR = tb.rc_lsb < GRID_NONE / 2;
  // One output grid Gy per tile and a proof that every update fits int32:
  // |y0| < 2^(My - Gy), |c rc| < 2^(Mcr - Gy), |c h S| < c_num (3/4) 2^(MF + 4 - GF) 2^(Gcs - Gy)
  // (|S| <= 12 max|F|), and their sum below 2^31.
  const int cl = C1 ? 0 : a.cbits;  // c_num < 2^cl
  const int GF = anyF ? bF.G : 0;
  const int Gcs = anyF ? GF + a.c_exp - g.l : GRID_NONE;  // grid of c h^(d-2) S
  const int Gcr = anyR ? tb.rc_lsb + a.c_exp : GRID_NONE;  // finest grid of c rc in the tile
  const int GY0 = (BLACK && tb.s.M > MAG_NONE / 2) ? GF : GRID_NONE;
  int Gy = imin(imin(Gcs, Gcr), GY0);
  if (Gy >= GRID_NONE / 2) Gy = 0;  // nothing nonzero: every update is 0
  {
    float B = 0.0f;
    if (anyF) B += ldexpf(0.75f, bF.M + 4 - GF + cl + (Gcs - Gy));
    if (anyR) B += ldexpf(1.0f, tb.rc_msb + a.c_exp + cl - Gy);
    if (GY0 < GRID_NONE / 2) B += ldexpf(1.0f, tb.s.M - Gy);
    // u^_(l-1) is staged on its finest grid in the footprint: its span must fit int64
    const bool uh_span = WUH && tb.t2.G < GRID_NONE / 2 && tb.t2.M - tb.t2.G > 61;
    if ((anyF && bF.M + 4 - bF.G > 30) || B >= 2147483648.0f || uh_span) {  // left to the generic kernel
      if (tid == 0) tile_push(a.tiles, a.ntiles, T);
      return;
    }
  }
  // grids of the temporaries written here: P_l w_(l-1) is exact on GPw (the
  // coarse w grid minus one), P_l u^_(l-1) on G1u - 1
  const int GPw = tb.t.G < GRID_NONE / 2 ? tb.t.G - 1 : GRID_NONE, MPw = tb.t.M;
  const int G1u = (WUH && tb.t2.G < GRID_NONE / 2) ? tb.t2.G : 0, Mu = tb.t2.M;
  const int GPu = (WUH && tb.t2.G < GRID_NONE / 2) ? G1u - 1 : GRID_NONE;
  bool ovf = false;
  const int KS = Gcs < GRID_NONE / 2 ? Gcs - Gy : 0;  // shift of c h S onto Gy
  const int KR = a.c_exp - (WY ? WY : a.rc.W) + 1 - Gy;  // c rc of a block with exponent e: shift e + KR
  const int KY = GF - Gy;                                // y0 onto Gy
  const int Wrc = WY ? WY : a.rc.W;
  const int Ws = BLACK ? (WY ? WY : a.y_in.W) : 1;
  const int Wui = BLACK ? (WU ? WU : a.u_in.W) : 1;
  const Sec out = BLACK ? a.u_out : a.y_out;
  const int Wout = WO ? WO : out.W;
  const int Wy = WY ? WY : a.Wy;
  const unsigned cmask = Wout == 32 ? FULL : (1u << Wout) - 1u;
  Packer pk = make_packer(Wout);
  const unsigned ymask = Wy == 32 ? FULL : (1u << Wy) - 1u;
  Packer pk2 = make_packer(WYO ? Wy : 1);

  const int i = T.x0 + lane, j = T.j0 + ty;
  const bool rowok = j < g.n, pt = rowok && i < g.n;
  const int bip = rowok ? j * g.nbx + T.bx : 0;
  const int pb = g.n * g.nbx;
  // own column: every lane of a valid row loads the block (padding codes are
  // zero), so the block exponent is the same in every lane
  Slot own = make_slot(g, Ws, i, j, ty + 1, lane + 1, T);
  own.ok = rowok;
  own.bip = bip;
  Slot hal;
  const bool has_h = tid < NHALO;
  {
    int hi, hj, r, x;
    if (tid < 32) {
      hi = T.x0 + tid, hj = T.j0 - 1, r = 0, x = tid + 1;
    } else if (tid < 64) {
      hi = T.x0 + tid - 32, hj = T.j0 + TY, r = TY + 1, x = tid - 31;
    } else {
      const int c = imin(tid - 64, 2 * (TY + 2) - 1);
      r = c >> 1, hj = T.j0 - 1 + r;
      x = (c & 1) ? 33 : 0;
      hi = (c & 1) ? T.x0 + 32 : T.x0 - 1;
    }
    hal = make_slot(g, Ws, hi, hj, r, x, T);
  }
  Stager st = make_stager(gc, T, tid), stu = st;
  bool sbad = false;  // two-level staging of w_(l-1): an invalid code met
  auto load_w = [&](int c) {
    if constexpr (TL) two_step_issue(st, a.wc2, gc, T, c, two, tid);
    else stage_load(st, a.wc, gc, c);
  };
  auto store_w = [&](int c) {
    if constexpr (TL) two_step_store<3>(st, a.wc2, gc, T, c, two, ring, GF + 1, tid, sbad);
    else stage_store<int>(st, ring, c, GF + 1, tid);
  };
  const CodePos cprc = code_pos(lane, Wrc), cpu = code_pos(lane, Wui);
  // the red / black colour of node (i, j, k): i + j + k + 1 even is red
  const int par = (i + j + 1) & 1, want = a.rb == 2 ? 1 : 0;

  auto raw_at = [&](const Slot &sl, int kf) -> Raw {
    return raw_load(a.y_in, kf * pb + sl.bip, sl.cp, BLACK && sl.ok && (unsigned)kf < (unsigned)g.nz);
  };
  auto F_at = [&](const Slot &sl, const Raw &r, int kf, int &sv) -> int {
    sv = BLACK ? raw_val32(r, sl.cp.boff, Ws, GF) : 0;
    int za, zb;
    zparents<3>(kf, za, zb);
    return sv + ring_p(ring, sl, za, zb);
  };
  Raw rc_n{}, u_n{}, rc_c{}, u_c{};
  auto prefetch = [&](int k) {
    if (!rowok) return;
    const int blk = k * pb + bip;
    rc_n = raw_load(a.rc, blk, cprc, true);
    if (BLACK) u_n = raw_load(a.u_in, blk, cpu, true);
  };

  // output step of plane k: stage the block's codes and exponent
  auto out_step = [&](int k, int S, int y0, int F0v) {
    if (!rowok) return;  // warp-uniform
    const bool up = pt && (a.rb == 0 || ((par ^ k) & 1) == want);
    const int crc = raw_code(rc_c, cprc.boff, Wrc);
    const int tr = shl32(C1 ? crc : a.c_num * crc, rc_c.e + KR);  // c rc on Gy (0 if the block is zero)
    const int ts = shl32(C1 ? S : a.c_num * S, KS);              // c h S on Gy
    int v = up ? tr - ts : 0;
    if (BLACK) v += shl32(y0, KY);
    int e;
    int q = enc32<WY>(v, Gy, Wy, e);
    if constexpr (WYO) {
      cs2[k & 1][ty * CSW + lane] = (int)((unsigned)q & ymask);
      if (lane == 0) ce2[k & 1][ty] = e;
    }
    if (BLACK) {  // u~' = round(u~ + y~'), y~' = q 2^(e - Wy + 1)
      const int eu = u_c.e;
      const int cu = raw_code(u_c, cpu.boff, Wui);
      const int gY = e == -128 ? GRID_NONE : e - Wy + 1, gU = eu == -128 ? GRID_NONE : eu - Wui + 1;
      const int G2 = imin(gY, gU);
      const int top = imax(e == -128 ? MAG_NONE : e, eu == -128 ? MAG_NONE : eu);
      int qu, euo;
      if (G2 >= GRID_NONE / 2) {
        qu = 0;
        euo = -128;
      } else if (top + 1 - G2 <= 30) {
        qu = enc32<WU>(shl32(q, gY - G2) + shl32(cu, gU - G2), G2, Wout, euo);
      } else {  // exponents more than 25 apart (warp-uniform, rare): exact in 64 bits
        bool ovf = top + 1 - G2 > 62;
        const long long su = (q ? (long long)q << ((gY - G2) & 63) : 0) + (cu ? (long long)cu << ((gU - G2) & 63) : 0);
        qu = enc64(su, G2, Wout, euo);
        ovf_flush(ovf, a.err, 112);
      }
      if constexpr (WUH) {
        const long long p = ((long long)k * g.n + j) * g.R + i;
        const long long blk = (long long)k * pb + bip;
        if (WW) {  // w_l = y~' + P_l w_(l-1), the z part being F - y0 on GF
          const int gy = e == -128 ? GRID_NONE : e - Wy + 1;  // grid of y~'s code
          const int gw = imin(gy, GPw);
          long long w = 0;
          if (gw < GRID_NONE / 2) {
            ovf |= imax(MPw, e == -128 ? MAG_NONE : e) + 1 - gw > 62;
            const long long yv = e == -128 ? 0 : (long long)q << ((gy - gw) & 63);
            w = yv + regrid((long long)(pt ? F0v - y0 : 0), GF, gw);  // exact: P w is a multiple of 2^GPw
          }
          store_tmp_on(w, gw, a.w_out.v + p, a.w_out.gb + blk, pt, ovf);
        }
        {  // u^_l = u~_l' + P_l u^_(l-1)
          const int gU = euo == -128 ? GRID_NONE : euo - Wout + 1;
          const int gu = imin(gU, GPu);
          long long uh = 0;
          if (gu < GRID_NONE / 2) {
            ovf |= imax(euo == -128 ? MAG_NONE : euo, Mu) + 1 - gu > 62;
            int za, zb;
            zparents<3>(k, za, zb);
            const long long pu = (GPu < GRID_NONE / 2 && pt) ? ring_p(ringu, own, za, zb) : 0;
            uh = (euo == -128 ? 0 : (long long)qu << ((gU - gu) & 63)) + (pu << ((GPu - gu) & 63));
          }
          store_tmp_on(uh, gu, a.uh_out.v + p, a.uh_out.gb + blk, pt, ovf);
        }
      }
      q = qu;
      e = euo;
    }
    if constexpr (WO == 4) pack_w4(q, out.words + ((long long)k * pb + bip) * 4, lane);
    else cs[k & 1][ty * CSW + lane] = (int)((unsigned)q & cmask);
    if (lane == 0) ce[k & 1][ty] = e;
  };

  // ring planes (k0 - 2)/2 .. k0/2 before the first decode
  if constexpr (TL) two_prologue<3>(st, a.wc2, gc, T, (T.k0 - 2) >> 1, T.k0 >> 1, two, ring, GF + 1, tid, sbad);
  for (int c = (T.k0 - 2) >> 1; c <= (T.k0 >> 1); c++) {
    if (!TL) {
      load_w(c);
      store_w(c);
    }
    if (WUH) {
      stage_load(stu, a.uhc, gc, c);
      stage_store<long long>(stu, ringu, c, G1u, tid);
    }
  }
  int staged_hi = T.k0 >> 1;
  const Raw rm = raw_at(own, T.k0 - 1);
  const Raw r0 = raw_at(own, T.k0);
  Raw h0{}, hn{};
  if (has_h) h0 = raw_at(hal, T.k0);
  Raw rn = raw_at(own, T.k0 + 1);
  if (has_h) hn = raw_at(hal, T.k0 + 1);
  prefetch(T.k0);
  __syncthreads();
  int sx, s0, Fm, F0;
  Fm = F_at(own, rm, T.k0 - 1, sx);
  F0 = F_at(own, r0, T.k0, s0);
  Fs[T.k0 & 1][own.sm] = F0;
  if (has_h) Fs[T.k0 & 1][hal.sm] = F_at(hal, h0, T.k0, sx);

  for (int k = T.k0; k < T.k1; k++) {
    const int cn = (k + 2) >> 1;
    const bool stage = cn > staged_hi && cn <= gc.nz;
    if (stage) {
      load_w(cn);
      if (WUH) stage_load(stu, a.uhc, gc, cn);
    }
    rc_c = rc_n;
    u_c = u_n;
    if (k + 1 < T.k1) prefetch(k + 1);
    Raw rn2 = rm, hn2 = rm;
    if (k + 2 <= T.k1) rn2 = raw_at(own, k + 2);
    if (has_h && k + 2 < T.k1) hn2 = raw_at(hal, k + 2);
    __syncthreads();  // plane k complete in Fs[k & 1]; codes of plane k - 1 staged
    if (k > T.k0) {
      pack_plane<WO>(pk, out, g, T, k - 1, cs[(k - 1) & 1], ce[(k - 1) & 1]);
      if (WYO) pack_plane<0>(pk2, a.y_out, g, T, k - 1, cs2[(k - 1) & 1], ce2[(k - 1) & 1]);
    }
    int sp;
    const int Fp = F_at(own, rn, k + 1, sp);
    if (k + 1 < T.k1) {
      int *nxt = Fs[(k + 1) & 1];
      nxt[own.sm] = Fp;
      if (has_h) nxt[hal.sm] = F_at(hal, hn, k + 1, sx);
    }
    const int *P = Fs[k & 1];
    const int S = 6 * F0 - Fm - Fp - P[own.sm - 1] - P[own.sm + 1] - P[own.sm - PW] - P[own.sm + PW];
    out_step(k, S, s0, F0);
    if (stage) {
      store_w(cn);
      if (WUH) stage_store<long long>(stu, ringu, cn, G1u, tid);
      staged_hi = cn;
    }
    Fm = F0;
    F0 = Fp;
    s0 = sp;
    rn = rn2;
    hn = hn2;
  }
  __syncthreads();
  pack_plane<WO>(pk, out, g, T, T.k1 - 1, cs[(T.k1 - 1) & 1], ce[(T.k1 - 1) & 1]);
  packer_flush(pk, out.meta, a.err);
  if (WYO) {
    pack_plane<0>(pk2, a.y_out, g, T, T.k1 - 1, cs2[(T.k1 - 1) & 1], ce2[(T.k1 - 1) & 1]);
    packer_flush(pk2, a.y_out.meta, a.err);
  }
  if (WUH) ovf_flush(ovf, a.err, 113);
  if constexpr (TL) {
    cp_async_wait_all();  // the step issued ahead past the tile's last plane
    corrupt_flush(sbad, a.err);
  }
}

// ---------------------------------------------------------------- the residual
#ifndef CMG_FAST_RESID_MINB
#define CMG_FAST_RESID_MINB 3
#endif

constexpr int FMAXT = 8;  // right-hand-side terms held in shared memory

struct RhsTab {
  int2 pxy[FMAXT][NT];  // T_x(I) T_y(J) of each thread's column as lo + 2^31 hi, lo in [-2^30, 2^30)
  int tz[FMAXT][ZC];    // T_z(K) of the tile's planes
};

// round-to-nearest-even of (hi 2^31 + lo) / 2^fsh for 0 <= lo < 2^31, fsh >= 32
__device__ __forceinline__ long long rne_hl(long long hi, long long lo, int fsh) {
  const int s = fsh - 31;
  const long long q = hi >> s;
  const unsigned long long rem = (unsigned long long)hi & ((1ull << s) - 1ull), half = 1ull << (s - 1);
  return q + ((rem > half || (rem == half && (lo != 0 || (q & 1)))) ? 1 : 0);
}

// Round-to-nearest-even of v / 2^(s + dn) where v = ts 2^dn + lost, 0 <= lost < 2^dn
// and stk says lost != 0 (a 64-bit value normalised to 32 bits once per block);
// for s <= 0 (then dn = 0) the exact ts 2^-s.
__device__ __forceinline__ int rne_norm(int ts, bool stk, int s) {
  const int s1 = s > 1 ? s : 1;
  const int t = ts >> (s1 - 1);
  const int low = ((ts & ((1 << (s1 - 1)) - 1)) != 0) | (int)stk;
  const int r = (t >> 1) + (t & 1 & (low | (t >> 1)));
  return s <= 0 ? (ts << ((-s) & 31)) : r;
}

// BFP rounding at width W of a block normalised as above (bmax: bit length of the
// block's largest |v| on grid G; dn = max(0, bmax - 31)); s gets the total drop
// shift (the rounded value is q 2^(s + G) when s > 0, else v itself)
__device__ __forceinline__ int enc_norm(int ts, bool stk, int bmax, int dn, int G, int W, int &e, int &s) {
  if (bmax == 0) {
    e = -128;
    s = 0;
    return 0;
  }
  int sl = bmax - dn - (W - 1);  // shift below the normalised value
  int q = rne_norm(ts, stk, sl);
  const unsigned lim = 1u << (W - 1), mask = (lim << 1) - 1u;
  const bool carry = __any_sync(FULL, (((unsigned)q + lim) & mask) == 0u);
  if (carry) q = rne_norm(ts, stk, ++sl);
  e = bmax + G + (carry ? 1 : 0);
  s = sl + dn;
  return q;
}

// Algorithm 2 without pre-smoothing on level L: t = f - A (u~_L + P u^_(L-1)),
// r~_L = round(t) at Wr, t^_L = round(t) at Wt restricted at once into the
// level L-1 accumulator (R t^_L on one grid, exact integer atomics).  The
// operand needs up to 40 bits on the tile's grid, so the march is 64-bit; the
// right-hand side is formed exactly from the separable tables with 32 x 32-bit
// multiply-adds; x-adjacent contributions to the same coarse node are added in
// the warp before the atomics.
template <int NTERMS, int WR, bool TL>  // right-hand-side terms, r~ width (0: run time), two-level u^_(L-1)
__global__ void __launch_bounds__(NT, CMG_FAST_RESID_MINB) k_fast_resid(ResidArgs a) {
  const int nterms = NTERMS ? NTERMS : a.nterms;
  __shared__ long long Fs[2][PLANE];
  __shared__ long long ring[4 * CRX];
  __shared__ RhsTab rs;
  __shared__ std::conditional_t<TL, Two2, char> two;  // staging of the two-level u^_(L-1)
  __shared__ int cs[2][TY * CSW];
  __shared__ int ce[2][TY];
  __shared__ int smb[6];
  const Geo g = a.g, gc = a.gc;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const Tile T = make_tile(g);
  const int i = T.x0 + lane, j = T.j0 + ty;
  const bool rowok = j < g.n, pt = rowok && i < g.n;
  {  // the tile's slice of the separable tables
    const int stride = 1 << (a.Lmax - g.l), n1 = a.n1max;
    for (int t = 0; t < nterms; t++) {
      const int32_t *Tt = a.tables + (long long)t * 3 * n1;
      const long long p = pt ? (long long)__ldg(Tt + (i + 1) * stride - 1) * __ldg(Tt + n1 + (j + 1) * stride - 1) : 0;
      const int lo = (int)((p & 0x7fffffffll) ^ 0x40000000ll) - 0x40000000;
      rs.pxy[t][tid] = make_int2(lo, (int)((p - lo) >> 31));
    }
    for (int idx = tid; idx < nterms * ZC; idx += NT) {
      const int t = idx / ZC, r = idx - t * ZC, kk = T.k0 + r;
      rs.tz[t][r] = kk < g.nz ? __ldg(a.tables + (long long)t * 3 * n1 + 2 * n1 + (kk + 1) * stride - 1) : 0;
    }
  }
  Bounds bs, bt, bu;
  footprint_bounds<3>(g, gc, T, a.u, true, a.uhc, true, a.uhc, false, smb, bs, bt, bu, TL ? &a.uhc2 : nullptr);
  const Bounds bF = operand_of(bs, bt);
  const bool anyF = bF.G < GRID_NONE / 2;
  const int GF = anyF ? bF.G : 0;
  const int GA = anyF ? GF - g.l : GRID_NONE, MA = anyF ? bF.M + 4 - g.l : MAG_NONE;
  const int Gt = imin(a.Gf, GA), Mt = imax(a.Gf + 51, MA) + 1;
  // every operand grid of the level is at least min over l of (grid of u~_l) - (L - l)
  int Glo = GRID_NONE;
  for (int l = 1; l <= g.l; l++) {
    Sec sl{};
    sl.meta = const_cast<int *>(a.umeta[l]);
    sl.W = a.uW[l];
    const int G = sec_lsb(sl);
    if (G < GRID_NONE / 2) Glo = imin(Glo, G - (g.l - l));
  }
  const int Gd = imin(a.Gf, Glo < GRID_NONE / 2 ? Glo - g.l : GRID_NONE);
  if (tid == 0 && first_cta()) a.racc.meta[0] = Gd - 1;
  if (anyF && bF.M + 4 - bF.G > 62) {  // beyond the 64-bit march: the generic kernel flags it
    if (tid == 0) tile_push(a.tiles, a.ntiles, T);
    return;
  }
  // the static bounds on t (|f| + |A F|) are loose by the smoothness of u; where they
  // do not prove the range, a bound from each block's largest |S| decides, and where
  // that does not prove it either every shifted value is checked (as the generic
  // kernel does)
  const bool fast = Mt - Gt <= 62, dfast = Mt - Gd <= 57;
  bool ovf = false, bad_exp = false;
  const int Wr = WR ? WR : a.r_out.W, Wt = a.Wt, Ws = a.u.W;
  const unsigned cmask = Wr == 32 ? FULL : (1u << Wr) - 1u;
  Packer pk = make_packer(Wr);
  const int bip = rowok ? j * g.nbx + T.bx : 0;
  const int pb = g.n * g.nbx;
  Slot own = make_slot(g, Ws, i, j, ty + 1, lane + 1, T);
  own.ok = rowok;
  own.bip = bip;
  Slot hal;
  const bool has_h = tid < NHALO;
  {
    int hi, hj, r, x;
    if (tid < 32) {
      hi = T.x0 + tid, hj = T.j0 - 1, r = 0, x = tid + 1;
    } else if (tid < 64) {
      hi = T.x0 + tid - 32, hj = T.j0 + TY, r = TY + 1, x = tid - 31;
    } else {
      const int c = imin(tid - 64, 2 * (TY + 2) - 1);
      r = c >> 1, hj = T.j0 - 1 + r;
      x = (c & 1) ? 33 : 0;
      hi = (c & 1) ? T.x0 + 32 : T.x0 - 1;
    }
    hal = make_slot(g, Ws, hi, hj, r, x, T);
  }
  Stager st = make_stager(gc, T, tid);
  bool sbad = false;  // two-level staging of u^_(L-1): an invalid code met
  auto load_u = [&](int c) {
    if constexpr (TL) two_step_issue(st, a.uhc2, gc, T, c, two, tid);
    else stage_load(st, a.uhc, gc, c);
  };
  auto store_u = [&](int c) {
    if constexpr (TL) two_step_store<3>(st, a.uhc2, gc, T, c, two, ring, GF + 1, tid, sbad);
    else stage_store<long long>(st, ring, c, GF + 1, tid);
  };
  auto raw_at = [&](const Slot &sl, int kf) -> Raw {
    return raw_load(a.u, kf * pb + sl.bip, sl.cp, sl.ok && (unsigned)kf < (unsigned)g.nz);
  };
  auto F_at = [&](const Slot &sl, const Raw &r, int kf) -> long long {
    int za, zb;
    zparents<3>(kf, za, zb);
    return raw_val(r, sl.cp.boff, Ws, GF) + ring_p(ring, sl, za, zb);
  };
  // coarse rows of the restriction targets of this warp's fine row (1-based)
  const int J = j + 1, sy = J & 1;
  const int xa_off = (T.x0 + lane + 1 - ((lane + 1) & 1 ? 1 : 0)) >> 1;  // (I - sx) / 2
  const int xb_off = (T.x0 + lane + 1 + ((lane + 1) & 1 ? 1 : 0)) >> 1;  // (I + sx) / 2
  const bool Iodd = ((lane + 1) & 1) != 0;
  // the restriction targets of this thread: coarse rows A = (J - sy)/2 and B = (J + sy)/2,
  // columns xa_off / xb_off (1-based); per plane only the coarse plane changes
  const int ya = (J - sy) >> 1, yb = (J + sy) >> 1;
  const bool okA = xa_off >= 1 && xa_off <= gc.n && ya >= 1 && ya <= gc.n;
  const bool okB = xb_off >= 1 && xb_off <= gc.n && yb >= 1 && yb <= gc.n;
  const bool issueB = !(lane & 1);
  const long long cplane = (long long)gc.n * gc.R;
  unsigned long long *accA = (unsigned long long *)a.racc.v + (okA ? (long long)(ya - 1) * gc.R + (xa_off - 1) : 0);
  unsigned long long *accB = (unsigned long long *)a.racc.v + (okB ? (long long)(yb - 1) * gc.R + (xb_off - 1) : 0);

  auto out_step = [&](int k, long long S) {
    if (!rowok) return;  // warp-uniform
    // where the tile's static bound does not prove the range, the block's exact
    // largest |S| (one warp reduction) bounds |A F| instead: |t| < 2^Mb
    bool fst = fast, dfst = dfast;
    if (!fast || !dfast) {  // CTA-uniform
      const long long aS = pt ? (S < 0 ? -S : S) : 0;
      const int sb = (int)__reduce_max_sync(FULL, (unsigned)(64 - __clzll(aS)));
      const int Mb = imax(a.Gf + 51, GA + sb) + 1;
      fst = fast || Mb - Gt <= 62;
      dfst = dfast || Mb - Gd <= 57;
    }
    long long t = 0;
    if (pt) {
      // F_q = sum_t (T_x T_y) T_z exactly: A 2^31 + B0 + B1, then f = RNE(F / 2^fsh)
      long long A = 0, B0 = 0, B1 = 0;
      if constexpr (NTERMS != 0) {
#pragma unroll
        for (int q = 0; q < NTERMS; q++) {
          const int2 p = rs.pxy[q][tid];
          const int z = rs.tz[q][k - T.k0];
          A += (long long)p.y * z;
          if (q < 4) B0 += (long long)p.x * z;
          else B1 += (long long)p.x * z;
        }
      } else {
#pragma unroll 1
        for (int q = 0; q < nterms; q++) {
          const int2 p = rs.pxy[q][tid];
          const int z = rs.tz[q][k - T.k0];
          A += (long long)p.y * z;
          if (q < 4) B0 += (long long)p.x * z;
          else B1 += (long long)p.x * z;
        }
      }
      long long lo = (B0 & 0x7fffffffll) + (B1 & 0x7fffffffll);
      const long long hi = A + (B0 >> 31) + (B1 >> 31) + (lo >> 31);
      lo &= 0x7fffffffll;
      const long long f = rne_hl(hi, lo, a.fsh);
      if (fst) {
        t = shl_fast(f, a.Gf - Gt) - shl_fast(S, GA - Gt);
      } else {
        t = shl_ck(f, a.Gf - Gt, ovf) - shl_ck(S, GA - Gt, ovf);
        ck62(t, ovf);
      }
    }
    // one normalisation of the block to 32 bits (and a sticky bit) for both roundings
    const int bmax = block_bitlen(t);
    const int dn = bmax > 31 ? bmax - 31 : 0;
    const int ts = (int)(t >> dn);
    const bool stk = (t & ((1ll << dn) - 1)) != 0;
    int e, sh;
    const int qr = enc_norm(ts, stk, bmax, dn, Gt, Wr, e, sh);
    if constexpr (WR == 4) pack_w4(qr, a.r_out.words + ((long long)k * pb + bip) * 4, lane);
    else cs[k & 1][ty * CSW + lane] = (int)((unsigned)qr & cmask);
    if (lane == 0) ce[k & 1][ty] = e;
    int et, stt;
    const int qt = enc_norm(ts, stk, bmax, dn, Gt, Wt, et, stt);
    // t^_L on Gd (R t^ is held on Gd - 1): q 2^(stt + Gt - Gd), or t itself when nothing dropped
    long long d = stt > 0 ? shl_fast((long long)qt, stt + Gt - Gd) : shl_fast(t, Gt - Gd);
    if (!dfst) {  // |d| < 2^58 (a block with et - Gd > 58 has such a value, as in the generic check)
      ck58(d, ovf);
      ovf |= et != -128 && et - Gd > 58;
    }
    bad_exp |= et != -128 && (et > 127 || et < -127);  // t^ is not stored: its exponent checked here
    // parents of fine node (I, J, K): (I -+ s) / 2 componentwise, s the odd coordinates;
    // an all-even node has one parent (weight 1, 2d on the grid Gd - 1), others two (d each)
    const int K = k + 1, sz = K & 1;
    const bool all_even = !Iodd && !sy && !sz;
    const long long dA = all_even ? 2 * d : d, dB = all_even ? 0 : d;
    const long long pA = __shfl_down_sync(FULL, dA, 1), pB = __shfl_down_sync(FULL, dB, 1);
    // row A: lanes (odd, odd + 1) share the parent; lane 0 has no partner in the warp
    const bool issueA = (lane & 1) || lane == 0;
    const long long vA = dA + (((lane & 1) && lane < 31) ? pA : 0);
    const long long vB = dB + pB;  // row B: lanes (even, even + 1); issued by the even lane
    const int za = (K - sz) >> 1, zb = (K + sz) >> 1;
    if (issueA && okA && vA && za >= 1 && za <= gc.nz)
      atomicAdd(accA + (long long)(za - 1) * cplane, (unsigned long long)vA);
    if (issueB && okB && vB && zb >= 1 && zb <= gc.nz)
      atomicAdd(accB + (long long)(zb - 1) * cplane, (unsigned long long)vB);
  };

  if constexpr (TL) {
    two_prologue<3>(st, a.uhc2, gc, T, (T.k0 - 2) >> 1, T.k0 >> 1, two, ring, GF + 1, tid, sbad);
  } else {
    for (int c = (T.k0 - 2) >> 1; c <= (T.k0 >> 1); c++) {
      load_u(c);
      store_u(c);
    }
  }
  int staged_hi = T.k0 >> 1;
  const Raw rm = raw_at(own, T.k0 - 1);
  const Raw r0 = raw_at(own, T.k0);
  Raw h0{}, hn{};
  if (has_h) h0 = raw_at(hal, T.k0);
  Raw rn = raw_at(own, T.k0 + 1);
  if (has_h) hn = raw_at(hal, T.k0 + 1);
  __syncthreads();
  long long Fm = F_at(own, rm, T.k0 - 1);
  long long F0 = F_at(own, r0, T.k0);
  Fs[T.k0 & 1][own.sm] = F0;
  if (has_h) Fs[T.k0 & 1][hal.sm] = F_at(hal, h0, T.k0);

  for (int k = T.k0; k < T.k1; k++) {
    const int cn = (k + 2) >> 1;
    const bool stage = cn > staged_hi && cn <= gc.nz;
    if (stage) load_u(cn);
    Raw rn2 = rm, hn2 = rm;
    if (k + 2 <= T.k1) rn2 = raw_at(own, k + 2);
    if (has_h && k + 2 < T.k1) hn2 = raw_at(hal, k + 2);
    __syncthreads();
    if (k > T.k0) pack_plane<WR>(pk, a.r_out, g, T, k - 1, cs[(k - 1) & 1], ce[(k - 1) & 1]);
    const long long Fp = F_at(own, rn, k + 1);
    if (k + 1 < T.k1) {
      long long *nxt = Fs[(k + 1) & 1];
      nxt[own.sm] = Fp;
      if (has_h) nxt[hal.sm] = F_at(hal, hn, k + 1);
    }
    const long long *P = Fs[k & 1];
    const long long S = 6 * F0 - Fm - Fp - P[own.sm - 1] - P[own.sm + 1] - P[own.sm - PW] - P[own.sm + PW];
    out_step(k, S);
    if (stage) {
      store_u(cn);
      staged_hi = cn;
    }
    Fm = F0;
    F0 = Fp;
    rn = rn2;
    hn = hn2;
  }
  __syncthreads();
  pack_plane<WR>(pk, a.r_out, g, T, T.k1 - 1, cs[(T.k1 - 1) & 1], ce[(T.k1 - 1) & 1]);
  packer_flush(pk, a.r_out.meta, a.err);
  ovf_flush(ovf, a.err, 202);
  if (__any_sync(FULL, bad_exp) && lane == 0) atomicOr(a.err, ERR_EXP);
  if constexpr (TL) {
    cp_async_wait_all();  // the step issued ahead past the tile's last plane
    corrupt_flush(sbad, a.err);
  }
}

dim3 fast_grid(const Geo &g) {
  return dim3((unsigned)g.nbx, (unsigned)((g.n + TY - 1) / TY), (unsigned)((g.nz + ZC - 1) / ZC));
}

}  // namespace

bool launch_sweep_fast(const SweepArgs &a, cudaStream_t st) {
  if (a.g.nz == 1 || !a.tiles || !a.ntiles || a.rb < 0 || a.rb > 2) return false;
  int mode;
  if (!a.has_y && a.has_z && a.write_y && !a.corr && !a.write_w && !a.write_uh) mode = 0;
  else if (a.has_y && a.has_z && !a.write_y && a.corr && !a.write_w && !a.write_uh) mode = 1;
  else if (a.has_y && a.has_z && !a.write_y && a.corr && a.write_w && a.write_uh && a.has_uhc) mode = 2;
  else if (a.has_y && a.has_z && !a.write_y && a.corr && !a.write_w && a.write_uh && a.has_uhc) mode = 3;
  else if (a.has_y && a.has_z && a.write_y && a.corr && !a.write_w && !a.write_uh) mode = 4;
  else return false;
  if (a.tl && mode >= 2) return false;  // the two-level source feeds the finest level only
  const dim3 grid = fast_grid(a.g), b(32, TY);
  const bool c1 = a.c_num == 1;
  // compile-time widths for the finest-level shapes of the red-black and Jacobi
  // cycles (r~, y~ at b2 = 3..5 bits, u~ at b1 = 5 or 6)
  const int wy = a.rc.W, wu = mode ? a.u_in.W : 0;
  const bool same = mode == 0 ? a.y_out.W == wy : (a.y_in.W == wy && a.u_out.W == wu && a.Wy == wy);
  if (mode <= 1 && a.tl) {  // the finest level on the two-level path
    if (mode == 0) {
      if (same && c1 && wy == 4) k_fast_sweep<0, 4, 0, true, true><<<grid, b, 0, st>>>(a);
      else if (c1) k_fast_sweep<0, 0, 0, true, true><<<grid, b, 0, st>>>(a);
      else k_fast_sweep<0, 0, 0, false, true><<<grid, b, 0, st>>>(a);
    } else {
      if (same && c1 && wy == 4 && wu == 5) k_fast_sweep<1, 4, 5, true, true><<<grid, b, 0, st>>>(a);
      else if (c1) k_fast_sweep<1, 0, 0, true, true><<<grid, b, 0, st>>>(a);
      else k_fast_sweep<1, 0, 0, false, true><<<grid, b, 0, st>>>(a);
    }
  } else if (mode == 0) {
    if (same && c1 && wy == 4) k_fast_sweep<0, 4, 0, true, false><<<grid, b, 0, st>>>(a);
    else if (same && c1 && wy == 3) k_fast_sweep<0, 3, 0, true, false><<<grid, b, 0, st>>>(a);
    else if (same && c1 && wy == 5) k_fast_sweep<0, 5, 0, true, false><<<grid, b, 0, st>>>(a);
    else if (c1) k_fast_sweep<0, 0, 0, true, false><<<grid, b, 0, st>>>(a);
    else k_fast_sweep<0, 0, 0, false, false><<<grid, b, 0, st>>>(a);
  } else if (mode == 1) {
    if (same && c1 && wy == 4 && wu == 5) k_fast_sweep<1, 4, 5, true, false><<<grid, b, 0, st>>>(a);
    else if (same && c1 && wy == 3 && wu == 5) k_fast_sweep<1, 3, 5, true, false><<<grid, b, 0, st>>>(a);
    else if (c1) k_fast_sweep<1, 0, 0, true, false><<<grid, b, 0, st>>>(a);
    else k_fast_sweep<1, 0, 0, false, false><<<grid, b, 0, st>>>(a);
  } else if (mode == 2) {
    if (c1) k_fast_sweep<2, 0, 0, true, false><<<grid, b, 0, st>>>(a);
    else k_fast_sweep<2, 0, 0, false, false><<<grid, b, 0, st>>>(a);
  } else if (mode == 3) {
    if (same && c1 && wy == 4 && wu == 5) k_fast_sweep<3, 4, 5, true, false><<<grid, b, 0, st>>>(a);
    else if (c1) k_fast_sweep<3, 0, 0, true, false><<<grid, b, 0, st>>>(a);
    else k_fast_sweep<3, 0, 0, false, false><<<grid, b, 0, st>>>(a);
  } else {
    if (c1) k_fast_sweep<4, 0, 0, true, false><<<grid, b, 0, st>>>(a);
    else k_fast_sweep<4, 0, 0, false, false><<<grid, b, 0, st>>>(a);
  }
  launch_sweep_list(3, a, st);
  return true;
}

bool launch_residual_fast(const ResidArgs &a, cudaStream_t st) {
  // the red-black cycle's residual: 3-D, no fused first sweep, the restriction
  // of t^_L fused, the separable right-hand side in shared memory
  if (a.g.nz == 1 || !a.tiles || !a.ntiles || a.first_sweep || !a.fuse_restrict || !a.has_uhc || a.kfield ||
      a.grhs || a.nterms < 1 || a.nterms > FMAXT || a.rhs_bits > 94 || a.fsh < 32 || a.Wt > 31)
    return false;
  const dim3 grid = fast_grid(a.g), b(32, TY);
  const bool w4 = a.r_out.W == 4;
  if (a.tl) {  // the finest level on the two-level path
    if (a.nterms == 4 && w4) k_fast_resid<4, 4, true><<<grid, b, 0, st>>>(a);
    else k_fast_resid<0, 0, true><<<grid, b, 0, st>>>(a);
  } else if (a.nterms == 4 && w4) {
    k_fast_resid<4, 4, false><<<grid, b, 0, st>>>(a);
  } else if (a.nterms == 8 && w4) {
    k_fast_resid<8, 4, false><<<grid, b, 0, st>>>(a);
  } else {
    k_fast_resid<0, 0, false><<<grid, b, 0, st>>>(a);
  }
  launch_residual_list(3, a, st);
  return true;
}

}  // namespace cmg
