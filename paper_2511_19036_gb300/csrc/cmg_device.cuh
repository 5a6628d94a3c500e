// Device-side building blocks of the compact FMG kernels (sm_103a).
//
// Number representation on the GPU.  Every quantity of the method is a dyadic
// rational.  Kernels compute exactly in int64 fixed point: a value v on grid G
// stands for v * 2^G.  Grids are chosen locally, never globally, because the
// BFP blocks of a section adapt to the local magnitude (blocks next to the
// Dirichlet boundary are orders of magnitude smaller, with much finer last
// bits, than interior blocks), so one grid per array would need far more than
// 64 bits:
//   * BFP sections carry their grid in each block exponent (e - W + 1);
//   * int64 temporaries (decoded solution chain, w = y~ + z) carry one
//     descriptor per 32-value block, written by the warp that produced the
//     block: its grid and the bit length of its largest magnitude;
//   * a stencil kernel converts its operand to one grid per CTA tile, the
//     finest grid found in the tile's footprint;
//   * each warp chooses the grid of its output block from its own inputs.
// Exact arithmetic makes the order of evaluation irrelevant; the only rounding
// is the round-to-nearest-even into a BFP section (Sec. 4 of the paper).  Every
// shift and constant multiply of a computed value is checked (shl_ck, mul_ck);
// a value that would not fit raises ERR_RANGE rather than wrapping.
//
// Section metadata (two ints per written section, fresh for every write):
//   m[0] = max over nonzero blocks of (e + META_BIAS)  (0: no nonzero block)
//   m[1] = max over nonzero blocks of (META_BIAS - e)
// Restriction accumulators (exact sums from many CTAs by integer atomics) use
// one global grid: m[0] = G.
#pragma once
#include <cstdint>

namespace cmg {

constexpr int META_BIAS = 1000;
constexpr int GRID_NONE = 1 << 20;    // grid of an all-zero input: no constraint
constexpr int MAG_NONE = -(1 << 20);  // magnitude exponent of an all-zero input

// error flags accumulated in a device word
constexpr int ERR_EXP = 1;      // block exponent outside [-127, 127]
constexpr int ERR_RANGE = 2;    // exact integer range would exceed 62 bits
constexpr int ERR_CORRUPT = 4;  // code -2^(W-1) met in decoding
constexpr int ERR_INPUT = 8;    // non-finite input to the codec

constexpr int TY = 8;     // rows per CTA in the stencil kernels (one warp per row)
constexpr int ZC = 32;    // z-planes marched per CTA
constexpr int NT = 32 * TY;

struct Geo {
  int l;        // level
  int n;        // interior nodes per axis
  int nz;       // n in 3-D, 1 in 2-D
  int R;        // padded row length (multiple of 32)
  int nbx;      // blocks per row
  long long nblocks;
};

struct Sec {
  uint32_t *words;  // nblocks * W words
  int8_t *exps;     // nblocks exponents
  int W;
  int *meta;        // 2 ints (see above)
};

struct Tmp {
  long long *v;     // padded layout ((k*n + j)*R + i)
  int *gb;          // per 32-value block descriptor (grid << 8 | bits); nullptr for accumulators
  int *meta;        // accumulators: {G, unused}
};

// A temporary of level lc held in two levels instead of materialized (the
// finest level's coarse sources, decoded on the fly): x_lc = s_lc + P_lc x_(lc-1)
// with s the BFP section of level lc (y~ or u~) and x_(lc-1) the materialized
// temporary of level lc - 1 (w or u^).
struct Tmp2 {
  Sec s;   // level lc section
  Tmp b;   // level lc - 1 temporary
  Geo gb;  // level lc - 1 geometry
};

__host__ __device__ inline int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ inline int imax(int a, int b) { return a > b ? a : b; }

// Range failures record the first offending site and its (M, G) pair in
// err[1..3] so that the host can report them.
__device__ inline void flag_range(int *err, int site, int M, int G) {
  atomicOr(err, ERR_RANGE);
  if (atomicCAS(err + 1, 0, site) == 0) {
    err[2] = M;
    err[3] = G;
  }
}

// ---------------------------------------------------------------- metadata
__device__ inline int sec_lsb(const Sec &s) {  // finest grid of a section's values
  int m1 = __ldg(s.meta + 1);
  if (m1 == 0) return GRID_NONE;
  int emin = META_BIAS - m1;
  return emin - s.W + 1;
}
__device__ inline int sec_msb(const Sec &s) {  // |value| < 2^msb
  int m0 = __ldg(s.meta);
  if (m0 == 0) return MAG_NONE;
  return m0 - META_BIAS;
}
__device__ __forceinline__ int blk_lsb(int e, int W) { return e == -128 ? GRID_NONE : e - W + 1; }
// temporary block descriptor: values v of the block stand for v * 2^grid with
// |v| < 2^bits; bits == 0 marks an all-zero block
__device__ __forceinline__ int gb_grid(int gb) { return (gb & 0xff) ? (gb >> 8) : GRID_NONE; }
__device__ __forceinline__ int gb_mag(int gb) { return (gb & 0xff) ? (gb >> 8) + (gb & 0xff) : MAG_NONE; }

// ---------------------------------------------------------------- checked integer ops
// exact left shift of an int64 (0 stays 0)
__device__ __forceinline__ long long shl(long long v, int s) {
  return (s >= 63) ? 0 : (long long)((unsigned long long)v << s);
}

// left shift that records whether the result leaves (-2^62, 2^62)
__device__ __forceinline__ long long shl_ck(long long v, int s, bool &ovf) {
  if (s >= 63) {
    ovf |= (v != 0);
    return 0;
  }
  long long hi = v >> (62 - s);
  ovf |= (unsigned long long)(hi + 1) > 1ull;
  return (long long)((unsigned long long)v << s);
}

// v * c for a constant with bit length cbits, recording a possible overflow
__device__ __forceinline__ long long mul_ck(long long v, int c, int cbits, bool &ovf) {
  long long hi = v >> (62 - cbits);
  ovf |= (unsigned long long)(hi + 1) > 1ull;
  return v * (long long)c;
}

// |v| < 2^62 check of a computed value before rounding
__device__ __forceinline__ void ck62(long long v, bool &ovf) {
  ovf |= (unsigned long long)((v >> 62) + 1) > 1ull;
}
// |v| < 2^58: stencil operands (a 7-point sum stays in 62 bits) and restriction
// contributions (a sum of at most 15 stays in 62 bits)
__device__ __forceinline__ void ck58(long long v, bool &ovf) {
  ovf |= (unsigned long long)((v >> 58) + 1) > 1ull;
}

// ---------------------------------------------------------------- decoding
// W-bit two's-complement code i of a block (words of that block)
__device__ __forceinline__ int code_at(const uint32_t *bw, int W, int lane) {
  int pos = lane * W, wd = pos >> 5, off = pos & 31;
  uint32_t lo = __ldg(bw + wd);
  uint32_t hi = (off + W > 32) ? __ldg(bw + wd + 1) : 0u;
  uint32_t bits = __funnelshift_r(lo, hi, off);
  return ((int)(bits << (32 - W))) >> (32 - W);
}

__device__ __forceinline__ bool inside(const Geo &g, int i, int j, int k) {
  return (unsigned)i < (unsigned)g.n && (unsigned)j < (unsigned)g.n && (unsigned)k < (unsigned)g.nz;
}
__device__ __forceinline__ long long blk_index(const Geo &g, int i, int j, int k) {
  return ((long long)k * g.n + j) * g.nbx + (i >> 5);
}

// value of section s at 0-based (i, j, k) on grid 2^G (G <= its block's grid);
// zero outside the interior.  The invalid code -2^(W-1) sets bad (and decodes
// as that number, so that the caller's range checks stay meaningful).
__device__ __forceinline__ long long sec_val_ck(const Sec &s, const Geo &g, int i, int j, int k, int G,
                                                bool &ovf, bool &bad) {
  if (!inside(g, i, j, k)) return 0;
  long long b = blk_index(g, i, j, k);
  int e = __ldg(s.exps + b);
  if (e == -128) return 0;
  int q = code_at(s.words + b * s.W, s.W, i & 31);
  bad |= (unsigned)q == (0xffffffffu << (s.W - 1));
  return shl_ck((long long)q, e - s.W + 1 - G, ovf);
}

// temporary value and grid at 0-based (i, j, k); zero outside the interior
__device__ __forceinline__ long long tmp_raw(const Tmp &t, const Geo &g, int i, int j, int k, int &G) {
  if (!inside(g, i, j, k)) {
    G = GRID_NONE;
    return 0;
  }
  G = gb_grid(__ldg(t.gb + blk_index(g, i, j, k)));
  return __ldg(t.v + ((long long)k * g.n + j) * g.R + i);
}

// coarse parents of fine node (I, J, K) (1-based) for P_l: an all-even node has
// one parent I/2, any other node the two parents (I -+ e_S)/2 (S = odd axes).
template <int DIM>
struct Parents {
  int ia, ja, ka, ib, jb, kb;
  bool two;
  __device__ __forceinline__ Parents(int I, int J, int K) {
    int sx = I & 1, sy = J & 1, sz = (DIM == 3) ? (K & 1) : 0;
    two = (sx | sy | sz) != 0;
    ia = ((I - sx) >> 1) - 1;
    ja = ((J - sy) >> 1) - 1;
    ka = (DIM == 3) ? ((K - sz) >> 1) - 1 : 0;
    ib = ((I + sx) >> 1) - 1;
    jb = ((J + sy) >> 1) - 1;
    kb = (DIM == 3) ? ((K + sz) >> 1) - 1 : 0;
  }
};

// (P_l c)(I, J, K) on grid G: linear interpolation along the Kuhn edge through
// the node (Sec. 3.1 prolongation of the nested P1 spaces)
template <int DIM>
__device__ __forceinline__ long long prolong_tmp(const Tmp &c, const Geo &gc, int I, int J, int K, int G,
                                                 bool &ovf) {
  Parents<DIM> p(I, J, K);
  int ga, gb;
  long long a = tmp_raw(c, gc, p.ia, p.ja, p.ka, ga);
  if (!p.two) return a ? shl_ck(a, ga - G, ovf) : 0;
  long long b = tmp_raw(c, gc, p.ib, p.jb, p.kb, gb);
  return (a ? shl_ck(a, ga - 1 - G, ovf) : 0) + (b ? shl_ck(b, gb - 1 - G, ovf) : 0);
}

// grid on which (P_l c)(I, J, K) is exact
template <int DIM>
__device__ __forceinline__ int prolong_grid(const Tmp &c, const Geo &gc, int I, int J, int K) {
  Parents<DIM> p(I, J, K);
  int G = GRID_NONE;
  if (inside(gc, p.ia, p.ja, p.ka)) G = gb_grid(__ldg(c.gb + blk_index(gc, p.ia, p.ja, p.ka)));
  if (!p.two) return G;
  if (inside(gc, p.ib, p.jb, p.kb)) G = imin(G, gb_grid(__ldg(c.gb + blk_index(gc, p.ib, p.jb, p.kb))));
  return G >= GRID_NONE / 2 ? G : G - 1;
}

// value and grid of a two-level temporary at 0-based (i, j, k) of its level g:
// the section's code on its block grid plus P of the lower temporary, exact on
// the returned grid G (GRID_NONE: zero); zero outside the interior.  bad: the
// invalid code -2^(W-1).
template <int DIM>
__device__ __forceinline__ long long tmp2_raw(const Tmp2 &t, const Geo &g, int i, int j, int k, int &G, bool &ovf,
                                              bool &bad) {
  G = GRID_NONE;
  if (!inside(g, i, j, k)) return 0;
  const long long blk = blk_index(g, i, j, k);
  const int e = __ldg(t.s.exps + blk);
  long long vs = 0;
  int Gs = GRID_NONE;
  if (e != -128) {
    const int q = code_at(t.s.words + blk * t.s.W, t.s.W, i & 31);
    bad |= (unsigned)q == (0xffffffffu << (t.s.W - 1));
    vs = q;
    Gs = e - t.s.W + 1;
  }
  Parents<DIM> p(i + 1, j + 1, k + 1);
  int ga, gb2 = GRID_NONE;
  const long long a = tmp_raw(t.b, t.gb, p.ia, p.ja, p.ka, ga);
  const long long b = p.two ? tmp_raw(t.b, t.gb, p.ib, p.jb, p.kb, gb2) : 0;
  // P x_(lc-1): a copy on ga, or (a + b) / 2 on min(ga, gb) - 1
  const int Gp = p.two ? imin(ga, gb2) - 1 : ga;
  G = imin(Gs, Gp);
  if (G >= GRID_NONE / 2) {
    G = GRID_NONE;
    return 0;
  }
  long long v = vs ? shl_ck(vs, Gs - G, ovf) : 0;
  if (p.two) {
    if (a) v += shl_ck(a, ga - 1 - G, ovf);
    if (b) v += shl_ck(b, gb2 - 1 - G, ovf);
  } else if (a) {
    v += shl_ck(a, ga - G, ovf);
  }
  return v;
}

// (P_l x)(I, J, K) of a two-level temporary x of level l - 1 (geometry gc),
// exact on the returned grid G (GRID_NONE: zero)
template <int DIM>
__device__ __forceinline__ long long prolong2(const Tmp2 &t, const Geo &gc, int I, int J, int K, int &G, bool &ovf,
                                              bool &bad) {
  Parents<DIM> p(I, J, K);
  int ga, gb2 = GRID_NONE;
  const long long a = tmp2_raw<DIM>(t, gc, p.ia, p.ja, p.ka, ga, ovf, bad);
  const long long b = p.two ? tmp2_raw<DIM>(t, gc, p.ib, p.jb, p.kb, gb2, ovf, bad) : 0;
  G = p.two ? imin(ga, gb2) - 1 : ga;
  if (G >= GRID_NONE / 2) {
    G = GRID_NONE;
    return 0;
  }
  if (!p.two) return a;
  return (a ? shl_ck(a, ga - 1 - G, ovf) : 0) + (b ? shl_ck(b, gb2 - 1 - G, ovf) : 0);
}

// ---------------------------------------------------------------- rounding
// round-to-nearest-even of v / 2^s for s > 0; v * 2^-s (exact) for s <= 0
__device__ __forceinline__ long long rne_shift(long long v, int s) {
  if (s <= 0) return shl(v, -s);
  long long q = v >> s;  // floor
  unsigned long long rem = (unsigned long long)v & ((1ull << s) - 1ull);
  unsigned long long half = 1ull << (s - 1);
  if (rem > half || (rem == half && (q & 1))) q += 1;
  return q;
}

// rne_shift for a warp-uniform s: for s > 0, floor((v + 2^(s-1) - 1 + lsb) /
// 2^s) with lsb the last bit of floor(v / 2^s) rounds to nearest, ties to even
// (|v| < 2^62, so the sum cannot overflow)
__device__ __forceinline__ long long rne_shift_w(long long v, int s) {
  if (s <= 0) return (long long)((unsigned long long)v << (-s));
  const long long lsb = (v >> s) & 1;
  return (v + ((1ll << (s - 1)) - 1) + lsb) >> s;
}

__device__ __forceinline__ int bitlen64(long long v) {
  unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  return a ? 64 - __clzll((long long)a) : 0;
}

// Warp-collective bit length of the largest |v| of a block (0: all zero),
// from two 32-bit warp reductions.
__device__ __forceinline__ int block_bitlen(long long v) {
  const unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
  const unsigned hmax = __reduce_max_sync(0xffffffffu, (unsigned)(a >> 32));
  if (hmax) return 64 - __clz((int)hmax);
  const unsigned lmax = __reduce_max_sync(0xffffffffu, (unsigned)a);
  return lmax ? 32 - __clz((int)lmax) : 0;
}

// Warp-collective BFP rounding of one block: every lane passes its exact value
// v on grid 2^G (padding lanes pass 0).  Returns the W-bit code; e receives the
// block exponent (-128 for an all-zero block) and s the drop shift, so that the
// rounded value on grid G is rne_shift(v, s) << s when s > 0, else v itself.
__device__ __forceinline__ int encode_block(long long v, int G, int W, int &e, int &s, int *err) {
  const int bmax = block_bitlen(v);
  if (bmax == 0) {
    e = -128;
    s = 0;
    return 0;
  }
  e = bmax + G;  // 2^(e-1) <= max|v| 2^G < 2^e
  s = bmax - (W - 1);
  long long q = rne_shift_w(v, s);
  // |q| <= 2^(W-1); |q| == 2^(W-1) (rounding carried into the next power of
  // two) iff q + 2^(W-1) is 0 mod 2^W, tested on the low 32 bits
  const unsigned lim = 1u << (W - 1), mask = (lim << 1) - 1u;
  if (__any_sync(0xffffffffu, (((unsigned)q + lim) & mask) == 0u)) {
    e += 1;
    s += 1;
    q = rne_shift_w(v, s);
  }
  if ((e > 127 || e < -127) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_EXP);
  return (int)q;
}

// Warp-collective BFP rounding of one block of FP64 values x (padding lanes
// pass 0), as the oracle rounds doubles: e = the smallest integer with
// max|x| < 2^e, q = RNE(x 2^(W-1-e)) (the scaling is exact), and a carry into
// 2^(W-1) raises e by one and re-rounds.  A subnormal block maximum or an
// exponent outside [-127, 127] sets an error flag.
__device__ __forceinline__ int encode_block_f64(double x, int W, int &e, int *err) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  const unsigned emx = __reduce_max_sync(0xffffffffu, (unsigned)(bits >> 52));
  if (emx == 0) {
    if (__any_sync(0xffffffffu, bits != 0ull) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_RANGE);
    e = -128;
    return 0;
  }
  e = (int)emx - 1022;  // max|x| in [2^(e-1), 2^e)
  if (e > 127 || e < -127) {
    if ((threadIdx.x & 31) == 0) atomicOr(err, ERR_EXP);
    e = imax(-127, imin(127, e));
  }
  const double scale = __longlong_as_double((long long)(W - 1 - e + 1023) << 52);
  long long q = __double2ll_rn(__dmul_rn(x, scale));
  const long long lim = 1ll << (W - 1);
  if (__any_sync(0xffffffffu, q == lim || q == -lim)) {
    e += 1;
    q = __double2ll_rn(__dmul_rn(x, __dmul_rn(scale, 0.5)));
  }
  return (int)q;
}

// Exact binary64 of a binary32 value by assembling the bits with integer
// instructions (normal inputs; zero, subnormal, infinite and NaN inputs take the
// conversion instruction).
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)x;
  return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) |
                                          ((unsigned long long)(e + 896u) << 52) |
                                          ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// v 2^G rounded to nearest-even into binary64 with integer instructions (exact
// for |v| < 2^53); |v| < 2^63 - 1.  A result outside the normal range sets bad.
__device__ __forceinline__ double i64_to_f64_rne(long long v, int G, bool &bad) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
  const unsigned long long u = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  int nb = 64 - __clzll((long long)u);  // 2^(nb-1) <= u < 2^nb
  unsigned long long m;
  if (nb <= 53) {
    m = u << (53 - nb);
  } else {
    const int sh = nb - 53;
    m = u >> sh;
    const unsigned long long rem = u & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) m += 1ull;
    if (m >> 53) {  // rounded up to the next power of two
      m >>= 1;
      nb += 1;
    }
  }
  const int be = nb - 1 + G + 1023;  // m in [2^52, 2^53): value = m 2^(nb - 53 + G)
  if (be <= 0 || be >= 2047) {
    bad = true;
    return 0.0;
  }
  return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | (m & ((1ull << 52) - 1ull))));
}

// fl(a + b) in binary64 of two binary32 values with integer instructions: the
// significands aligned in int64 and summed exactly, then rounded to nearest-even
// (what the FP64 addition of the two exact doubles gives).  Zero, subnormal and
// non-finite inputs, and exponents more than 38 apart, take the FP64 addition.
__device__ __forceinline__ double f32_sum_f64(float a, float b, bool &bad) {
  const unsigned ua = __float_as_uint(a), ub = __float_as_uint(b);
  const int ea = (int)((ua >> 23) & 0xffu), eb = (int)((ub >> 23) & 0xffu);
  if (ea == 0 || ea == 0xff || eb == 0 || eb == 0xff || ea - eb > 38 || eb - ea > 38)
    return __dadd_rn((double)a, (double)b);
  long long ma = (long long)((ua & 0x7fffffu) | 0x800000u), mb = (long long)((ub & 0x7fffffu) | 0x800000u);
  if (ua >> 31) ma = -ma;
  if (ub >> 31) mb = -mb;
  const int e = ea < eb ? ea : eb;
  return i64_to_f64_rne((ma << (ea - e)) + (mb << (eb - e)), e - 150, bad);  // value m 2^(e - 127 - 23)
}

__device__ __forceinline__ long long rounded_value(long long v, int q, int s) {
  return s > 0 ? shl((long long)q, s) : v;
}

// Warp-collective packing of 32 W-bit codes into W words (code i at bits
// [iW, iW+W)), through a per-warp scratch of 33 shared words.
__device__ __forceinline__ void pack_block(int q, int W, uint32_t *scratch, uint32_t *out) {
  int lane = threadIdx.x & 31;
  if (lane < W + 1) scratch[lane] = 0u;
  __syncwarp();
  unsigned long long code = (unsigned long long)((unsigned)q & (W == 32 ? 0xffffffffu : ((1u << W) - 1u)));
  int pos = lane * W, wd = pos >> 5, off = pos & 31;
  unsigned long long sh = code << off;
  if ((uint32_t)sh) atomicOr(scratch + wd, (uint32_t)sh);
  if ((uint32_t)(sh >> 32)) atomicOr(scratch + wd + 1, (uint32_t)(sh >> 32));
  __syncwarp();
  if (lane < W) out[lane] = scratch[lane];
  __syncwarp();
}

// Warp-collective store of one 32-value block of a temporary: the values v on
// grid G are renormalised to the coarsest grid that holds them all exactly
// (common trailing zero bits removed) and written with the block descriptor.
__device__ __forceinline__ void store_tmp_block(long long v, int G, long long *dst, int *gb, bool active,
                                                bool &ovf) {
  unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)(unsigned long long)v);
  unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)((unsigned long long)v >> 32));
  int lane = threadIdx.x & 31;
  if (!(lo | hi)) {  // all-zero block
    if (active) *dst = 0;
    if (lane == 0) *gb = 0;
    return;
  }
  int tz = lo ? __ffs(lo) - 1 : 32 + __ffs(hi) - 1;
  long long vn = v >> tz;
  int bits = __reduce_max_sync(0xffffffffu, bitlen64(vn));
  int g = G + tz;
  if (g > (1 << 22) || g < -(1 << 22)) ovf = true;
  if (active) *dst = vn;
  if (lane == 0) *gb = (int)((unsigned)g << 8) | bits;
}

// Warp-collective store of one 32-value block of a temporary whose values w are
// already on their block grid g (a grid the caller knows every value to be a
// multiple of); writes the descriptor with the exact bit length.
__device__ __forceinline__ void store_tmp_on(long long w, int g, long long *dst, int *gb, bool active, bool &ovf) {
  const int bits = block_bitlen(w);
  if (active) *dst = w;
  if ((threadIdx.x & 31) == 0) {
    if (bits && (g > (1 << 22) || g < -(1 << 22))) ovf = true;
    *gb = bits ? (int)((unsigned)g << 8) | bits : 0;
  }
}

// CTA-level reduction of written exponents into the section metadata.
struct MetaAcc {
  int emax, emin_neg;  // running max of (e + BIAS) and (BIAS - e)
  __device__ void init() { emax = 0; emin_neg = 0; }
  __device__ void add(int e) {
    if (e != -128) {
      emax = imax(emax, e + META_BIAS);
      emin_neg = imax(emin_neg, META_BIAS - e);
    }
  }
};

// lane 0 of each warp holds a MetaAcc; reduce over the CTA and publish once
__device__ inline void meta_flush(MetaAcc a, int *meta, int *sm2) {
  // sm2: 2 shared ints, zero-initialised by the caller before a __syncthreads
  if ((threadIdx.x & 31) == 0 && a.emax) {
    atomicMax(sm2, a.emax);
    atomicMax(sm2 + 1, a.emin_neg);
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0 && sm2[0]) {
    // the pair only grows: skip the (same-address, serialising) atomic when
    // the current value already dominates
    if (sm2[0] > *(volatile int *)meta) atomicMax(meta, sm2[0]);
    if (sm2[1] > *(volatile int *)(meta + 1)) atomicMax(meta + 1, sm2[1]);
  }
}

// warp-collective: report per-thread overflow flags once
__device__ inline void ovf_flush(bool ovf, int *err, int site) {
  if (__any_sync(0xffffffffu, ovf) && (threadIdx.x & 31) == 0) flag_range(err, site, 0, 0);
}

// warp-collective: report invalid codes met in decoding once
__device__ inline void corrupt_flush(bool bad, int *err) {
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_CORRUPT);
}

}  // namespace cmg
