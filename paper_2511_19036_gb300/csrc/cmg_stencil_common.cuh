// Building blocks shared by the stencil kernels (exact int64 and FP32 cycle):
// compact reads into registers, the CTA tile and its per-thread decode slots,
// the coarse-value ring that serves P_l, the footprint scan of grids and
// magnitudes, and the exact restriction scatter R_l = P_l^T.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "cmg_device.cuh"
#include "cmg_kernels.h"

namespace cmg {

constexpr int CR = 7;               // coarse rows feeding fine rows j0-1 .. j0+TY
constexpr int CX = 19;              // coarse columns feeding fine columns x0-1 .. x0+32
constexpr int CRX = CR * CX;        // values of one ring plane
constexpr int PW = 34;              // plane buffer row: 32 values and one halo value each side
constexpr int PLANE = (TY + 2) * PW;
constexpr int NHALO = 2 * 32 + 2 * (TY + 2);  // halo values of one plane
__device__ inline bool first_cta() { return blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0; }

// ------------------------------------------------------------------ compact reads
struct Raw {
  int e;            // block exponent (-128: all-zero block or outside)
  uint32_t w0, w1;  // the word(s) holding the code
};

struct CodePos {
  int woff, boff, two;  // word offset in the block, bit offset, code spans two words
};

__device__ __forceinline__ CodePos code_pos(int x, int W) {
  CodePos c;
  const int pos = x * W;
  c.woff = pos >> 5;
  c.boff = pos & 31;
  c.two = c.boff + W > 32;
  return c;
}

// issue the loads of one code and its block exponent (no use of the result yet)
__device__ __forceinline__ Raw raw_load(const Sec &s, int blk, CodePos cp, bool ok) {
  Raw r;
  r.e = -128;
  r.w0 = 0u;
  r.w1 = 0u;
  if (ok) {
    r.e = __ldg(s.exps + blk);
    const uint32_t *w = s.words + (long long)blk * s.W + cp.woff;
    r.w0 = __ldg(w);
    if (cp.two) r.w1 = __ldg(w + 1);
  }
  return r;
}

__device__ __forceinline__ int raw_code(const Raw &r, int boff, int W) {
  const uint32_t bits = __funnelshift_r(r.w0, r.w1, boff);
  return ((int)(bits << (32 - W))) >> (32 - W);
}

// the value on grid G (G at or below the block's grid e - W + 1)
__device__ __forceinline__ long long raw_val(const Raw &r, int boff, int W, int G) {
  if (r.e == -128) return 0;
  return (long long)((unsigned long long)(long long)raw_code(r, boff, W) << (r.e - W + 1 - G));
}

// the same value as a 32-bit integer, for a caller that proved |value| < 2^31
// on grid G (then the shift is below 31)
__device__ __forceinline__ int raw_val32(const Raw &r, int boff, int W, int G) {
  if (r.e == -128) return 0;
  return (int)((unsigned)raw_code(r, boff, W) << (r.e - W + 1 - G));
}

template <class V>
__device__ __forceinline__ V raw_val_as(const Raw &r, int boff, int W, int G) {
  if constexpr (sizeof(V) == 4) return raw_val32(r, boff, W, G);
  else return raw_val(r, boff, W, G);
}

// Left shift for the paths whose static range check passed: there every shift
// of a nonzero value is below 63, and a shift of 64 or more only meets a zero
// (an operand whose footprint is all zero), so the count is taken mod 64.
__device__ __forceinline__ long long shl_fast(long long v, int s) {
  return (long long)((unsigned long long)v << (s & 63));
}

// v on grid `from` re-expressed on grid `to`: exact right shift when to >= from
// (the caller knows v to be a multiple of 2^(to - from)), left shift otherwise
// (the caller checked the range)
__device__ __forceinline__ long long regrid(long long v, int from, int to) {
  const int d = to - from;
  return d >= 0 ? (v >> (d & 63)) : (long long)((unsigned long long)v << ((-d) & 63));
}

// ------------------------------------------------------------------ tile geometry
struct Tile {
  int bx, x0, j0, k0, k1;
  int cr0, cx0;  // coarse row / column of ring entry (0, 0)
};

__device__ __forceinline__ Tile make_tile_at(const Geo &g, int bx, int by, int bz) {
  Tile T;
  T.bx = bx;
  T.x0 = T.bx * 32;
  T.j0 = by * TY;
  T.k0 = bz * ZC;
  T.k1 = imin(g.nz, T.k0 + ZC);
  T.cr0 = ((T.j0 - 1) >> 1) - 1;
  T.cx0 = ((T.x0 - 1) >> 1) - 1;
  return T;
}

__device__ __forceinline__ Tile make_tile(const Geo &g) { return make_tile_at(g, blockIdx.x, blockIdx.y, blockIdx.z); }

// Fallback tile lists: a CTA of a specialised kernel whose footprint does not fit
// that kernel's number range appends its tile, and the generic kernel of the
// same step then runs the listed tiles only.  Entry: bx | by << 10 | bz << 22
// (blocks per row < 1024, row tiles < 4096, plane tiles < 1024 for L <= 14).
__device__ __forceinline__ unsigned tile_code(const Tile &T) {
  return (unsigned)T.bx | ((unsigned)(T.j0 / TY) << 10) | ((unsigned)(T.k0 / ZC) << 22);
}
__device__ __forceinline__ Tile tile_of_code(const Geo &g, unsigned c) {
  return make_tile_at(g, (int)(c & 1023u), (int)((c >> 10) & 4095u), (int)(c >> 22));
}
__device__ __forceinline__ void tile_push(unsigned *list, int *count, const Tile &T) {
  list[atomicAdd(count, 1)] = tile_code(T);
}

// One decode slot of a thread: a fixed (i, j) column of the CTA footprint.
struct Slot {
  bool ok;     // (i, j) inside the level's plane
  int bip;     // block index inside a plane
  int sm;      // index in a plane buffer
  int oa, ob;  // P_l parents of (i, j) in a ring plane (row * CX + column)
  CodePos cp;  // code position for the operand section's width
};

// (i, j) fine 0-based, (r, x) its place in the plane buffer.  The parents of
// every footprint node fall in ring rows 1..6 and columns 1..18.
__device__ __forceinline__ Slot make_slot(const Geo &g, int W, int i, int j, int r, int x, const Tile &T) {
  Slot s;
  s.ok = (unsigned)i < (unsigned)g.n && (unsigned)j < (unsigned)g.n;
  s.bip = s.ok ? j * g.nbx + (i >> 5) : 0;
  s.sm = r * PW + x;
  const int I = i + 1, J = j + 1, sx = I & 1, sy = J & 1;
  s.oa = (((J - sy) >> 1) - 1 - T.cr0) * CX + (((I - sx) >> 1) - 1 - T.cx0);
  s.ob = (((J + sy) >> 1) - 1 - T.cr0) * CX + (((I + sx) >> 1) - 1 - T.cx0);
  s.cp = code_pos(i & 31, W);
  return s;
}

// coarse planes of the P_l parents of fine plane kf (3-D): K = kf + 1 odd has
// parents in planes kf/2 - 1 and kf/2, K even in (kf - 1)/2 only
template <int DIM>
__device__ __forceinline__ void zparents(int kf, int &za, int &zb) {
  if (DIM == 2) {
    za = zb = 0;
  } else if (kf & 1) {
    za = zb = (kf - 1) >> 1;
  } else {
    za = (kf >> 1) - 1;
    zb = kf >> 1;
  }
}

// (P_l t) at a slot from a ring, on the ring's grid minus one
template <class V>
__device__ __forceinline__ V ring_p(const V *ring, const Slot &s, int za, int zb) {
  return ring[(za & 3) * CRX + s.oa] + ring[(zb & 3) * CRX + s.ob];
}

// One ring entry per thread (tid < CRX): a fixed coarse (ci, cj) column.
struct Stager {
  bool on, ok;
  int bip;          // block index inside a coarse plane
  int cj, ci;       // coarse row and column
  long long v;      // loaded value, not yet stored
  int gb;           // loaded descriptor
};

__device__ __forceinline__ Stager make_stager(const Geo &gc, const Tile &T, int tid) {
  Stager s;
  s.on = tid < CRX;
  const int r = tid / CX, x = tid - (tid / CX) * CX;
  const int cj = T.cr0 + r, ci = T.cx0 + x;
  s.ok = s.on && (unsigned)ci < (unsigned)gc.n && (unsigned)cj < (unsigned)gc.n;
  s.bip = s.ok ? cj * gc.nbx + (ci >> 5) : 0;
  s.cj = s.ok ? cj : 0;
  s.ci = s.ok ? ci : 0;
  s.v = 0;
  s.gb = 0;
  return s;
}

__device__ __forceinline__ void stage_load(Stager &s, const Tmp &t, const Geo &gc, int c) {
  s.v = 0;
  s.gb = 0;
  if (s.ok && (unsigned)c < (unsigned)gc.nz) {
    s.gb = __ldg(t.gb + c * gc.n * gc.nbx + s.bip);
    s.v = __ldg(t.v + (long long)(c * gc.n + s.cj) * gc.R + s.ci);
  }
}

// Two-level ring entries (x = s + P x_(l-2), see Tmp2).  A second, smaller
// ring holds the level-(l-2) parents of the tile's level-(l-1) window (5 rows x
// 11 columns per plane, 4 planes) on the ring's grid; a level-(l-1) entry is
// then its section code plus one or two reads of that ring.  The global loads
// of a staging step go into shared memory by cp.async one step ahead (two
// buffers), so that two planes of compute hide their latency.  Steps are
// consecutive level-(l-1) planes c; step c also stages level-(l-2) plane
// (c + 1) / 2 exactly when c is odd (the first plane its successor needs).
// The tile's footprint bounds put every part of an entry on or above the
// ring's grid and within the ring's integer type, so the shifts are
// unchecked; a parent on the ring's grid is even (its own grid is at least one
// above), so the half sum of two is exact.
constexpr int BR2 = 5, BX2 = 11, BRX2 = BR2 * BX2;

struct Two2 {
  unsigned e4[2][CRX], w0[2][CRX], w1[2][CRX];  // raw section words of the level-(l-1) entries
  int par[CRX];                                 // each entry's parents in the level-(l-2) ring:
                                                // in-plane offsets a | b << 8, odd in x or y << 16
  long long bv[2][BRX2];                        // raw level-(l-2) values
  int bg[2][BRX2];                              // and their block descriptors
  long long rb[4 * BRX2];                       // the level-(l-2) ring, on the ring's grid
};

// the threads that stage the level-(l-2) ring: the last two warps, which
// stage no level-(l-1) entry
constexpr int TB0 = NT - 64;
static_assert(CRX <= TB0 && BRX2 <= 64, "staging thread ranges");

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// level-(l-2) window origin of a tile: the lowest parent row / column of its
// level-(l-1) window
__device__ __forceinline__ int two_row0(const Tile &T) { return (T.cr0 >> 1) - 1; }
__device__ __forceinline__ int two_col0(const Tile &T) { return (T.cx0 >> 1) - 1; }

// issue the loads of level-(l-1) plane c (if lc) and of level-(l-2) plane p
// (if lb) into buffer buf
__device__ __forceinline__ void two_issue(const Stager &s, const Tmp2 &t, const Geo &gc, const Tile &T, bool lc,
                                          int c, bool lb, int p, Two2 &sh, int tid, int buf) {
  if (lc && s.ok && (unsigned)c < (unsigned)gc.nz) {
    const int blk = c * gc.n * gc.nbx + s.bip;  // block counts of a level fit in int
    // exponent arrays are allocated in whole 16-byte units, so the aligned word is inside
    cp_async4(&sh.e4[buf][tid], t.s.exps + (blk & ~3));
    const int W = t.s.W, pos = (s.ci & 31) * W;
    const uint32_t *wp = t.s.words + (long long)blk * W + (pos >> 5);
    cp_async4(&sh.w0[buf][tid], wp);
    if ((pos & 31) + W > 32) cp_async4(&sh.w1[buf][tid], wp + 1);
  }
  const int tb = tid - TB0;
  if (lb && (unsigned)tb < (unsigned)BRX2) {
    const Geo &g = t.gb;
    const int bi = two_col0(T) + tb % BX2, bj = two_row0(T) + tb / BX2;
    if (inside(g, bi, bj, p)) {
      cp_async4(&sh.bg[buf][tb], t.b.gb + blk_index(g, bi, bj, p));
      cp_async8(&sh.bv[buf][tb], t.b.v + ((long long)p * g.n + bj) * g.R + bi);
    } else {
      sh.bg[buf][tb] = 0;
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// level-(l-2) plane p (if lb) into its ring, and level-(l-1) plane c (if lc)
// into the ring, from buffer buf (its parents' planes were stored by earlier
// steps, before a CTA barrier); ahead: a later step's loads are in flight.
// bad: the invalid code -2^(W-1)
template <int DIM, class V>
__device__ __forceinline__ void two_store(const Stager &s, const Tmp2 &t, const Geo &gc, const Tile &T, bool lc,
                                          int c, bool lb, int p, Two2 &sh, V *ring, int G1, int tid, bool &bad,
                                          int buf, bool ahead) {
  if (ahead) asm volatile("cp.async.wait_group 1;" ::: "memory");
  else cp_async_wait_all();
  const int tb = tid - TB0;
  if (lb && (unsigned)tb < (unsigned)BRX2) {
    const int gbv = sh.bg[buf][tb];
    sh.rb[(p & 3) * BRX2 + tb] = (gbv & 0xff) ? shl_fast(sh.bv[buf][tb], (gbv >> 8) - G1) : 0;
  }
  if (!lc || !s.on) return;
  long long x = 0;
  if (s.ok && (unsigned)c < (unsigned)gc.nz) {
    const int blk = c * gc.n * gc.nbx + s.bip;
    const int e = (int)(signed char)(sh.e4[buf][tid] >> (8 * (blk & 3)));
    const int W = t.s.W, off = ((s.ci & 31) * W) & 31;
    if (e != -128) {
      const uint32_t bits = __funnelshift_r(sh.w0[buf][tid], off + W > 32 ? sh.w1[buf][tid] : 0u, off);
      const int q = ((int)(bits << (32 - W))) >> (32 - W);
      bad |= (unsigned)q == (0xffffffffu << (W - 1));
      x = shl_fast(q, e - W + 1 - G1);
    }
    // P x_(l-2): parents (I -+ s)/2 of the 1-based node, in the level-(l-2) ring
    const int par = sh.par[tid], K = c + 1, sz = DIM == 3 ? (K & 1) : 0;
    const int ka = DIM == 3 ? ((K - sz) >> 1) - 1 : 0, kb = DIM == 3 ? ((K + sz) >> 1) - 1 : 0;
    const long long pa = sh.rb[(ka & 3) * BRX2 + (par & 0xff)];
    if ((par >> 16) | sz) x += (pa + sh.rb[(kb & 3) * BRX2 + ((par >> 8) & 0xff)]) >> 1;
    else x += pa;
  }
  ring[(c & 3) * CRX + tid] = (V)x;
}

// The ring planes before the first decode: level-(l-1) planes c0 .. c1 and the
// level-(l-2) planes their parents lie in (and the next one), the latter first
// with a CTA barrier between; then the loads of the first step of the march
// (plane c1 + 1) are issued.
template <int DIM, class V>
__device__ __forceinline__ void two_prologue(const Stager &s, const Tmp2 &t, const Geo &gc, const Tile &T, int c0,
                                             int c1, Two2 &sh, V *ring, int G1, int tid, bool &bad) {
  if (s.on && s.ok) {  // the entry's parents in the level-(l-2) ring (fixed per tile)
    const int I = s.ci + 1, J = s.cj + 1, sx = I & 1, sy = J & 1;
    const int r0 = two_row0(T), q0 = two_col0(T);
    const int oa = (((J - sy) >> 1) - 1 - r0) * BX2 + ((I - sx) >> 1) - 1 - q0;
    const int ob = (((J + sy) >> 1) - 1 - r0) * BX2 + ((I + sx) >> 1) - 1 - q0;
    sh.par[tid] = oa | ob << 8 | (sx | sy) << 16;
  }
  const int p0 = DIM == 3 ? (c0 >> 1) - 1 : 0, p1 = DIM == 3 ? (c1 + 1) >> 1 : 0;
  for (int p = p0; p <= p1; p++) {
    two_issue(s, t, gc, T, false, 0, true, p, sh, tid, 0);
    two_store<DIM>(s, t, gc, T, false, 0, true, p, sh, ring, G1, tid, bad, 0, false);
  }
  __syncthreads();
  for (int c = c0; c <= c1; c++) {
    two_issue(s, t, gc, T, true, c, false, 0, sh, tid, 0);
    two_store<DIM>(s, t, gc, T, true, c, false, 0, sh, ring, G1, tid, bad, 0, false);
  }
  if (DIM == 3) two_issue(s, t, gc, T, true, c1 + 1, (c1 + 1) & 1, (c1 + 2) >> 1, sh, tid, (c1 + 1) & 1);
}

// one staging step of the march for level-(l-1) plane c: issue the next
// step's loads (before the plane's compute) / store plane c (after it)
__device__ __forceinline__ void two_step_issue(const Stager &s, const Tmp2 &t, const Geo &gc, const Tile &T, int c,
                                               Two2 &sh, int tid) {
  two_issue(s, t, gc, T, true, c + 1, (c + 1) & 1, (c + 2) >> 1, sh, tid, (c + 1) & 1);
}
template <int DIM, class V>
__device__ __forceinline__ void two_step_store(const Stager &s, const Tmp2 &t, const Geo &gc, const Tile &T, int c,
                                               Two2 &sh, V *ring, int G1, int tid, bool &bad) {
  two_store<DIM>(s, t, gc, T, true, c, c & 1, (c + 1) >> 1, sh, ring, G1, tid, bad, c & 1, true);
}

// the staged value on the ring's grid G1 (a 32-bit ring only where the caller
// proved every value below 2^31 on G1)
template <class V>
__device__ __forceinline__ void stage_store(const Stager &s, V *ring, int c, int G1, int tid) {
  if (s.on) ring[(c & 3) * CRX + tid] = (V)((s.gb & 0xff) ? shl_fast(s.v, (s.gb >> 8) - G1) : 0);
}

// ------------------------------------------------------------------ footprint bounds
// Bounds of a two-level temporary over the coarse footprint planes ck0..ck1,
// rows cj0..cj1, blocks cb0..cb1 of its level (all inside it): the section's
// block exponents there and the lower temporary's descriptors over their
// parents; G = min(G_s, G_b - 1), |x| < 2^(max(M_s, M_b) + 1).  CTA-cooperative:
// atomics into sm[0] (G) and sm[1] (M), which the caller has initialised.
__device__ __forceinline__ void bounds2_scan(const Tmp2 &t, const Geo &gc, int ck0, int ck1, int cj0, int cj1,
                                             int cb0, int cb1, int *sm, int tid) {
  int G = GRID_NONE, M = MAG_NONE;
  {
    const int nb = cb1 - cb0 + 1, nr = cj1 - cj0 + 1, np = ck1 - ck0 + 1, cnt = nb * nr * np;
    for (int idx = tid; idx < cnt; idx += NT) {
      const int kk = ck0 + idx / (nb * nr), rem = idx % (nb * nr);
      const int e = __ldg(t.s.exps + ((long long)kk * gc.n + cj0 + rem / nb) * gc.nbx + cb0 + rem % nb);
      if (e != -128) {
        G = imin(G, e - t.s.W + 1);
        M = imax(M, e);
      }
    }
  }
  {  // parents of coarse index c lie in c / 2 - 1 .. c / 2 of the level below
    const Geo &gb = t.gb;
    const int k0 = gc.nz > 1 ? imax(0, ck0 / 2 - 1) : 0, k1 = gc.nz > 1 ? imin(gb.nz - 1, ck1 / 2) : 0;
    const int j0 = imax(0, cj0 / 2 - 1), j1 = imin(gb.n - 1, cj1 / 2);
    const int i0 = imax(0, (cb0 * 32) / 2 - 1), i1 = imin(gb.n - 1, imin(gc.n - 1, cb1 * 32 + 31) / 2);
    const int b0 = i0 >> 5, b1 = i1 >> 5;
    const int nb = b1 - b0 + 1, nr = j1 - j0 + 1, np = k1 - k0 + 1;
    if (nb > 0 && nr > 0 && np > 0) {
      const int cnt = nb * nr * np;
      for (int idx = tid; idx < cnt; idx += NT) {
        const int kk = k0 + idx / (nb * nr), rem = idx % (nb * nr);
        const int gbv = __ldg(t.b.gb + ((long long)kk * gb.n + j0 + rem / nb) * gb.nbx + b0 + rem % nb);
        if (gbv & 0xff) {
          G = imin(G, gb_grid(gbv) - 1);
          M = imax(M, gb_mag(gbv));
        }
      }
    }
  }
  if (G < GRID_NONE / 2) atomicMin(sm, G);
  if (M > MAG_NONE / 2) atomicMax(sm + 1, M + 1);
}

struct Bounds {
  int G;  // finest grid (GRID_NONE: all zero)
  int M;  // |v| < 2^M (MAG_NONE: all zero)
};

// Scans the CTA footprint: the exponents of section s over planes k0-1..k1,
// rows j0-1..j0+TY and blocks bx-1..bx+1, and the descriptors of the coarse
// temporaries t and u over the coarse planes, rows and blocks P_l reads.
// sm: 6 ints; ends with a CTA barrier.
// t2 / u2 (if not null): t / u are two-level temporaries (Tmp2) instead.
template <int DIM>
__device__ __forceinline__ void footprint_bounds(const Geo &g, const Geo &gc, const Tile &T, const Sec &s,
                                                 bool has_s, const Tmp &t, bool has_t, const Tmp &u, bool has_u,
                                                 int *sm, Bounds &bs, Bounds &bt, Bounds &bu,
                                                 const Tmp2 *t2 = nullptr, const Tmp2 *u2 = nullptr) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid == 0) {
    sm[0] = sm[2] = sm[4] = GRID_NONE;
    sm[1] = sm[3] = sm[5] = MAG_NONE;
  }
  __syncthreads();
  const int klo = DIM == 3 ? T.k0 - 1 : 0, khi = DIM == 3 ? T.k1 : 0;
  if (has_s) {
    int G = GRID_NONE, M = MAG_NONE;
    const int per = (TY + 2) * 3, cnt = (khi - klo + 1) * per;
    for (int idx = tid; idx < cnt; idx += NT) {
      const int kk = klo + idx / per, rem = idx - (idx / per) * per;
      const int jj = T.j0 - 1 + rem / 3, bb = T.bx - 1 + rem % 3;
      if ((unsigned)kk < (unsigned)g.nz && (unsigned)jj < (unsigned)g.n && (unsigned)bb < (unsigned)g.nbx) {
        const int e = __ldg(s.exps + ((long long)kk * g.n + jj) * g.nbx + bb);
        if (e != -128) {
          G = imin(G, e - s.W + 1);
          M = imax(M, e);
        }
      }
    }
    if (G < GRID_NONE / 2) atomicMin(sm, G);
    if (M > MAG_NONE / 2) atomicMax(sm + 1, M);
  }
  if (has_t || has_u) {
    const int cj0 = imax(0, T.cr0), cj1 = imin(gc.n - 1, T.cr0 + CR - 1);
    const int ck0 = DIM == 3 ? imax(0, (klo - 1) >> 1) : 0;
    const int ck1 = DIM == 3 ? imin(gc.nz - 1, khi >> 1) : 0;
    const int cb0 = imax(0, T.cx0) >> 5, cb1 = imin(gc.n - 1, T.cx0 + CX - 1) >> 5;
    const int nb = cb1 - cb0 + 1, nr = cj1 - cj0 + 1, np = ck1 - ck0 + 1;
    if (nb > 0 && nr > 0 && np > 0) {
      const int cnt = nb * nr * np;
      for (int which = 0; which < 2; which++) {
        if (!(which ? has_u : has_t)) continue;
        const Tmp2 *x2 = which ? u2 : t2;
        if (x2) {
          bounds2_scan(*x2, gc, ck0, ck1, cj0, cj1, cb0, cb1, sm + 2 + 2 * which, tid);
          continue;
        }
        const int *xgb = which ? u.gb : t.gb;
        int G = GRID_NONE, M = MAG_NONE;
        for (int idx = tid; idx < cnt; idx += NT) {
          const int kk = ck0 + idx / (nb * nr), rem = idx % (nb * nr);
          const int jj = cj0 + rem / nb, bb = cb0 + rem % nb;
          const int gbv = __ldg(xgb + ((long long)kk * gc.n + jj) * gc.nbx + bb);
          if (gbv & 0xff) {
            G = imin(G, gb_grid(gbv));
            M = imax(M, gb_mag(gbv));
          }
        }
        if (G < GRID_NONE / 2) atomicMin(sm + 2 + 2 * which, G);
        if (M > MAG_NONE / 2) atomicMax(sm + 3 + 2 * which, M);
      }
    }
  }
  __syncthreads();
  bs.G = sm[0];
  bs.M = sm[1];
  bt.G = sm[2];
  bt.M = sm[3];
  bu.G = sm[4];
  bu.M = sm[5];
}

// Operand bounds: F = s + P t on grid GF = min(G_s, G_t - 1), |F| < 2^MF.
__device__ __forceinline__ Bounds operand_of(const Bounds &bs, const Bounds &bt) {
  Bounds b;
  b.G = imin(bs.G, bt.G < GRID_NONE / 2 ? bt.G - 1 : GRID_NONE);
  const int M = imax(bs.M, bt.M);
  b.M = M > MAG_NONE / 2 ? M + 1 : MAG_NONE;
  return b;
}

// R_l = P_l^T on grid G-1: an all-even node gives 2d to its coarse node, any
// other node gives d to each of the two coarse nodes (I -+ e_S)/2.
template <int DIM>
__device__ __forceinline__ void scatter_restrict(unsigned long long *acc, const Geo &gc, int I, int J, int K,
                                                 long long d) {
  Parents<DIM> p(I, J, K);
  if (!p.two) {
    atomicAdd(acc + ((long long)p.ka * gc.n + p.ja) * gc.R + p.ia, (unsigned long long)(2 * d));
    return;
  }
  if (inside(gc, p.ia, p.ja, p.ka))
    atomicAdd(acc + ((long long)p.ka * gc.n + p.ja) * gc.R + p.ia, (unsigned long long)d);
  if (inside(gc, p.ib, p.jb, p.kb))
    atomicAdd(acc + ((long long)p.kb * gc.n + p.jb) * gc.R + p.ib, (unsigned long long)d);
}

}  // namespace cmg
