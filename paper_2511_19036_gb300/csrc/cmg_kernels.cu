// Compact FMG kernels for GB300 (sm_103a).
//
// Every kernel reads its operands in the compact BFP form (Sec. 6.1.3 of the
// paper), computes exactly in int64 fixed point on locally chosen grids (see
// cmg_device.cuh), and writes BFP sections rounded to nearest-even (Sec. 4).
// The stencil kernels march a CTA through z, keeping three planes of the
// decoded stencil operand in shared memory (one x-block of 32 plus a one-node
// halo, by TY rows plus halo); one warp owns one output block row.
//
// Kernels (one launch covers one level):
//   k_sweep     weighted-Jacobi sweep y~ <- round(y~ + c (rc - A (y~ + P w_(l-1))))
//               (Algorithm 1 smoothing step on eq. cfas), with optional fused
//               correction u~ <- round(u~ + y~) (Algorithm 3), w_l = y~ + z_l and
//               u^_l = u~_l + P u^_(l-1) for the next level / residual
//   k_residual  Algorithm 2 on the finest level: t = f - A (u~_L + P u^_(L-1)),
//               r = round(t); optional first Jacobi sweep from y~ = 0 fused in,
//               or t^ (Table 1 width) stored for the restriction chain
//   k_restrict  d = rc - A y~ (or d = rc) scattered as R_l d into an int64
//               accumulator by exact, order-free integer atomics
//   k_acc_encode round an accumulator into BFP section(s) (+ optional first sweep)
//   k_coarse    the single unknown of level 1
//   k_repack    FMG level step: widen a section by appending zero bits
//   k_chain, k_axpy, k_decode_solution: unfused pieces for step-wise use
//   k_encode_f64, k_decode_f64: stand-alone codec
#include <cuda_runtime.h>

#include <cstdint>

#include "cmg_device.cuh"
#include "cmg_kernels.h"

namespace cmg {

__device__ inline bool first_cta() { return blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0; }

// ------------------------------------------------------------------ stencil operand tile
// The stencil operand F = [BFP section s] + [P_l t] (t a coarse temporary) is
// held for three z-planes in shared memory on one grid GF per CTA.  The coarse
// values that P_l needs are staged once per CTA, per coarse plane, in a ring of
// three coarse planes (CR x CX values around the tile), already on grid GF + 1,
// so a fine value of P_l t is two shared-memory reads.
constexpr int CR = 7;   // coarse rows feeding fine rows j0-1 .. j0+TY
constexpr int CX = 19;  // coarse columns feeding fine columns x0-1 .. x0+32

struct Operand {
  int has_s, has_t;
  Sec s;
  Tmp t;
};

struct TileBounds {
  int G;  // grid of F over the CTA footprint
  int M;  // |F| < 2^M over the footprint
};

// footprint scan: planes k0-1..k1, rows j0-1..j0+TY, x x0-1..x0+32.  sm: two
// shared ints set to (GRID_NONE, MAG_NONE) before a barrier.
template <int DIM>
__device__ TileBounds operand_bounds(const Operand &o, const Geo &g, const Geo &gc, int bx, int j0, int k0, int k1,
                                     int *sm) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
  int G = GRID_NONE, M = MAG_NONE;
  const int klo = DIM == 3 ? k0 - 1 : 0, khi = DIM == 3 ? k1 : 0;
  if (o.has_s) {
    const int per = (TY + 2) * 3, cnt = (khi - klo + 1) * per;
    for (int idx = tid; idx < cnt; idx += NT) {
      int kk = klo + idx / per, rem = idx - (idx / per) * per;
      int jj = j0 - 1 + rem / 3, bb = bx - 1 + rem % 3;
      if ((unsigned)kk < (unsigned)g.nz && (unsigned)jj < (unsigned)g.n && (unsigned)bb < (unsigned)g.nbx) {
        int e = __ldg(o.s.exps + ((long long)kk * g.n + jj) * g.nbx + bb);
        if (e != -128) {
          G = imin(G, e - o.s.W + 1);
          M = imax(M, e);
        }
      }
    }
  }
  if (o.has_t) {
    const int x0 = bx * 32;
    const int cj0 = imax(0, ((j0 - 1) >> 1) - 1), cj1 = imin(gc.n - 1, ((j0 + TY + 2) >> 1) - 1);
    const int ck0 = DIM == 3 ? imax(0, ((klo - 1) >> 1)) : 0;
    const int ck1 = DIM == 3 ? imin(gc.nz - 1, khi >> 1) : 0;
    const int cx0 = imax(0, ((x0 - 1) >> 1) - 1), cx1 = imin(gc.n - 1, ((x0 + 34) >> 1) - 1);
    const int cb0 = cx0 >> 5, cb1 = cx1 >> 5;
    const int nb = cb1 - cb0 + 1, nr = cj1 - cj0 + 1, np = ck1 - ck0 + 1;
    if (nb > 0 && nr > 0 && np > 0) {
      const int cnt = nb * nr * np;
      for (int idx = tid; idx < cnt; idx += NT) {
        int kk = ck0 + idx / (nb * nr), rem = idx % (nb * nr);
        int jj = cj0 + rem / nb, bb = cb0 + rem % nb;
        int gbv = __ldg(o.t.gb + ((long long)kk * gc.n + jj) * gc.nbx + bb);
        if (gbv & 0xff) {
          G = imin(G, gb_grid(gbv) - 1);
          M = imax(M, gb_mag(gbv));
        }
      }
    }
  }
  if (G < GRID_NONE / 2) atomicMin(sm, G);
  if (M > MAG_NONE / 2) atomicMax(sm + 1, M);
  __syncthreads();
  TileBounds b;
  b.G = sm[0];
  b.M = sm[1] > MAG_NONE / 2 ? sm[1] + 1 : MAG_NONE;  // s + P t: one more bit
  return b;
}

// stage coarse plane c (0-based) of t into ring slot c % 3, on grid G1
template <int DIM>
__device__ void stage_coarse(long long (*C)[CR][CX], const Tmp &t, const Geo &gc, int c, int cr0, int cx0,
                             int G1) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int idx = tid; idx < CR * CX; idx += NT) {
    const int r = idx / CX, x = idx - r * CX;
    const int cj = cr0 + r, ci = cx0 + x;
    long long v = 0;
    if (inside(gc, ci, cj, c)) {
      const int gbv = __ldg(t.gb + blk_index(gc, ci, cj, c));
      if (gbv & 0xff) v = shl(__ldg(t.v + ((long long)c * gc.n + cj) * gc.R + ci), (gbv >> 8) - G1);
    }
    C[c % 3][r][x] = v;
  }
}

// (P_l t) at fine node (I, J, K) from the staged ring, on grid G1 - 1
template <int DIM>
__device__ __forceinline__ long long p_staged(const long long (*C)[CR][CX], int I, int J, int K, int cr0, int cx0,
                                              int ncz) {
  Parents<DIM> p(I, J, K);
  long long a = 0, b = 0;
  if ((unsigned)p.ka < (unsigned)ncz) a = C[p.ka % 3][p.ja - cr0][p.ia - cx0];
  if (!p.two) return 2 * a;
  if ((unsigned)p.kb < (unsigned)ncz) b = C[p.kb % 3][p.jb - cr0][p.ib - cx0];
  return a + b;
}

// BFP value of section s at (i, j, k) on grid G, for a row block whose index and
// exponent the caller already has (warp-uniform); zero for padding lanes
__device__ __forceinline__ long long row_val(const Sec &s, long long blk, int e, int lane, int G) {
  if (e == -128) return 0;
  int q = code_at(s.words + blk * s.W, s.W, lane);
  return shl((long long)q, e - s.W + 1 - G);
}

// Fill smem plane (TY+2 rows x 34 columns) with F at fine plane k.  Warp ty owns
// row ty+1 (its own output row); warps 0 and 1 also fill halo rows 0 and TY+1,
// warp 2 the two halo columns.  Returns the s-part of this warp's own row.
template <int DIM>
__device__ __forceinline__ long long load_plane(long long (*Fs)[34], const long long (*C)[CR][CX], const Operand &o,
                                                const Geo &g, const Geo &gc, int bx, int j0, int k, int G, int cr0,
                                                int cx0) {
  const int lane = threadIdx.x, ty = threadIdx.y, x0 = bx * 32;
  long long own = 0;
  const bool kin = (unsigned)k < (unsigned)g.nz;
#pragma unroll
  for (int pass = 0; pass < 2; pass++) {
    int r;
    if (pass == 0) r = ty + 1;
    else if (ty < 2) r = ty == 0 ? 0 : TY + 1;
    else break;
    const int j = j0 - 1 + r, i = x0 + lane;
    long long sv = 0, v = 0;
    if (kin && (unsigned)j < (unsigned)g.n) {  // warp-uniform
      if (o.has_s) {
        const long long blk = ((long long)k * g.n + j) * g.nbx + bx;
        sv = row_val(o.s, blk, __ldg(o.s.exps + blk), lane, G);
      }
      if (i < g.n) {
        v = sv;
        if (o.has_t) v += p_staged<DIM>(C, i + 1, j + 1, k + 1, cr0, cx0, gc.nz);
      } else {
        sv = 0;
      }
    }
    Fs[r][lane + 1] = v;
    if (pass == 0) own = sv;
  }
  if (ty == 2) {  // halo columns x0-1 and x0+32 of all TY+2 rows
    const int r = lane >> 1, side = lane & 1;
    if (r < TY + 2) {
      const int j = j0 - 1 + r, i = side ? x0 + 32 : x0 - 1;
      long long v = 0;
      if (kin && inside(g, i, j, k)) {
        if (o.has_s) {
          const long long blk = ((long long)k * g.n + j) * g.nbx + (i >> 5);
          v = row_val(o.s, blk, __ldg(o.s.exps + blk), i & 31, G);
        }
        if (o.has_t) v += p_staged<DIM>(C, i + 1, j + 1, k + 1, cr0, cx0, gc.nz);
      }
      Fs[r][side ? 33 : 0] = v;
    }
  }
  return own;
}

template <int DIM>
__device__ __forceinline__ long long stencil(const long long (*Fp)[34], const long long (*Fc)[34],
                                             const long long (*Fn)[34], int ty, int lane) {
  long long S = (long long)(2 * DIM) * Fc[ty + 1][lane + 1] - Fc[ty + 1][lane] - Fc[ty + 1][lane + 2] -
                Fc[ty][lane + 1] - Fc[ty + 2][lane + 1];
  if (DIM == 3) S -= Fp[ty + 1][lane + 1] + Fn[ty + 1][lane + 1];
  return S;
}

// Drives the z-march of a stencil kernel: stages coarse planes as the fine
// planes advance and fills the operand ring.  body(k, sp, sc, sn, own) runs for
// every output plane k with the slots of planes k-1, k, k+1.
template <int DIM, typename Body>
__device__ __forceinline__ void march(long long (*F)[TY + 2][34], long long (*C)[CR][CX], const Operand &op,
                                      const Geo &g, const Geo &gc, int bx, int j0, int k0, int k1, int GF,
                                      Body body) {
  const int x0 = bx * 32;
  const int cr0 = ((j0 - 1) >> 1) - 1, cx0 = ((x0 - 1) >> 1) - 1;
  const int G1 = GF + 1;
  int staged_hi = -1;
  if (op.has_t) {
    if (DIM == 3) {
      for (int c = imax(0, (k0 - 2) >> 1); c <= (k0 >> 1) && c < gc.nz; c++) {
        stage_coarse<DIM>(C, op.t, gc, c, cr0, cx0, G1);
        staged_hi = c;
      }
    } else {
      stage_coarse<DIM>(C, op.t, gc, 0, cr0, cx0, G1);
      staged_hi = 0;
    }
    __syncthreads();
  }
  long long own_next = 0;
  if (DIM == 3) load_plane<DIM>(F[0], C, op, g, gc, bx, j0, k0 - 1, GF, cr0, cx0);
  own_next = load_plane<DIM>(F[1], C, op, g, gc, bx, j0, k0, GF, cr0, cx0);
  for (int k = k0; k < k1; k++) {
    const int sp = (k - k0) % 3, sc = (k - k0 + 1) % 3, sn = (k - k0 + 2) % 3;
    const long long own = own_next;
    if (DIM == 3) {
      const int kf = k + 1;
      if (op.has_t && kf < g.nz && (kf >> 1) > staged_hi && (kf >> 1) < gc.nz) {
        stage_coarse<DIM>(C, op.t, gc, kf >> 1, cr0, cx0, G1);
        staged_hi = kf >> 1;
        __syncthreads();
      }
      own_next = load_plane<DIM>(F[sn], C, op, g, gc, bx, j0, kf, GF, cr0, cx0);
    }
    __syncthreads();
    body(k, sp, sc, sn, own);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ sweep
template <int DIM>
__global__ void __launch_bounds__(NT, 2) k_sweep(SweepArgs a) {
  __shared__ long long F[3][TY + 2][34];
  __shared__ long long C[3][CR][CX];
  __shared__ uint32_t pk[TY][33];
  __shared__ int smy[2], smu[2], smg[2];
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const int bx = blockIdx.x, j0 = blockIdx.y * TY, k0 = blockIdx.z * ZC;
  const int k1 = imin(g.nz, k0 + ZC), x0 = bx * 32;
  if (tid == 0) {
    smy[0] = smy[1] = smu[0] = smu[1] = 0;
    smg[0] = GRID_NONE;
    smg[1] = MAG_NONE;
  }
  __syncthreads();
  Operand op;
  op.has_s = a.has_y;
  op.s = a.y_in;
  op.has_t = a.has_z;
  op.t = a.wc;
  const TileBounds tb = operand_bounds<DIM>(op, g, a.gc, bx, j0, k0, k1, smg);
  const int GF = tb.G, MF = tb.M;
  const int sA = (DIM - 2) * g.l;
  const int GA = GF - sA, MA = MF + 4 - sA;  // |A F| < 2^MA on grid GA
  if (tid == 0 && GF < GRID_NONE / 2 && MF + 4 - GF > 62) flag_range(a.err, 101, MF + 4, GF);
  bool ovf = false;
  MetaAcc my, mu;
  my.init();
  mu.init();
  const int j = j0 + ty, i = x0 + lane;
  const bool rowok = j < g.n, pt = rowok && i < g.n;
  march<DIM>(F, C, op, g, a.gc, bx, j0, k0, k1, GF, [&](int k, int sp, int sc, int sn, long long own) {
    if (!rowok) return;  // warp-uniform: one warp per row
    const long long blk = ((long long)k * g.n + j) * g.nbx + bx;
    const int erc = __ldg(a.rc.exps + blk);
    const int Gres = imin(blk_lsb(erc, a.rc.W), GA);
    const int Mres = imax(erc == -128 ? MAG_NONE : erc, MA) + 1;
    const int Gcr = Gres + a.c_exp;
    const int Gy = a.has_y ? imin(GF, Gcr) : Gcr;
    long long S = pt ? stencil<DIM>(F[sp], F[sc], F[sn], ty, lane) : 0;
    long long ynew;
    // static range of this block's computation (warp-uniform); a block whose
    // bounds do not fit takes the per-value checked path instead
    if (Gres >= GRID_NONE / 2 || (Mres - Gres <= 62 - a.cbits && Mres + a.cbits + a.c_exp - Gy <= 61 &&
                                  (!a.has_y || MF - Gy <= 61))) {
      long long res = row_val(a.rc, blk, erc, lane, Gres) - shl(S, GA - Gres);
      ynew = shl(res * a.c_num, Gcr - Gy);
      if (a.has_y) ynew += shl(own, GF - Gy);
    } else {
      if (erc != -128 && erc - Gres > 61) ovf = true;
      long long res = row_val(a.rc, blk, erc, lane, Gres) - shl_ck(S, GA - Gres, ovf);
      ck62(res, ovf);
      ynew = shl_ck(mul_ck(res, a.c_num, a.cbits, ovf), Gcr - Gy, ovf);
      if (a.has_y) ynew += shl_ck(own, GF - Gy, ovf);
      ck62(ynew, ovf);
    }
    int e, sh;
    int q = encode_block(ynew, Gy, a.Wy, e, sh, a.err);
    long long yr = rounded_value(ynew, q, sh);
    if (a.write_y) {
      pack_block(q, a.Wy, pk[ty], a.y_out.words + blk * a.Wy);
      if (lane == 0) {
        a.y_out.exps[blk] = (int8_t)e;
        my.add(e);
      }
    }
    long long ur = 0;
    int Gu = Gy;
    if (a.corr) {
      const int eu0 = __ldg(a.u_in.exps + blk);
      Gu = imin(blk_lsb(eu0, a.u_in.W), Gy);
      if (e != -128 || eu0 != -128)
        if (imax(eu0 == -128 ? MAG_NONE : eu0, e) + 1 - Gu > 62) ovf = true;
      long long usum = row_val(a.u_in, blk, eu0, lane, Gu) + shl(yr, Gy - Gu);
      int eu, su;
      int qu = encode_block(usum, Gu, a.u_out.W, eu, su, a.err);
      ur = rounded_value(usum, qu, su);
      pack_block(qu, a.u_out.W, pk[ty], a.u_out.words + blk * a.u_out.W);
      if (lane == 0) {
        a.u_out.exps[blk] = (int8_t)eu;
        mu.add(eu);
      }
    }
    const long long p = ((long long)k * g.n + j) * g.R + i;
    if (a.write_w) {  // w_l = y~' + P w_(l-1); P w_(l-1) = F - y~ at this node
      const int Gw = imin(Gy, GF);
      long long w;
      if (imax(MF, e == -128 ? MAG_NONE : e) + 1 - Gw <= 62) {
        w = shl(yr, Gy - Gw);
        if (a.has_z && pt) w += shl(F[sc][ty + 1][lane + 1] - (a.has_y ? own : 0), GF - Gw);
      } else {
        w = shl_ck(yr, Gy - Gw, ovf);
        if (a.has_z && pt) w += shl_ck(F[sc][ty + 1][lane + 1] - (a.has_y ? own : 0), GF - Gw, ovf);
        ck62(w, ovf);
      }
      store_tmp_block(w, Gw, a.w_out.v + p, a.w_out.gb + blk, pt, ovf);
    }
    if (a.write_uh) {  // u^_l = u~_l' + P u^_(l-1)
      int gu = (pt && a.has_uhc) ? prolong_grid<DIM>(a.uhc, a.gc, i + 1, j + 1, k + 1) : GRID_NONE;
      const int Guh = imin(Gu, __reduce_min_sync(0xffffffffu, gu));
      long long uh = shl_ck(ur, Gu - Guh, ovf);
      if (pt && a.has_uhc) uh += prolong_tmp<DIM>(a.uhc, a.gc, i + 1, j + 1, k + 1, Guh, ovf);
      ck62(uh, ovf);
      store_tmp_block(uh, Guh, a.uh_out.v + p, a.uh_out.gb + blk, pt, ovf);
    }
  });
  ovf_flush(ovf, a.err, 102);
  if (a.write_y) meta_flush(my, a.y_out.meta, smy);
  if (a.corr) meta_flush(mu, a.u_out.meta, smu);
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

// F_q at level-L node (I, J, K): sum_t prod_a T[t][a][I_a * stride - 1], rounded
// to nearest-even after dropping fsh bits.
template <int DIM>
__device__ __forceinline__ long long rhs_at(const ResidArgs &a, int I, int J, int K) {
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

template <int DIM>
__global__ void __launch_bounds__(NT, 2) k_residual(ResidArgs a) {
  __shared__ long long F[3][TY + 2][34];
  __shared__ long long C[3][CR][CX];
  __shared__ uint32_t pk[TY][33];
  __shared__ int smr[2], smy[2], smt[2], smg[2];
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const int bx = blockIdx.x, j0 = blockIdx.y * TY, k0 = blockIdx.z * ZC;
  const int k1 = imin(g.nz, k0 + ZC), x0 = bx * 32;
  if (tid == 0) {
    smr[0] = smr[1] = smy[0] = smy[1] = smt[0] = smt[1] = 0;
    smg[0] = GRID_NONE;
    smg[1] = MAG_NONE;
  }
  __syncthreads();
  Operand op;
  op.has_s = 1;
  op.s = a.u;
  op.has_t = a.has_uhc;
  op.t = a.uhc;
  const TileBounds tb = operand_bounds<DIM>(op, g, a.gc, bx, j0, k0, k1, smg);
  const int GF = tb.G, MF = tb.M;
  const int sA = (DIM - 2) * g.l;
  const int GA = GF - sA, MA = MF + 4 - sA;
  const int Gt = imin(a.Gf, GA), Mt = imax(a.Gf + 51, MA) + 1;
  const int Gcr = Gt + a.c_exp;
  if (tid == 0 && GF < GRID_NONE / 2 && MF + 4 - GF > 62) flag_range(a.err, 201, MF + 4, GF);
  // the bound |t| < 2^Mt is loose (t is a residual, far below |f| + |A F|): when
  // it does not fit, the CTA checks every value instead
  const bool fast = Mt - Gt <= 62 && (!a.first_sweep || Mt + 1 + a.cbits - Gt <= 62);
  bool ovf = false;
  MetaAcc mr, my, mt;
  mr.init();
  my.init();
  mt.init();
  const int j = j0 + ty, i = x0 + lane;
  const bool rowok = j < g.n, pt = rowok && i < g.n;
  march<DIM>(F, C, op, g, a.gc, bx, j0, k0, k1, GF, [&](int k, int sp, int sc, int sn, long long) {
    if (!rowok) return;
    long long t = 0;
    if (pt) {
      long long S = stencil<DIM>(F[sp], F[sc], F[sn], ty, lane);
      long long fq = rhs_at<DIM>(a, i + 1, j + 1, k + 1);
      if (fast) {
        t = shl(fq, a.Gf - Gt) - shl(S, GA - Gt);
      } else {
        t = shl_ck(fq, a.Gf - Gt, ovf) - shl_ck(S, GA - Gt, ovf);
        ck62(t, ovf);
      }
    }
    int e, sh;
    int q = encode_block(t, Gt, a.r_out.W, e, sh, a.err);
    const long long blk = ((long long)k * g.n + j) * g.nbx + bx;
    pack_block(q, a.r_out.W, pk[ty], a.r_out.words + blk * a.r_out.W);
    if (lane == 0) {
      a.r_out.exps[blk] = (int8_t)e;
      mr.add(e);
    }
    if (a.first_sweep) {  // y~ = round(c r): the first Jacobi sweep from y~ = 0
      long long rr = rounded_value(t, q, sh);
      int ey, sy;
      int qy = encode_block(fast ? rr * a.c_num : mul_ck(rr, a.c_num, a.cbits, ovf), Gcr, a.y_out.W, ey, sy,
                            a.err);
      pack_block(qy, a.y_out.W, pk[ty], a.y_out.words + blk * a.y_out.W);
      if (lane == 0) {
        a.y_out.exps[blk] = (int8_t)ey;
        my.add(ey);
      }
    }
    if (a.write_t) {  // t^_L at the width of Table 1, for the restriction chain
      int et, st;
      int qt = encode_block(t, Gt, a.t_out.W, et, st, a.err);
      pack_block(qt, a.t_out.W, pk[ty], a.t_out.words + blk * a.t_out.W);
      if (lane == 0) {
        a.t_out.exps[blk] = (int8_t)et;
        mt.add(et);
      }
    }
  });
  ovf_flush(ovf, a.err, 202);
  meta_flush(mr, a.r_out.meta, smr);
  if (a.first_sweep) meta_flush(my, a.y_out.meta, smy);
  if (a.write_t) meta_flush(mt, a.t_out.meta, smt);
}

// ------------------------------------------------------------------ restriction
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
  if (inside(gc, p.ia, p.ja, p.ka)) atomicAdd(acc + ((long long)p.ka * gc.n + p.ja) * gc.R + p.ia, (unsigned long long)d);
  if (inside(gc, p.ib, p.jb, p.kb)) atomicAdd(acc + ((long long)p.kb * gc.n + p.jb) * gc.R + p.ib, (unsigned long long)d);
}

template <int DIM>
__global__ void __launch_bounds__(NT, 2) k_restrict(RestrictArgs a) {
  __shared__ long long F[3][TY + 2][34];
  __shared__ long long C[1][CR][CX];  // unused: the operand has no coarse part
  __shared__ int smg[2];
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const int bx = blockIdx.x, j0 = blockIdx.y * TY, k0 = blockIdx.z * ZC;
  const int k1 = imin(g.nz, k0 + ZC), x0 = bx * 32;
  // one grid for every contribution to the accumulator, from the sections'
  // global finest grids: the accumulator holds R d on Gd - 1
  const int sA = (DIM - 2) * g.l;
  const int Gd = imin(sec_lsb(a.rc), a.has_y ? sec_lsb(a.y) - sA : GRID_NONE);
  if (tid == 0) {
    smg[0] = GRID_NONE;
    smg[1] = MAG_NONE;
    if (first_cta()) a.acc.meta[0] = Gd - 1;
  }
  __syncthreads();
  Operand op;
  op.has_s = a.has_y;
  op.s = a.y;
  op.has_t = 0;
  TileBounds tb;
  tb.G = GRID_NONE;
  tb.M = MAG_NONE;
  if (a.has_y) tb = operand_bounds<DIM>(op, g, g, bx, j0, k0, k1, smg);
  const int GF = tb.G, MF = tb.M;
  const int GA = GF - sA, MA = MF + 4 - sA;
  if (tid == 0 && a.has_y && GF < GRID_NONE / 2 && MF + 4 - GF > 62) flag_range(a.err, 301, MF + 4, GF);
  const bool fast = !a.has_y || GF >= GRID_NONE / 2 || MA - Gd <= 57;  // else every d is checked
  bool ovf = false;
  const int j = j0 + ty, i = x0 + lane;
  const bool rowok = j < g.n, pt = rowok && i < g.n;
  auto body = [&](int k, int sp, int sc, int sn, long long) {
    if (!rowok) return;
    const long long blk = ((long long)k * g.n + j) * g.nbx + bx;
    const int erc = __ldg(a.rc.exps + blk);
    if (erc != -128 && erc - Gd > 57) ovf = true;
    long long d = row_val(a.rc, blk, erc, lane, Gd);
    if (a.has_y && pt) {
      const long long S = stencil<DIM>(F[sp], F[sc], F[sn], ty, lane);
      if (fast) {
        d -= shl(S, GA - Gd);
      } else {
        d -= shl_ck(S, GA - Gd, ovf);
        ck58(d, ovf);
      }
    }
    if (pt && d) scatter_restrict<DIM>((unsigned long long *)a.acc.v, a.gc, i + 1, j + 1, k + 1, d);
  };
  if (a.has_y) {
    march<DIM>(F, C, op, g, g, bx, j0, k0, k1, GF, body);
  } else {
    for (int k = k0; k < k1; k++) body(k, 0, 0, 0, 0);
  }
  ovf_flush(ovf, a.err, 302);
}

// ------------------------------------------------------------------ accumulator -> BFP
template <int DIM>
__global__ void __launch_bounds__(NT) k_acc_encode(AccArgs a) {
  __shared__ uint32_t pk[TY][33];
  __shared__ int smr[2], smy[2], smt[2];
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const int G = __ldg(a.acc.meta);
  const int Gcr = G + a.c_exp;
  if (tid == 0) smr[0] = smr[1] = smy[0] = smy[1] = smt[0] = smt[1] = 0;
  __syncthreads();
  bool ovf = false;
  MetaAcc mr, my, mt;
  mr.init();
  my.init();
  mt.init();
  const long long blk = (long long)blockIdx.x * TY + ty;
  if (blk < g.nblocks) {
    const long long row = blk / g.nbx;
    const int bx = (int)(blk - row * g.nbx);
    const int i = bx * 32 + lane;
    const long long p = row * g.R + i;
    long long v = 0;
    if (i < g.n) {
      v = a.acc.v[p];
      a.acc.v[p] = 0;  // ready for the next accumulation
    }
    ck62(v, ovf);
    if (a.chain) {  // t^_l = round(R t^_(l+1)) at the width of Table 1, stored
      int et, st;
      int qt = encode_block(v, G, a.t_out.W, et, st, a.err);
      v = rounded_value(v, qt, st);
      pack_block(qt, a.t_out.W, pk[ty], a.t_out.words + blk * a.t_out.W);
      if (lane == 0) {
        a.t_out.exps[blk] = (int8_t)et;
        mt.add(et);
      }
    }
    int e, sh;
    int q = encode_block(v, G, a.r_out.W, e, sh, a.err);
    pack_block(q, a.r_out.W, pk[ty], a.r_out.words + blk * a.r_out.W);
    if (lane == 0) {
      a.r_out.exps[blk] = (int8_t)e;
      mr.add(e);
    }
    if (a.first_sweep) {
      long long rr = rounded_value(v, q, sh);
      int ey, sy;
      int qy = encode_block(mul_ck(rr, a.c_num, a.cbits, ovf), Gcr, a.y_out.W, ey, sy, a.err);
      pack_block(qy, a.y_out.W, pk[ty], a.y_out.words + blk * a.y_out.W);
      if (lane == 0) {
        a.y_out.exps[blk] = (int8_t)ey;
        my.add(ey);
      }
    }
  }
  ovf_flush(ovf, a.err, 401);
  meta_flush(mr, a.r_out.meta, smr);
  if (a.first_sweep) meta_flush(my, a.y_out.meta, smy);
  if (a.chain) meta_flush(mt, a.t_out.meta, smt);
}

// ------------------------------------------------------------------ level 1
// rounding of the rational value N * 2^G / a (a = 1 or 3) into a one-value
// block of width W; returns the code, sets e.
__device__ int encode_rational(__int128 N, int G, int a, int W, int &e) {
  if (N == 0) {
    e = -128;
    return 0;
  }
  __int128 aN = N < 0 ? -N : N;
  int b = 0;
  for (__int128 t = aN; t; t >>= 1) b++;
  int Ep;  // 2^(Ep-1) <= |N| / a < 2^Ep
  if (a == 1) Ep = b;
  else Ep = (b >= 2 && aN >= ((__int128)3 << (b - 2))) ? b - 1 : b - 2;
  e = Ep + G;
  for (int pass = 0; pass < 2; pass++) {
    int k = W - 1 - (e - G);  // code = RNE(N * 2^k / a)
    __int128 num = N, den = a;
    if (k >= 0) num = N << k;
    else den = (__int128)a << (-k);
    __int128 q = num / den;  // truncates toward zero
    __int128 rem = num - q * den;
    if (rem < 0) {  // make it floor
      q -= 1;
      rem += den;
    }
    if (2 * rem > den || (2 * rem == den && (q & 1))) q += 1;
    __int128 lim = (__int128)1 << (W - 1);
    if (q == lim || q == -lim) {
      e += 1;
      continue;
    }
    return (int)q;
  }
  return 0;
}

__device__ inline void set_tmp1(const Tmp &t, long long v, int G) {
  // a one-value temporary (level 1): value and block descriptor
  t.v[0] = v;
  t.gb[0] = v ? (int)((unsigned)G << 8) | bitlen64(v) : 0;
}

__global__ void k_coarse(CoarseArgs a) {
  // one warp; lane 0 owns the single unknown, lanes 1..31 are block padding
  __shared__ uint32_t pk[33];
  const int lane = threadIdx.x;
  const int dim = a.dim;
  int e = -128, q = 0;
  __int128 N;
  int G;
  if (a.mode_start) {  // u~_1 = round(f_1 / A_1)
    N = (__int128)a.f1;
    G = a.Gf1;
  } else {  // y~_1 = round(rc_1 / A_1)
    int er = a.rc.exps[0];
    N = er == -128 ? 0 : (__int128)code_at(a.rc.words, a.rc.W, 0);
    G = er - a.rc.W + 1;
  }
  // A_1 = 2d h^(d-2) at h = 1/2: 4 in 2-D, 3 in 3-D
  int div = dim == 2 ? 1 : 3;
  if (dim == 2) G -= 2;
  Sec out = a.mode_start ? a.u_out : a.y_out;
  if (lane == 0) q = encode_rational(N, G, div, out.W, e);
  e = __shfl_sync(0xffffffffu, e, 0);
  if ((e > 127 || e < -127) && e != -128 && lane == 0) atomicOr(a.err, ERR_EXP);
  pack_block(lane == 0 ? q : 0, out.W, pk, out.words);
  if (lane == 0) {
    out.exps[0] = (int8_t)e;
    if (e != -128) {
      out.meta[0] = e + META_BIAS;
      out.meta[1] = META_BIAS - e;
    }
  }
  if (lane != 0) return;
  const int yG = e == -128 ? 0 : e - out.W + 1;
  if (a.mode_start) {
    set_tmp1(a.uh_out, q, yG);
    return;
  }
  set_tmp1(a.w_out, q, yG);  // w_1 = y~_1 (z_1 = 0)
  if (!a.corr) return;
  // u~_1 <- round(u~_1 + y~_1), u^_1 = u~_1
  int eu0 = a.u_in.exps[0];
  long long uq = eu0 == -128 ? 0 : code_at(a.u_in.words, a.u_in.W, 0);
  int uG = eu0 == -128 ? yG : eu0 - a.u_in.W + 1;
  int Gs = imin(uG, yG);
  __int128 sum = ((__int128)uq << (uG - Gs)) + ((__int128)q << (yG - Gs));
  int eu;
  int qu = encode_rational(sum, Gs, 1, a.u_out.W, eu);
  a.u_out.exps[0] = (int8_t)eu;
  if (eu > 127 || (eu < -127 && eu != -128)) atomicOr(a.err, ERR_EXP);
  for (int w = 0; w < a.u_out.W; w++) a.u_out.words[w] = 0;
  a.u_out.words[0] = (uint32_t)qu & (a.u_out.W == 32 ? 0xffffffffu : ((1u << a.u_out.W) - 1u));
  if (eu != -128) {
    a.u_out.meta[0] = eu + META_BIAS;
    a.u_out.meta[1] = META_BIAS - eu;
  }
  set_tmp1(a.uh_out, qu, eu == -128 ? 0 : eu - a.u_out.W + 1);
}

// ------------------------------------------------------------------ repack
__global__ void __launch_bounds__(NT) k_repack(RepackArgs a) {
  __shared__ uint32_t pk[TY][33];
  __shared__ int sm[2];
  const int lane = threadIdx.x, ty = threadIdx.y;
  if (lane == 0 && ty == 0) sm[0] = sm[1] = 0;
  __syncthreads();
  MetaAcc m;
  m.init();
  const long long blk = (long long)blockIdx.x * TY + ty;
  if (blk < a.nblocks) {
    int e = a.in.exps[blk];
    int q = e == -128 ? 0 : code_at(a.in.words + blk * a.in.W, a.in.W, lane);
    q = (int)((unsigned)q << (a.out.W - a.in.W));  // widen: append zero bits
    pack_block(q, a.out.W, pk[ty], a.out.words + blk * a.out.W);
    if (lane == 0) {
      a.out.exps[blk] = (int8_t)e;
      m.add(e);
    }
  }
  meta_flush(m, a.out.meta, sm);
}

// ------------------------------------------------------------------ unfused pieces
template <int DIM>
__global__ void __launch_bounds__(NT) k_chain(ChainArgs a) {
  // u^_l = u~_l + P_l u^_(l-1), one warp per 32-value block
  const Geo g = a.g;
  const int lane = threadIdx.x, ty = threadIdx.y;
  bool ovf = false;
  const long long blk = (long long)blockIdx.x * TY + ty;
  if (blk < g.nblocks) {
    const long long row = blk / g.nbx;
    const int bx = (int)(blk - row * g.nbx);
    const int i = bx * 32 + lane, j = (int)(row % g.n), k = (int)(row / g.n);
    const bool pt = i < g.n;
    int gp = (pt && a.has_uhc) ? prolong_grid<DIM>(a.uhc, a.gc, i + 1, j + 1, k + 1) : GRID_NONE;
    const int G = imin(blk_lsb(__ldg(a.u.exps + blk), a.u.W), __reduce_min_sync(0xffffffffu, gp));
    long long v = 0;
    if (pt) {
      v = sec_val_ck(a.u, g, i, j, k, G, ovf);
      if (a.has_uhc) v += prolong_tmp<DIM>(a.uhc, a.gc, i + 1, j + 1, k + 1, G, ovf);
    }
    ck62(v, ovf);
    store_tmp_block(v, G, a.uh_out.v + row * g.R + i, a.uh_out.gb + blk, pt, ovf);
  }
  ovf_flush(ovf, a.err, 501);
}

__global__ void __launch_bounds__(NT) k_axpy(AxpyArgs a) {
  // u~ <- round(u~ + y~), one warp per block
  __shared__ uint32_t pk[TY][33];
  __shared__ int sm[2];
  const int lane = threadIdx.x, ty = threadIdx.y;
  if (lane == 0 && ty == 0) sm[0] = sm[1] = 0;
  __syncthreads();
  bool ovf = false;
  MetaAcc m;
  m.init();
  const long long blk = (long long)blockIdx.x * TY + ty;
  if (blk < a.g.nblocks) {
    const long long row = blk / a.g.nbx;
    const int bx = (int)(blk - row * a.g.nbx);
    const int i = bx * 32 + lane, j = (int)(row % a.g.n), k = (int)(row / a.g.n);
    const int G = imin(blk_lsb(__ldg(a.u_in.exps + blk), a.u_in.W), blk_lsb(__ldg(a.y.exps + blk), a.y.W));
    long long v = sec_val_ck(a.u_in, a.g, i, j, k, G, ovf) + sec_val_ck(a.y, a.g, i, j, k, G, ovf);
    ck62(v, ovf);
    int e, s;
    int q = encode_block(v, G, a.u_out.W, e, s, a.err);
    pack_block(q, a.u_out.W, pk[ty], a.u_out.words + blk * a.u_out.W);
    if (lane == 0) {
      a.u_out.exps[blk] = (int8_t)e;
      m.add(e);
    }
  }
  ovf_flush(ovf, a.err, 601);
  meta_flush(m, a.u_out.meta, sm);
}

template <int DIM>
__global__ void k_decode_solution(DecodeSolArgs a) {
  const Geo g = a.g;
  bool ovf = false;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = a.nz * (long long)g.n * g.n;
  if (p < total) {
    const int i = (int)(p % g.n);
    const long long row = p / g.n;
    const int j = (int)(row % g.n), k = (int)(row / g.n) + (int)a.z0;
    int G = blk_lsb(__ldg(a.u.exps + blk_index(g, i, j, k)), a.u.W);
    if (a.has_uhc) G = imin(G, prolong_grid<DIM>(a.uhc, a.gc, i + 1, j + 1, k + 1));
    long long v = 0;
    if (G < GRID_NONE / 2) {
      v = sec_val_ck(a.u, g, i, j, k, G, ovf);
      if (a.has_uhc) v += prolong_tmp<DIM>(a.uhc, a.gc, i + 1, j + 1, k + 1, G, ovf);
    }
    a.out[p] = v == 0 ? 0.0 : scalbn(__ll2double_rn(v), G);
  }
  ovf_flush(ovf, a.err, 701);
}

// ------------------------------------------------------------------ codec
// Exact decomposition of a finite double: x = m * 2^ex, |m| < 2^53.
__device__ __forceinline__ bool split_double(double x, long long &m, int &ex) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  int be = (int)((b >> 52) & 0x7ff);
  unsigned long long frac = b & ((1ull << 52) - 1);
  if (be == 0x7ff) return false;
  if (be == 0) {  // zero or subnormal
    m = (long long)frac;
    ex = -1074;
  } else {
    m = (long long)(frac | (1ull << 52));
    ex = be - 1075;
  }
  if (b >> 63) m = -m;
  return true;
}

__global__ void __launch_bounds__(256) k_encode_f64(CodecArgs a) {
  __shared__ uint32_t pk[8][33];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long blk = (long long)blockIdx.x * 8 + wid;
  const long long nb = (a.n + 31) / 32;
  if (blk >= nb) return;  // warp-uniform
  const long long p = blk * 32 + lane;
  long long m = 0;
  int ex = 0;
  bool ok = true;
  if (p < a.n) ok = split_double(a.x[p], m, ex);
  if (!ok) {
    atomicOr(a.err, ERR_INPUT);
    m = 0;
  }
  // natural exponent of |x| = |m| 2^ex: bitlen(|m|) + ex
  int E = m ? bitlen64(m) + ex : -100000;
  int Emax = __reduce_max_sync(0xffffffffu, E);
  int e, q = 0;
  if (Emax == -100000) {
    e = -128;
  } else {
    e = Emax;
    for (int pass = 0; pass < 2; pass++) {
      // code = RNE(x 2^(W-1-e)) = RNE(m 2^(ex + W - 1 - e))
      int s = e - (a.W - 1) - ex;  // bits to drop
      long long qq = (m && s <= 62) ? rne_shift(m, s) : 0;  // s > 62: far below half a unit
      long long lim = 1ll << (a.W - 1);
      if (__any_sync(0xffffffffu, qq == lim || qq == -lim)) {
        e += 1;
        continue;
      }
      q = (int)qq;
      break;
    }
    if ((e > 127 || e < -127) && lane == 0) atomicOr(a.err, ERR_EXP);
  }
  pack_block(q, a.W, pk[wid], a.words + blk * a.W);
  if (lane == 0) a.exps[blk] = (int8_t)(e > 127 ? 127 : (e < -128 ? -128 : e));
}

__global__ void k_decode_f64(CodecArgs a) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  long long blk = p >> 5;
  int e = a.exps[blk];
  int q = code_at(a.words + blk * a.W, a.W, (int)(p & 31));
  if ((long long)q == -(1ll << (a.W - 1))) atomicOr(a.err, ERR_CORRUPT);
  a.x[p] = (e == -128) ? 0.0 : scalbn((double)q, e - a.W + 1);
}

// ------------------------------------------------------------------ launchers
static dim3 stencil_grid(const Geo &g) {
  return dim3((unsigned)g.nbx, (unsigned)((g.n + TY - 1) / TY), (unsigned)((g.nz + ZC - 1) / ZC));
}

void launch_sweep(int dim, const SweepArgs &a, cudaStream_t st) {
  dim3 b(32, TY);
  if (dim == 3) k_sweep<3><<<stencil_grid(a.g), b, 0, st>>>(a);
  else k_sweep<2><<<stencil_grid(a.g), b, 0, st>>>(a);
}

void launch_residual(int dim, const ResidArgs &a, cudaStream_t st) {
  dim3 b(32, TY);
  if (dim == 3) k_residual<3><<<stencil_grid(a.g), b, 0, st>>>(a);
  else k_residual<2><<<stencil_grid(a.g), b, 0, st>>>(a);
}

void launch_restrict(int dim, const RestrictArgs &a, cudaStream_t st) {
  dim3 b(32, TY);
  if (dim == 3) k_restrict<3><<<stencil_grid(a.g), b, 0, st>>>(a);
  else k_restrict<2><<<stencil_grid(a.g), b, 0, st>>>(a);
}

void launch_acc_encode(int dim, const AccArgs &a, cudaStream_t st) {
  dim3 b(32, TY);
  unsigned nb = (unsigned)((a.g.nblocks + TY - 1) / TY);
  if (dim == 3) k_acc_encode<3><<<nb, b, 0, st>>>(a);
  else k_acc_encode<2><<<nb, b, 0, st>>>(a);
}

void launch_coarse(const CoarseArgs &a, cudaStream_t st) { k_coarse<<<1, 32, 0, st>>>(a); }

void launch_repack(const RepackArgs &a, cudaStream_t st) {
  dim3 b(32, TY);
  k_repack<<<(unsigned)((a.nblocks + TY - 1) / TY), b, 0, st>>>(a);
}

void launch_chain(int dim, const ChainArgs &a, cudaStream_t st) {
  dim3 b(32, TY);
  unsigned nb = (unsigned)((a.g.nblocks + TY - 1) / TY);
  if (dim == 3) k_chain<3><<<nb, b, 0, st>>>(a);
  else k_chain<2><<<nb, b, 0, st>>>(a);
}

void launch_axpy(const AxpyArgs &a, cudaStream_t st) {
  dim3 b(32, TY);
  k_axpy<<<(unsigned)((a.g.nblocks + TY - 1) / TY), b, 0, st>>>(a);
}

void launch_decode_solution(int dim, const DecodeSolArgs &a, cudaStream_t st) {
  long long total = a.nz * (long long)a.g.n * a.g.n;
  unsigned nb = (unsigned)((total + 255) / 256);
  if (dim == 3) k_decode_solution<3><<<nb, 256, 0, st>>>(a);
  else k_decode_solution<2><<<nb, 256, 0, st>>>(a);
}

void launch_encode_f64(const CodecArgs &a, cudaStream_t st) {
  long long nb = (a.n + 31) / 32;
  k_encode_f64<<<(unsigned)((nb + 7) / 8), 256, 0, st>>>(a);
}

void launch_decode_f64(const CodecArgs &a, cudaStream_t st) {
  k_decode_f64<<<(unsigned)((a.n + 255) / 256), 256, 0, st>>>(a);
}

}  // namespace cmg
