// Compact FMG kernels for GB300 (sm_103a).
//
// Every kernel reads its operands in the compact BFP form (Sec. 6.1.3 of the
// paper), computes exactly in int64 fixed point on locally chosen grids (see
// cmg_device.cuh), and writes BFP sections rounded to nearest-even (Sec. 4).
// The stencil kernels (cmg_stencil.cu, cmg_stencil_fp.cu) march a CTA through
// z, keeping the planes k-1, k, k+1 of each column's decoded operand in
// registers and the in-plane neighbours in two shared-memory plane buffers
// (one x-block of 32 plus a one-node halo, by TY rows plus halo); one warp owns
// one output block row.
//
// Kernels (one launch covers one level):
//   k_sweep     smoothing sweep y~ <- round(y~ + c (rc - A (y~ + P w_(l-1))))
//               (Algorithm 1 smoothing step on eq. cfas) at every node, or at
//               the nodes of one colour (red-black Gauss-Seidel half-sweep),
//               with optional fused correction u~ <- round(u~ + y~)
//               (Algorithm 3), w_l = y~ + z_l and u^_l = u~_l + P u^_(l-1) for
//               the next level / residual
//   k_residual  Algorithm 2 on the finest level: t = f - A (u~_L + P u^_(L-1)),
//               r = round(t); optional first Jacobi sweep from y~ = 0 fused in,
//               or t^ (Table 1 width) restricted into the level L-1 accumulator
//   k_restrict  d = rc - A y~ (or d = rc) scattered as R_l d into an int64
//               accumulator by exact, order-free integer atomics
//   k_acc_encode round an accumulator into BFP section(s) (+ optional first sweep)
//   k_coarse    the single unknown of level 1
//   k_repack    FMG level step: widen a section by appending zero bits
//   k_chain, k_axpy, k_decode_solution: unfused pieces for step-wise use
//   k_encode_f64, k_decode_f64: stand-alone codec
//   k_copy_out  device bytes into page-locked host memory through its mapping
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "cmg_device.cuh"
#include "cmg_kernels.h"

namespace cmg {


// ------------------------------------------------------------------ accumulator -> BFP
template <int DIM>
__global__ void __launch_bounds__(NT, 6) k_acc_encode(AccArgs a) {
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
  // each warp rounds a contiguous run of blocks (block indices of a level fit in int)
  const int nwarps = gridDim.x * TY, w = blockIdx.x * TY + ty;
  const int nbl = (int)g.nblocks, chunk = (nbl + nwarps - 1) / nwarps;
  const int b0 = imin(nbl, w * chunk), b1 = imin(nbl, b0 + chunk);
  int row = b0 / g.nbx, bx = b0 - row * g.nbx;
  long long vn = 0;  // value of the next block, loaded one block ahead
  auto load = [&](int r, int x) -> long long {
    const int i = x * 32 + lane;
    return i < g.n ? a.acc.v[(long long)r * g.R + i] : 0;
  };
  if (b0 < b1) vn = load(row, bx);
  for (int blk = b0; blk < b1; blk++) {
    const int i = bx * 32 + lane;
    const long long p = (long long)row * g.R + i;
    long long v = vn;
    if (i < g.n) a.acc.v[p] = 0;  // ready for the next accumulation
    int nrow = row, nbx = bx + 1;
    if (nbx == g.nbx) {
      nbx = 0;
      nrow++;
    }
    if (blk + 1 < b1) vn = load(nrow, nbx);
    ck62(v, ovf);
    if (a.chain) {  // t^_l = round(R t^_(l+1)) at the width of Table 1, stored
      int et, st;
      int qt = encode_block(v, G, a.t_out.W, et, st, a.err);
      v = rounded_value(v, qt, st);
      pack_block(qt, a.t_out.W, pk[ty], a.t_out.words + (long long)blk * a.t_out.W);
      if (lane == 0) {
        a.t_out.exps[blk] = (int8_t)et;
        mt.add(et);
      }
    }
    int e, sh;
    int q = encode_block(v, G, a.r_out.W, e, sh, a.err);
    pack_block(q, a.r_out.W, pk[ty], a.r_out.words + (long long)blk * a.r_out.W);
    if (lane == 0) {
      a.r_out.exps[blk] = (int8_t)e;
      mr.add(e);
    }
    if (a.first_sweep) {
      long long rr = rounded_value(v, q, sh);
      int ey, sy;
      int qy = encode_block(mul_ck(rr, a.c_num, a.cbits, ovf), Gcr, a.y_out.W, ey, sy, a.err);
      pack_block(qy, a.y_out.W, pk[ty], a.y_out.words + (long long)blk * a.y_out.W);
      if (lane == 0) {
        a.y_out.exps[blk] = (int8_t)ey;
        my.add(ey);
      }
    }
    row = nrow;
    bx = nbx;
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
  if (a.kfield) {
    // diffusion: x = num / D_1 in FP64 with D_1 = h^(d-2) sum over the
    // neighbours -x,+x,-y,+y,-z,+z of (k_q + k_p) * 0.5, then rounded as the
    // oracle rounds doubles
    double x = 0.0;
    if (lane == 0) {
      auto kat = [&](int I, int J, int K) -> double {
        return (double)__ldg(a.kfield + ((long long)(dim == 3 ? K * a.kstride : 0) * a.kN + J * a.kstride) * a.kN +
                             I * a.kstride);
      };
      const double kp = kat(1, 1, 1);
      double acc = 0.0;
      for (int e6 = 0; e6 < 2 * dim; e6++) {
        const int Iq = 1 + (e6 == 0 ? -1 : e6 == 1 ? 1 : 0), Jq = 1 + (e6 == 2 ? -1 : e6 == 3 ? 1 : 0);
        const int Kq = 1 + (e6 == 4 ? -1 : e6 == 5 ? 1 : 0);
        acc = __dadd_rn(acc, __dmul_rn(__dadd_rn(kat(Iq, Jq, Kq), kp), 0.5));
      }
      const double D = __dmul_rn(acc, dim == 3 ? 0.5 : 1.0);
      const int Gn = a.mode_start ? a.Gf1 : G + (dim == 2 ? 2 : 0);  // grid of N as read
      double num = __dmul_rn((double)(long long)N, __longlong_as_double((long long)(Gn + 1023) << 52));
      if (a.mode_start && a.grhs)  // nodal right-hand side: f_1 = 2^(grhs_log2 - d) g at the centre node
        num = scalbn(__ldg(a.grhs + a.gidx), a.grhs_log2 - dim);
      x = __ddiv_rn(num, D);
    }
    q = encode_block_f64(x, out.W, e, a.err);
    if (lane != 0) q = 0;
  } else {
    if (lane == 0) q = encode_rational(N, G, div, out.W, e);
    e = __shfl_sync(0xffffffffu, e, 0);
  }
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
  if (a.w_out_r) {  // w_1 = y~_1 in the cycle's type (exact: binary32 needs W <= 24, checked at setup)
    if (a.w_f64) ((double *)a.w_out_r)[0] = e == -128 ? 0.0 : ldexp((double)q, yG);
    else ((float *)a.w_out_r)[0] = e == -128 ? 0.0f : ldexpf((float)q, yG);
  } else {
    set_tmp1(a.w_out, q, yG);  // w_1 = y~_1 (z_1 = 0)
  }
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
  bool ovf = false, bad = false;
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
      v = sec_val_ck(a.u, g, i, j, k, G, ovf, bad);
      if (a.has_uhc) v += prolong_tmp<DIM>(a.uhc, a.gc, i + 1, j + 1, k + 1, G, ovf);
    }
    ck62(v, ovf);
    store_tmp_block(v, G, a.uh_out.v + row * g.R + i, a.uh_out.gb + blk, pt, ovf);
  }
  ovf_flush(ovf, a.err, 501);
  corrupt_flush(bad, a.err);
}

__global__ void __launch_bounds__(NT) k_axpy(AxpyArgs a) {
  // u~ <- round(u~ + y~), one warp per block
  __shared__ uint32_t pk[TY][33];
  __shared__ int sm[2];
  const int lane = threadIdx.x, ty = threadIdx.y;
  if (lane == 0 && ty == 0) sm[0] = sm[1] = 0;
  __syncthreads();
  bool ovf = false, bad = false;
  MetaAcc m;
  m.init();
  const long long blk = (long long)blockIdx.x * TY + ty;
  if (blk < a.g.nblocks) {
    const long long row = blk / a.g.nbx;
    const int bx = (int)(blk - row * a.g.nbx);
    const int i = bx * 32 + lane, j = (int)(row % a.g.n), k = (int)(row / a.g.n);
    const int G = imin(blk_lsb(__ldg(a.u_in.exps + blk), a.u_in.W), blk_lsb(__ldg(a.y.exps + blk), a.y.W));
    long long v = sec_val_ck(a.u_in, a.g, i, j, k, G, ovf, bad) + sec_val_ck(a.y, a.g, i, j, k, G, ovf, bad);
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
  corrupt_flush(bad, a.err);
  meta_flush(m, a.u_out.meta, sm);
}

template <int DIM>
__global__ void k_decode_solution(DecodeSolArgs a) {
  const Geo g = a.g;
  bool ovf = false, bad = false;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = a.nz * (long long)g.n * g.n;
  if (p < total) {
    const int i = (int)(p % g.n);
    const long long row = p / g.n;
    const int j = (int)(row % g.n), k = (int)(row / g.n) + (int)a.z0;
    int G = blk_lsb(__ldg(a.u.exps + blk_index(g, i, j, k)), a.u.W);
    long long p2 = 0;  // two-level u^_(L-1): P of it on its own grid G2
    int G2 = GRID_NONE;
    if (a.tl) {
      p2 = prolong2<DIM>(a.uhc2, a.gc, i + 1, j + 1, k + 1, G2, ovf, bad);
      G = imin(G, G2);
    } else if (a.has_uhc) {
      G = imin(G, prolong_grid<DIM>(a.uhc, a.gc, i + 1, j + 1, k + 1));
    }
    long long v = 0;
    if (G < GRID_NONE / 2) {
      v = sec_val_ck(a.u, g, i, j, k, G, ovf, bad);
      if (a.tl) {
        if (p2) v += shl_ck(p2, G2 - G, ovf);
      } else if (a.has_uhc) {
        v += prolong_tmp<DIM>(a.uhc, a.gc, i + 1, j + 1, k + 1, G, ovf);
      }
    }
    a.out[p] = v == 0 ? 0.0 : scalbn(__ll2double_rn(v), G);
  }
  ovf_flush(ovf, a.err, 701);
  corrupt_flush(bad, a.err);
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
// SMs of the current device (queried once; 152 on GB300)
static int sm_count() {
  static int n = 0;
  if (n <= 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else
      return 152;
  }
  return n;
}

void launch_acc_encode(int dim, const AccArgs &a, cudaStream_t st) {
  dim3 b(32, TY);
  // one wave of 6 CTAs of 8 warps per SM, each warp a contiguous run of blocks
  const long long want = (a.g.nblocks + TY - 1) / TY, cap = 6ll * sm_count();
  unsigned nb = (unsigned)(want < cap ? want : cap);
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

namespace {
// Copy of device bytes into host memory the GPU maps (page-locked memory):
// 16-byte words by a grid-stride loop, then the tail bytes.  src and dst are
// 16-byte aligned.
__global__ void k_copy_out(const uint4 *__restrict__ src, uint4 *__restrict__ dst, size_t n16,
                           const unsigned char *__restrict__ tsrc, unsigned char *__restrict__ tdst, int ntail) {
  const size_t step = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += step) dst[i] = src[i];
  if (blockIdx.x == 0 && (int)threadIdx.x < ntail) tdst[threadIdx.x] = tsrc[threadIdx.x];
}
}  // namespace

void launch_copy_out(const void *src, void *dst, size_t bytes, int nsm, cudaStream_t st) {
  const size_t n16 = bytes / 16;
  const int ntail = (int)(bytes - 16 * n16);
  const size_t want = (n16 + 511) / 512;
  const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>(want, (size_t)4 * nsm));
  k_copy_out<<<blocks, 512, 0, st>>>((const uint4 *)src, (uint4 *)dst, n16, (const unsigned char *)src + 16 * n16,
                                     (unsigned char *)dst + 16 * n16, ntail);
}

}  // namespace cmg
