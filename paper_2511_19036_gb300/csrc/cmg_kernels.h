// Launch interface of the compact FMG kernels (host side, internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "cmg_device.cuh"

namespace cmg {

struct SweepArgs {
  Geo g, gc;           // level l and level l-1
  int has_y;           // y~ input present (else y~ = 0)
  int has_z;           // z_l = P w_(l-1) present
  int write_y;         // store y~'
  int corr;            // fused u~ <- round(u~ + y~')
  int write_w;         // w_l = y~' + z_l
  int write_uh;        // u^_l = u~' + P u^_(l-1)
  int has_uhc;         // u^_(l-1) present (l >= 2)
  int Wy;              // width of y~'
  Sec y_in, rc, y_out, u_in, u_out;
  Tmp wc, w_out, uhc, uh_out;
  int tl;              // w_(l-1) held in two levels (wc2) instead of wc
  Tmp2 wc2;
  int c_num, c_exp, cbits;  // Jacobi factor c_l = c_num 2^c_exp, cbits = bitlen(c_num)
  const void *wc_r;    // floating-point cycle: w_(l-1) in the cycle's type (padded level layout)
  void *w_out_r;       // floating-point cycle: w_l in the cycle's type
  const float *kfield; // diffusion (floating-point cycle): nodal binary32 k, boundary included
  int kN, kstride;     // 2^Lmax + 1, and the level's stride 2^(Lmax - l) in it
  float omega;         // diffusion: Jacobi weight (factor omega / D_p per node)
  int rb;              // 0: every node; 1 / 2: only the red / black nodes (red: the
                       // 1-based node numbers I + J [+ K] even), the others keep y~
  // fallback tiles: the specialised kernel appends the tiles it leaves to the
  // generic one; the generic kernel with list_mode = 1 runs only those
  unsigned *tiles;
  int *ntiles;
  int list_mode;
  int *err;
};

struct ResidArgs {
  Geo g, gc;
  Sec u;               // u~_L
  int has_uhc;
  Tmp uhc;             // u^_(L-1)
  int tl;              // u^_(L-1) held in two levels (uhc2) instead of uhc
  Tmp2 uhc2;
  const int32_t *tables;
  int nterms, n1max, Lmax, fsh;
  int rhs_bits;        // bit length of the bound sum_t prod_a max|T| on |F_q| before the shift
  int Gf;              // grid of f_L: scale_exp + fsh - d L
  Sec r_out;
  int first_sweep;     // also y~ = round(c r)
  Sec y_out;
  // no pre-smoothing: t^_L = round(t) at the width Wt of Table 1, restricted
  // here: R t^_L accumulated into racc (level L-1, padded layout) on one grid
  // below every t^_L value, derived from the u~_l sections' metadata (umeta,
  // uW for l = 1..L); the grid goes to racc.meta[0]
  int fuse_restrict;
  int Wt;
  Tmp racc;
  const int *umeta[16];
  int uW[16];
  int c_num, c_exp, cbits;
  const float *kfield;  // diffusion: nodal k on the finest grid, boundary included
  int kN;               // 2^Lmax + 1 (the field is kN^dim, x fastest)
  const double *grhs;   // diffusion: nodal right-hand side g on the finest interior, or null
  int grhs_log2;        // f_L = h_L^d 2^grhs_log2 g
  unsigned *tiles;      // fallback tiles (as in SweepArgs)
  int *ntiles;
  int list_mode;
  int *err;
};

struct RestrictArgs {
  Geo g, gc;
  int has_y;           // d = rc - A y~ (else d = rc)
  Sec y, rc;
  Tmp acc;             // exact R_l d on one global grid
  void *d_out;         // diffusion: d = fl(rc - A y~) in the cycle's type (padded level layout)
  const float *kfield; // diffusion: nodal k, boundary included
  int kN, kstride;
  int *err;
};

// diffusion: rc_(l-1) = round(R_l d) with R_l d in binary32 in the fixed order
struct GatherArgs {
  Geo g, gc;           // fine level l, coarse level l - 1
  const void *d;       // d on level l in the cycle's type (padded layout)
  Sec rc_out;
  int *err;
};

struct AccArgs {
  Geo g, gc;
  Tmp acc;             // exact values on level l (zeroed after reading)
  Sec r_out;
  int first_sweep;
  Sec y_out;
  int chain;           // restriction chain of t^: t^ = round(R t^) at the width
  Sec t_out;           // of Table 1, stored, and r = round(t^)
  int c_num, c_exp, cbits;
  int *err;
};

struct CoarseArgs {
  int dim;
  int mode_start;      // 1: u~_1 = round(f_1 / A_1); 0: y~_1 = round(rc_1 / A_1)
  long long f1;        // F_q at the level-1 node (start mode)
  int Gf1;             // its grid
  Sec rc, y_out, u_in, u_out;
  int corr;            // fused u~_1 += y~_1 (cycle mode)
  Tmp w_out, uh_out;
  void *w_out_r;       // floating-point cycle: w_1 = y~_1 in its type (else w_out)
  int w_f64;           // ... binary64 (else binary32)
  const float *kfield; // diffusion: the level-1 diagonal from k (FP64 division)
  int kN, kstride;
  const double *grhs;  // diffusion start mode: f_1 = 2^(grhs_log2 - d) g[gidx] (else f1 on Gf1)
  int grhs_log2;
  long long gidx;
  int *err;
};

struct RepackArgs {
  Sec in, out;
  long long nblocks;
};

struct ChainArgs {
  Geo g, gc;
  Sec u;
  int has_uhc;
  Tmp uhc, uh_out;
  int *err;
};

struct AxpyArgs {
  Geo g;
  Sec u_in, y, u_out;
  int *err;
};

struct DecodeSolArgs {
  Geo g, gc;
  Sec u;
  int has_uhc;
  Tmp uhc;
  int tl;              // u^_(L-1) held in two levels (uhc2) instead of uhc
  Tmp2 uhc2;
  long long z0, nz;
  double *out;
  int *err;
};

struct CodecArgs {
  double *x;
  long long n;
  int W;
  uint32_t *words;
  int8_t *exps;
  int *err;
};

void launch_sweep(int dim, const SweepArgs &a, cudaStream_t st);
void launch_residual(int dim, const ResidArgs &a, cudaStream_t st);
// the generic kernels over a fallback tile list (a.tiles, a.ntiles on the device)
void launch_sweep_list(int dim, const SweepArgs &a, cudaStream_t st);
void launch_residual_list(int dim, const ResidArgs &a, cudaStream_t st);
// specialised 3-D Poisson kernels of the exact path (cmg_fast.cu); each returns
// false (launching nothing) when the step is not one it covers
bool launch_sweep_fast(const SweepArgs &a, cudaStream_t st);
bool launch_residual_fast(const ResidArgs &a, cudaStream_t st);
void launch_restrict(int dim, const RestrictArgs &a, cudaStream_t st);
void launch_residual_diffusion(int dim, const ResidArgs &a, cudaStream_t st);

// adjoint gradients of J for the diffusion problem (FP64, fixed order)
struct GradArgs {
  int dim, L;          // finest level
  const double *u, *lam;  // interior arrays (2^L - 1)^dim
  const float *kfield; // unused by the formula; kept for the layout size kN
  int kN;
  double *dk;          // dJ/dk at every node, boundary included, kN^dim
  double *dg;          // dJ/dg = h^d lam on the interior, or null
};
void launch_gradient(const GradArgs &a, cudaStream_t st);
// the floating-point cycle, binary64 (f64) or binary32
void launch_sweep_fp(int dim, bool f64, const SweepArgs &a, cudaStream_t st);
void launch_restrict_fp(int dim, bool f64, const RestrictArgs &a, cudaStream_t st);
void launch_dvec_diffusion(int dim, bool f64, const RestrictArgs &a, cudaStream_t st);
void launch_gather_restrict_fp(int dim, bool f64, const GatherArgs &a, cudaStream_t st);
void launch_acc_encode(int dim, const AccArgs &a, cudaStream_t st);
void launch_coarse(const CoarseArgs &a, cudaStream_t st);
void launch_repack(const RepackArgs &a, cudaStream_t st);
void launch_chain(int dim, const ChainArgs &a, cudaStream_t st);
void launch_axpy(const AxpyArgs &a, cudaStream_t st);
void launch_decode_solution(int dim, const DecodeSolArgs &a, cudaStream_t st);
void launch_encode_f64(const CodecArgs &a, cudaStream_t st);
void launch_decode_f64(const CodecArgs &a, cudaStream_t st);
// bytes from device memory into page-locked host memory through the GPU's
// mapping of it (dst: the device address of the host buffer; both 16-byte aligned)
void launch_copy_out(const void *src, void *dst, size_t bytes, int nsm, cudaStream_t st);

}  // namespace cmg
