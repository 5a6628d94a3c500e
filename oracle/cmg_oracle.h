/*
 * CPU oracle for the compact full multigrid (CMG) solver.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct FP64
 * restatement of the method of "Multigrid with Linear Storage Complexity"
 * (Bauer, Kohl, McCormick, Tamstorf): the compact representation (Sec. 2,
 * eq. compact-to-standard), the compact FAS cycle (Sec. 3.2, Algorithm 1,
 * eq. cfas), fmgResidual (Algorithm 2), compact FMG with iterative refinement
 * (Algorithm 3), the precision rules of Table 1 and the rounding rules of
 * Sec. 4, and BFP storage (Sec. 6.1.3).  Only the test-suite, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the product library never
 * links or calls it, and it shares no code with the CUDA path.
 *
 * Arithmetic reading.  The paper performs every operation in (arbitrary
 * precision) floating point at least as wide as Table 1 requires and rounds
 * only where a quantity is stored.  The oracle reads this as: intermediate
 * arithmetic is exact, stores round to nearest with ties to even into the
 * block-floating-point (BFP) format.  FP64 realises exact arithmetic whenever
 * no operation rounds; every add, subtract and multiply is checked with an
 * error-free transformation and the number of inexact operations is counted
 * (cmgo_inexact).  A run with a zero count equals exact arithmetic.
 *
 * BFP format (bit-exact contract shared with the CUDA path by specification).
 * A section on level l holds the interior nodes of a (2^l-1)^d grid, x fastest.
 * Each x-row is split into blocks of 32 consecutive values, the last one padded
 * with zeros.  A block stores one int8 exponent e and 32 W-bit two's-complement
 * codes q (2 <= W <= 32, sign bit included as in Table 2):
 *     value_i = q_i * 2^(e - W + 1).
 * e is the smallest integer with max|x| < 2^e; codes are RNE(x * 2^(W-1-e)); if
 * a code reaches 2^(W-1) the exponent is raised by one and the block is
 * re-quantised.  An all-zero block stores e = -128.  Code i occupies bits
 * [iW, iW+W) of the block's little-endian stream of W uint32 words.
 */
#ifndef CMG_ORACLE_H
#define CMG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CMGO_OK = 0,
  CMGO_EINVAL = 1,
  CMGO_ENOMEM = 2,
  CMGO_ERANGE = 3,   /* exponent outside [-127, 127] */
  CMGO_ECORRUPT = 5  /* code -2^(W-1) found while decoding */
};

/* Parameters of Algorithm 3 and Table 1 for P1 elements (p = 1, m = 1). */
typedef struct {
  int dim;      /* 2 or 3 */
  int Lmax;     /* finest level, h = 2^-Lmax */
  int b1, b2;   /* finest-level widths of u~ and of r, y~ (0 = lossless) */
  int ku, kr;   /* regressive increments (p+1 and m) */
  int N;        /* IR iterations per FMG level */
  int nu1, nu2; /* pre- and post-smoothing sweeps per level, nu2 >= 1 */
  double omega; /* Jacobi weight */
  int arith;    /* 0: exact V-cycle; 1: binary32 V-cycle, 2: binary64 V-cycle,
                   each inside exact iterative refinement (cycle_real.inc) */
  int coef;     /* 0: Poisson; 1: diffusion -div(k grad u) with a nodal binary32
                   coefficient field (cmgo_set_coefficient); needs arith = 1 or 2
                   and nu1 >= 1 (see cmg_oracle.c, "diffusion") */
  int smoother; /* 0: weighted Jacobi; 1: red-black Gauss-Seidel (each sweep a red
                   then a black half-sweep; needs nu1 = 0, the paper's V(0,1)) */
} cmgo_params;

/* Section selectors. */
enum { CMGO_U = 0, CMGO_R = 1, CMGO_RC = 2, CMGO_Y = 3 };

/* ---- stand-alone codec on a flat array (blocks of 32 consecutive values) ---- */
int cmgo_encode(const double *x, int64_t n, int W, uint32_t *words, int8_t *e);
int cmgo_decode(const uint32_t *words, const int8_t *e, int64_t n, int W, double *x);

/* ---- operators on dense level arrays (index (k*n + j)*n + i, n = 2^l-1) ---- */
int64_t cmgo_npoints(int dim, int level);
int64_t cmgo_nblocks(int dim, int level);
void cmgo_apply_A(int dim, int level, const double *x, double *out);
void cmgo_prolong(int dim, int level, const double *coarse, double *fine);
void cmgo_restrict(int dim, int level, const double *fine, double *coarse);

/* ---- compact FMG (Algorithm 3) ---- */
typedef struct cmgo_ctx cmgo_ctx;
/* tables: int32 [nterms][dim][2^Lmax - 1]; F = 2^scale_exp * sum_t prod_a T */
cmgo_ctx *cmgo_create(const cmgo_params *p, int nterms, const int32_t *tables, int scale_exp);
void cmgo_destroy(cmgo_ctx *c);
int cmgo_status(const cmgo_ctx *c);
long long cmgo_inexact(const cmgo_ctx *c);
int cmgo_level(const cmgo_ctx *c);
int cmgo_rhs_shift(const cmgo_ctx *c);
int cmgo_width(const cmgo_ctx *c, int which, int level);

/* Diffusion: the nodal coefficient k at every node of the finest grid,
 * boundary included: (2^Lmax + 1)^dim binary32 values, x fastest.  Copied. */
int cmgo_set_coefficient(cmgo_ctx *c, const float *k);
/* (A_level x) of the diffusion operator with the FP64 order of the outer
 * residual (dense interior arrays, as cmgo_apply_A) */
int cmgo_apply_A_diffusion(const cmgo_ctx *c, int level, const double *x, double *out);

/* Diffusion: a right-hand side given by its nodal values g at the interior
 * nodes of the finest grid ((2^Lmax - 1)^dim doubles, copied), replacing the
 * separable one: f_L = h_L^d g, injected at stride 2^(Lmax - L) on coarser
 * FMG levels. */
int cmgo_set_rhs_nodal(cmgo_ctx *c, const double *g);
/* Adjoint gradient of J with respect to the nodal coefficient k at every node
 * of the finest grid, boundary included ((2^Lmax + 1)^dim doubles):
 *   G_i = -((sum_q (u_i - u_q)(lam_i - lam_q)) * 0.5) * h^(d-2)
 * over the neighbours q of i inside the closed grid in the order -x,+x,-y,+y,
 * -z,+z, with u = lam = 0 on the boundary; u and lam are interior arrays. */
int cmgo_gradient_k(const cmgo_ctx *c, const double *u, const double *lam, double *out);

int cmgo_start(cmgo_ctx *c);        /* L = 1: u~_1 = round(f_1 / A_1) */
int cmgo_next_level(cmgo_ctx *c);   /* L += 1: zero new section, widen the others */
int cmgo_residual(cmgo_ctx *c);     /* Algorithm 2 */
int cmgo_down(cmgo_ctx *c, int level);
int cmgo_coarse(cmgo_ctx *c);
int cmgo_up(cmgo_ctx *c, int level);
int cmgo_vcycle(cmgo_ctx *c);       /* one compact V(nu1,nu2) cycle from y~ = 0 */
int cmgo_correct(cmgo_ctx *c);      /* u~ += y~ (Algorithm 3, apply correction) */
int cmgo_ir_iteration(cmgo_ctx *c); /* residual, cycle, correction */
int cmgo_fmg(cmgo_ctx *c);          /* the whole of Algorithm 3 */

/* Section access.  words: nblocks*W uint32 (may be NULL), e: nblocks int8 (may
 * be NULL), values: dense npoints doubles (may be NULL). */
int cmgo_get_section(const cmgo_ctx *c, int which, int level, uint32_t *words, int8_t *e,
                     double *values);
int cmgo_set_section(cmgo_ctx *c, int which, int level, int W, const uint32_t *words,
                     const int8_t *e);
int cmgo_decode_solution(const cmgo_ctx *c, double *out); /* u^_L, dense */
int cmgo_rhs(const cmgo_ctx *c, int level, double *out);  /* f_level, dense */
int cmgo_last_t(const cmgo_ctx *c, double *out);          /* exact t_L of the last residual */
int cmgo_last_w(const cmgo_ctx *c, int level, double *out); /* w_l = y~_l + z_l of the last up-leg */

#ifdef __cplusplus
}
#endif
#endif
