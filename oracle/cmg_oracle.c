/*
 * CPU oracle for the compact full multigrid solver -- TEST INFRASTRUCTURE ONLY.
 * See cmg_oracle.h for the reading of the paper that this file implements.
 *
 * Build: cc -O2 -std=c11 -fPIC -shared -ffp-contract=off -fno-fast-math [-fopenmp]
 * (-ffp-contract=off keeps the compiler from fusing the error-free
 * transformations below into FMAs).
 *
 * Every loop visits grid points independently, so OpenMP threads change no
 * result.  Index conventions: level l has n = 2^l - 1 interior nodes per axis
 * (h = 2^-l), 0-based array index i <-> 1-based node number I = i + 1 at the
 * coordinate I*h; node numbers 0 and 2^l are the Dirichlet boundary (value 0).
 * In 2-D the z extent is 1 and no z-neighbour exists.
 */
#define _GNU_SOURCE
#include "cmg_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXL 20

/* ------------------------------------------------------------------------- */
/* exactness-checked FP64 arithmetic                                          */
/* ------------------------------------------------------------------------- */

/* a + b, counting the operation when the rounded sum differs from the exact
 * one (Knuth's TwoSum error term is zero exactly when the sum is exact). */
static inline double xadd(double a, double b, long long *cnt) {
  double s = a + b;
  double bb = s - a;
  double err = (a - (s - bb)) + (b - bb);
  if (err != 0.0) (*cnt)++;
  return s;
}

static inline double xsub(double a, double b, long long *cnt) { return xadd(a, -b, cnt); }

/* a * b, counting the operation when fma(a, b, -p) shows a rounding error. */
static inline double xmul(double a, double b, long long *cnt) {
  double p = a * b;
  if (fma(a, b, -p) != 0.0) (*cnt)++;
  return p;
}

/* ------------------------------------------------------------------------- */
/* level geometry                                                             */
/* ------------------------------------------------------------------------- */

typedef struct {
  int dim, l, n, nz, nbx;
  int64_t np, nb;
} lev;

static lev mklev(int dim, int l) {
  lev g;
  g.dim = dim;
  g.l = l;
  g.n = (1 << l) - 1;
  g.nz = dim == 3 ? g.n : 1;
  g.nbx = (g.n + 31) / 32;
  g.np = (int64_t)g.nz * g.n * g.n;
  g.nb = (int64_t)g.nz * g.n * g.nbx;
  return g;
}

int64_t cmgo_npoints(int dim, int level) { return mklev(dim, level).np; }
int64_t cmgo_nblocks(int dim, int level) { return mklev(dim, level).nb; }

static inline int64_t idx(const lev *g, int i, int j, int k) {
  return ((int64_t)k * g->n + j) * g->n + i;
}

/* value at 0-based (i, j, k); zero outside the interior (Dirichlet boundary) */
static inline double get0(const double *x, const lev *g, int i, int j, int k) {
  if (i < 0 || i >= g->n || j < 0 || j >= g->n || k < 0 || k >= g->nz) return 0.0;
  return x[idx(g, i, j, k)];
}

/* value at 1-based node (I, J, K); zero on the boundary.  K ignored in 2-D. */
static inline double node(const double *x, const lev *g, int I, int J, int K) {
  if (g->dim == 2) K = 1;
  return get0(x, g, I - 1, J - 1, K - 1);
}

/* ------------------------------------------------------------------------- */
/* operators (Sec. 3.1: A_l, P_l, R_l = P_l^T; P1 elements on the Kuhn mesh)   */
/* ------------------------------------------------------------------------- */

/* (A_l x) at a node: the P1 stiffness of the structured Kuhn triangulation is
 * h^(d-2) (2d x_p - sum over the 2d axis neighbours).  Exact arithmetic makes
 * the order immaterial; this one is fixed anyway: centre, then -x,+x,-y,+y,-z,+z. */
static double A_at(const double *x, const lev *g, int i, int j, int k, long long *cnt) {
  double acc = xmul(x[idx(g, i, j, k)], 2.0 * g->dim, cnt);
  acc = xsub(acc, get0(x, g, i - 1, j, k), cnt);
  acc = xsub(acc, get0(x, g, i + 1, j, k), cnt);
  acc = xsub(acc, get0(x, g, i, j - 1, k), cnt);
  acc = xsub(acc, get0(x, g, i, j + 1, k), cnt);
  if (g->dim == 3) {
    acc = xsub(acc, get0(x, g, i, j, k - 1), cnt);
    acc = xsub(acc, get0(x, g, i, j, k + 1), cnt);
  }
  return ldexp(acc, -(g->dim - 2) * g->l); /* times h^(d-2), a power of two */
}

/* (P_l xc) at fine node (I, J, K): linear interpolation along the Kuhn edge
 * through the node.  With S the set of odd coordinates, an all-even node copies
 * the coarse node I/2; otherwise it averages the coarse nodes (I -+ e_S)/2. */
static double P_at(const double *xc, const lev *gc, int I, int J, int K, long long *cnt) {
  int sx = I & 1, sy = J & 1, sz = gc->dim == 3 ? (K & 1) : 0;
  if (!sx && !sy && !sz) return node(xc, gc, I / 2, J / 2, K / 2);
  double a = node(xc, gc, (I - sx) / 2, (J - sy) / 2, (K - sz) / 2);
  double b = node(xc, gc, (I + sx) / 2, (J + sy) / 2, (K + sz) / 2);
  return ldexp(xadd(a, b, cnt), -1);
}

/* the 2^d - 1 non-empty odd sets, in the order {x},{y},{x,y},{z},{x,z},{y,z},{x,y,z} */
static const int ODDSET[7][3] = {{1, 0, 0}, {0, 1, 0}, {1, 1, 0}, {0, 0, 1},
                                 {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};

/* (R_l xf) at coarse node (Ic, Jc, Kc): the transpose of P_l, i.e. the value at
 * the fine node 2J plus one half of the 2(2^d - 1) fine nodes 2J -+ e_S. */
static double R_at(const double *xf, const lev *gf, int Ic, int Jc, int Kc, long long *cnt) {
  int I = 2 * Ic, J = 2 * Jc, K = 2 * Kc;
  int ns = gf->dim == 3 ? 7 : 3;
  double sum = 0.0;
  for (int s = 0; s < ns; s++) {
    int ex = ODDSET[s][0], ey = ODDSET[s][1], ez = ODDSET[s][2];
    sum = xadd(sum, node(xf, gf, I - ex, J - ey, K - ez), cnt);
    sum = xadd(sum, node(xf, gf, I + ex, J + ey, K + ez), cnt);
  }
  return xadd(node(xf, gf, I, J, K), ldexp(sum, -1), cnt);
}

static void apply_A(const lev *g, const double *x, double *out, long long *cnt) {
  long long c = 0;
#pragma omp parallel for collapse(2) reduction(+ : c) schedule(static)
  for (int k = 0; k < g->nz; k++)
    for (int j = 0; j < g->n; j++)
      for (int i = 0; i < g->n; i++) out[idx(g, i, j, k)] = A_at(x, g, i, j, k, &c);
  *cnt += c;
}

static void prolong(const lev *gc, const lev *gf, const double *xc, double *xf, long long *cnt) {
  long long c = 0;
#pragma omp parallel for collapse(2) reduction(+ : c) schedule(static)
  for (int k = 0; k < gf->nz; k++)
    for (int j = 0; j < gf->n; j++)
      for (int i = 0; i < gf->n; i++) xf[idx(gf, i, j, k)] = P_at(xc, gc, i + 1, j + 1, k + 1, &c);
  *cnt += c;
}

static void restrict_(const lev *gf, const lev *gc, const double *xf, double *xc, long long *cnt) {
  long long c = 0;
#pragma omp parallel for collapse(2) reduction(+ : c) schedule(static)
  for (int k = 0; k < gc->nz; k++)
    for (int j = 0; j < gc->n; j++)
      for (int i = 0; i < gc->n; i++) xc[idx(gc, i, j, k)] = R_at(xf, gf, i + 1, j + 1, k + 1, &c);
  *cnt += c;
}

void cmgo_apply_A(int dim, int level, const double *x, double *out) {
  lev g = mklev(dim, level);
  long long c = 0;
  apply_A(&g, x, out, &c);
}

void cmgo_prolong(int dim, int level, const double *coarse, double *fine) {
  lev gc = mklev(dim, level - 1), gf = mklev(dim, level);
  long long c = 0;
  prolong(&gc, &gf, coarse, fine, &c);
}

void cmgo_restrict(int dim, int level, const double *fine, double *coarse) {
  lev gf = mklev(dim, level), gc = mklev(dim, level - 1);
  long long c = 0;
  restrict_(&gf, &gc, fine, coarse, &c);
}

/* ------------------------------------------------------------------------- */
/* floating-point V-cycles (the precision split of Table 1: the cycle works in  */
/* progressive(+m, b4) precision, the residual of fmgResidual in                */
/* progressive(+p+m+1, b3)).  arith = 1 runs the cycle in IEEE binary32,        */
/* arith = 2 in IEEE binary64 (the plain FP64 form), both round to nearest with */
/* no fused multiply-add, in the one fixed order of cycle_real.inc, while the   */
/* outer residual, the level-1 solve and the correction of u~ stay exact.       */
/* ------------------------------------------------------------------------- */

/* x as binary32; flags *bad when x is not exactly a normal-range float or 0 */
static inline float to_f32(double x, int *bad) {
  float f = (float)x;
  if ((double)f != x || (f != 0.0f && fabsf(f) < FLT_MIN)) *bad = 1;
  return f;
}

/* x as binary64: every stored value is one already */
static inline double to_f64(double x, int *bad) {
  (void)bad;
  return x;
}

/* ------------------------------------------------------------------------- */
/* BFP rounding (Sec. 4: round to nearest, ties to even; Sec. 6.1.3: BFP)      */
/* ------------------------------------------------------------------------- */

/* Round the values x[0..cnt) of one block to W-bit codes sharing one exponent.
 * Returns the exponent (-128 for an all-zero block) and writes the rounded
 * values to v; *st is set to CMGO_ERANGE if the exponent leaves [-127, 127].
 * W == 0 means lossless storage (the value is kept as it is). */
static int round_block(const double *x, int cnt, int W, double *v, int *st) {
  if (W == 0) {
    for (int i = 0; i < cnt; i++) v[i] = x[i];
    return 0;
  }
  double M = 0.0;
  for (int i = 0; i < cnt; i++) M = fmax(M, fabs(x[i]));
  if (M == 0.0) {
    for (int i = 0; i < cnt; i++) v[i] = 0.0;
    return -128;
  }
  int E;
  frexp(M, &E); /* M = f 2^E, 1/2 <= f < 1, so 2^(E-1) <= M < 2^E */
  double lim = ldexp(1.0, W - 1);
  for (int pass = 0; pass < 2; pass++) {
    int bump = 0;
    for (int i = 0; i < cnt; i++) {
      double q = rint(ldexp(x[i], W - 1 - E)); /* exact scaling, then RNE */
      if (fabs(q) >= lim) bump = 1;
      v[i] = q;
    }
    if (!bump) break;
    E += 1; /* a code rounded up to 2^(W-1): re-quantise with the next exponent */
  }
  if (E > 127 || E < -127) *st = CMGO_ERANGE;
  for (int i = 0; i < cnt; i++) v[i] = ldexp(v[i], E - W + 1);
  return E;
}

typedef struct {
  int W;
  double *v; /* rounded values, dense level layout */
  int8_t *e; /* one exponent per block */
} sec;

/* round a dense level array into section s with width W */
static int round_dense(const lev *g, const double *x, int W, sec *s) {
  int st = CMGO_OK;
  s->W = W;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < g->nz; k++)
    for (int j = 0; j < g->n; j++) {
      int lst = CMGO_OK;
      for (int bx = 0; bx < g->nbx; bx++) {
        int i0 = 32 * bx, cntv = g->n - i0 < 32 ? g->n - i0 : 32;
        int64_t p = idx(g, i0, j, k);
        int E = round_block(x + p, cntv, W, s->v + p, &lst);
        s->e[((int64_t)k * g->n + j) * g->nbx + bx] = (int8_t)(E < -128 ? -128 : E > 127 ? 127 : E);
      }
      if (lst != CMGO_OK) {
#pragma omp critical
        st = lst;
      }
    }
  return st;
}

static inline uint64_t wmask(int W) { return W >= 64 ? ~0ull : ((1ull << W) - 1); }

/* pack 32 integer codes into W words: code i at bits [iW, iW+W) */
static void pack_block(const int64_t *q, int W, uint32_t *words) {
  for (int w = 0; w < W; w++) words[w] = 0;
  for (int i = 0; i < 32; i++) {
    uint64_t code = (uint64_t)q[i] & wmask(W);
    int pos = i * W, wd = pos >> 5, off = pos & 31;
    uint64_t sh = code << off;
    words[wd] |= (uint32_t)sh;
    if (off + W > 32) words[wd + 1] |= (uint32_t)(sh >> 32);
  }
}

static int64_t unpack_code(const uint32_t *words, int W, int i) {
  int pos = i * W, wd = pos >> 5, off = pos & 31;
  uint64_t lo = words[wd];
  uint64_t hi = (off + W > 32) ? words[wd + 1] : 0;
  uint64_t bits = ((lo | (hi << 32)) >> off) & wmask(W);
  if ((bits >> (W - 1)) & 1) return (int64_t)bits - (int64_t)(1ull << W);
  return (int64_t)bits;
}

int cmgo_encode(const double *x, int64_t n, int W, uint32_t *words, int8_t *e) {
  if (W < 2 || W > 32 || n < 0) return CMGO_EINVAL;
  int64_t nb = (n + 31) / 32;
  int st = CMGO_OK;
  for (int64_t b = 0; b < nb; b++) {
    double xb[32] = {0}, vb[32];
    int64_t q[32];
    int cntv = (int)(n - 32 * b < 32 ? n - 32 * b : 32);
    for (int i = 0; i < cntv; i++) xb[i] = x[32 * b + i];
    int E = round_block(xb, 32, W, vb, &st);
    for (int i = 0; i < 32; i++) q[i] = E == -128 ? 0 : (int64_t)ldexp(vb[i], W - 1 - E);
    pack_block(q, W, words + b * W);
    e[b] = (int8_t)(E < -128 ? -128 : E > 127 ? 127 : E);
  }
  return st;
}

int cmgo_decode(const uint32_t *words, const int8_t *e, int64_t n, int W, double *x) {
  if (W < 2 || W > 32 || n < 0) return CMGO_EINVAL;
  int st = CMGO_OK;
  for (int64_t p = 0; p < n; p++) {
    int64_t b = p / 32;
    int64_t q = unpack_code(words + b * W, W, (int)(p % 32));
    if (q == -(int64_t)(1ull << (W - 1))) st = CMGO_ECORRUPT;
    x[p] = e[b] == -128 ? 0.0 : ldexp((double)q, e[b] - W + 1);
  }
  return st;
}

/* ------------------------------------------------------------------------- */
/* context                                                                    */
/* ------------------------------------------------------------------------- */

struct cmgo_ctx {
  cmgo_params P;
  int nterms, scale_exp, fsh, n1max;
  int32_t *tab;
  int L;
  sec u[MAXL + 1];  /* solution sections u~_l */
  sec r[MAXL + 1];  /* residual hierarchy r_l from fmgResidual */
  sec rc[MAXL + 1]; /* right-hand side of the level-l relaxation in the cycle */
  sec y[MAXL + 1];  /* correction sections y~_l */
  double *w[MAXL + 1]; /* w_l = y~_l + z_l after the up-leg on level l (exact) */
  double *t;           /* exact t_L of the last residual */
  int t_level;         /* t holds a level this fine (0: not allocated) */
  float *kfield;       /* diffusion: nodal k on the finest grid, boundary included */
  double *grhs;        /* diffusion: nodal right-hand side g (interior of the finest grid), or NULL */
  long long inexact;
  int status;
};

static int sec_alloc(sec *s, const lev *g) {
  s->W = 0;
  s->v = (double *)calloc((size_t)g->np, sizeof(double));
  s->e = (int8_t *)malloc((size_t)g->nb);
  if (!s->v || !s->e) return CMGO_ENOMEM;
  memset(s->e, -128, (size_t)g->nb);
  return CMGO_OK;
}

static void sec_zero(sec *s, const lev *g, int W) {
  s->W = W;
  memset(s->v, 0, (size_t)g->np * sizeof(double));
  memset(s->e, W == 0 ? 0 : -128, (size_t)g->nb);
}

static void sec_copy(sec *dst, const sec *src, const lev *g) {
  dst->W = src->W;
  memcpy(dst->v, src->v, (size_t)g->np * sizeof(double));
  memcpy(dst->e, src->e, (size_t)g->nb);
}

/* Table 1: u~ in regressive(+p+1, b1), r and y~ in regressive(+m, b2).  A zero
 * finest width selects lossless storage (oracle-only, used by pins). */
static int Wu(const cmgo_ctx *c, int l) { return c->P.b1 == 0 ? 0 : c->P.ku * (c->L - l) + c->P.b1; }
static int Wr(const cmgo_ctx *c, int l) { return c->P.b2 == 0 ? 0 : c->P.kr * (c->L - l) + c->P.b2; }
/* Table 1: u^ and t^ in fmgResidual carry (p+1)L + b1 bits */
static int Wt(const cmgo_ctx *c) { return c->P.b1 == 0 ? 0 : c->P.ku * c->L + c->P.b1; }

/* ------------------------------------------------------------------------- */
/* diffusion -div(k grad u) (the variable-coefficient workload): on level l the */
/* coefficient is the finest nodal field injected at stride 2^(Lmax - l); the   */
/* flux between neighbours p, q uses the face value (k_p + k_q) / 2, so         */
/*   (A_l u)_p = h^(d-2) sum over the 2d neighbours q of (k_p+k_q)/2 (u_p - u_q) */
/* with u = 0 on the boundary (k = 1 gives the Poisson stencil).  The outer     */
/* residual evaluates it in FP64 and the cycle in binary32 or binary64, each   */
/* in a fixed order (face sums are exact in FP64; products and sums round).     */
/* ------------------------------------------------------------------------- */

static const int NBR[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};

/* k at 1-based node (I, J, K) of level l (boundary nodes 0 and 2^l included) */
static inline float kcoef(const cmgo_ctx *c, int l, int I, int J, int K) {
  const int d = c->P.dim, s = 1 << (c->P.Lmax - l), N = (1 << c->P.Lmax) + 1;
  if (d == 2) K = 0;
  return c->kfield[((int64_t)(K * s) * N + J * s) * N + I * s];
}

/* FP64 (A_l x)_p, 0-based interior (i, j, k): acc = 0; for q in -x,+x,-y,+y,-z,+z:
 * acc = acc + ((k_p + k_q) * 0.5) * (x_p - x_q); times h^(d-2) */
static double A_at_diff64(const cmgo_ctx *c, const double *x, const lev *g, int i, int j, int k) {
  const int I = i + 1, J = j + 1, K = k + 1, nn = 2 * g->dim;
  const double kp = (double)kcoef(c, g->l, I, J, K), xp = x[idx(g, i, j, k)];
  volatile double acc = 0.0;
  for (int e = 0; e < nn; e++) {
    const int Iq = I + NBR[e][0], Jq = J + NBR[e][1], Kq = K + NBR[e][2];
    volatile double kf = ((double)kcoef(c, g->l, Iq, Jq, Kq) + kp) * 0.5;
    volatile double du = xp - get0(x, g, Iq - 1, Jq - 1, Kq - 1);
    volatile double pr = kf * du;
    acc = acc + pr;
  }
  return acc * ldexp(1.0, -(g->dim - 2) * g->l);
}

/* FP64 diagonal of A_l at the single level-1 node */
static double diag1_diff64(const cmgo_ctx *c) {
  const int nn = 2 * c->P.dim;
  const double kp = (double)kcoef(c, 1, 1, 1, 1);
  volatile double acc = 0.0;
  for (int e = 0; e < nn; e++) {
    volatile double kf = ((double)kcoef(c, 1, 1 + NBR[e][0], 1 + NBR[e][1], 1 + NBR[e][2]) + kp) * 0.5;
    acc = acc + kf;
  }
  return acc * ldexp(1.0, -(c->P.dim - 2));
}


int cmgo_width(const cmgo_ctx *c, int which, int level) {
  return which == CMGO_U ? Wu(c, level) : Wr(c, level);
}

static int bitlen_u128(unsigned __int128 v) {
  int b = 0;
  while (v) {
    b++;
    v >>= 1;
  }
  return b;
}

cmgo_ctx *cmgo_create(const cmgo_params *p, int nterms, const int32_t *tables, int scale_exp) {
  if (!p || p->dim < 2 || p->dim > 3 || p->Lmax < 1 || p->Lmax > MAXL || p->N < 1 ||
      p->nu1 < 0 || p->nu2 < 1 || p->b1 < 0 || p->b2 < 0 || nterms < 1 || !tables)
    return NULL;
  if (p->arith < 0 || p->arith > 2) return NULL;
  if (p->coef != 0 && (p->coef != 1 || p->arith == 0 || p->nu1 < 1)) return NULL;
  if (p->smoother != 0 && (p->smoother != 1 || p->nu1 != 0)) return NULL;
  cmgo_ctx *c = (cmgo_ctx *)calloc(1, sizeof(cmgo_ctx));
  if (!c) return NULL;
  c->P = *p;
  c->nterms = nterms;
  c->scale_exp = scale_exp;
  c->n1max = (1 << p->Lmax) - 1;
  size_t ntab = (size_t)nterms * p->dim * c->n1max;
  c->tab = (int32_t *)malloc(ntab * sizeof(int32_t));
  if (!c->tab) goto fail;
  memcpy(c->tab, tables, ntab * sizeof(int32_t));
  /* The load vector is rounded to 50 bits below a bound on |F| (the paper asks
   * that f be free of error other than quantisation, Sec. 4); the bound is the
   * sum over terms of the product of the table maxima. */
  {
    unsigned __int128 bound = 0;
    for (int t = 0; t < nterms; t++) {
      unsigned __int128 prod = 1;
      for (int a = 0; a < p->dim; a++) {
        int64_t m = 0;
        for (int i = 0; i < c->n1max; i++) {
          int64_t v = llabs((long long)c->tab[((size_t)t * p->dim + a) * c->n1max + i]);
          if (v > m) m = v;
        }
        prod *= (unsigned __int128)m;
      }
      bound += prod;
    }
    int B = bitlen_u128(bound);
    c->fsh = B > 50 ? B - 50 : 0;
  }
  c->L = 0;  /* level arrays come with the first visit of a level (ensure_level) */
  return c;
fail:
  cmgo_destroy(c);
  return NULL;
}

void cmgo_destroy(cmgo_ctx *c) {
  if (!c) return;
  for (int l = 1; l <= MAXL; l++) {
    sec *ss[4] = {&c->u[l], &c->r[l], &c->rc[l], &c->y[l]};
    for (int s = 0; s < 4; s++) {
      free(ss[s]->v);
      free(ss[s]->e);
    }
    free(c->w[l]);
  }
  free(c->t);
  free(c->tab);
  free(c->kfield);
  free(c->grhs);
  free(c);
}

int cmgo_status(const cmgo_ctx *c) { return c->status; }
long long cmgo_inexact(const cmgo_ctx *c) { return c->inexact; }
int cmgo_level(const cmgo_ctx *c) { return c->L; }
int cmgo_rhs_shift(const cmgo_ctx *c) { return c->fsh; }

int cmgo_set_coefficient(cmgo_ctx *c, const float *k) {
  if (!c || !k) return CMGO_EINVAL;
  const int64_t N = (1 << c->P.Lmax) + 1;
  const int64_t cnt = c->P.dim == 3 ? N * N * N : N * N;
  free(c->kfield);
  c->kfield = (float *)malloc((size_t)cnt * sizeof(float));
  if (!c->kfield) return CMGO_ENOMEM;
  memcpy(c->kfield, k, (size_t)cnt * sizeof(float));
  return CMGO_OK;
}

int cmgo_set_rhs_nodal(cmgo_ctx *c, const double *g) {
  if (!c || !g || !c->P.coef) return CMGO_EINVAL;
  const int64_t n1 = c->n1max, cnt = c->P.dim == 3 ? n1 * n1 * n1 : n1 * n1;
  free(c->grhs);
  c->grhs = (double *)malloc((size_t)cnt * sizeof(double));
  if (!c->grhs) return CMGO_ENOMEM;
  memcpy(c->grhs, g, (size_t)cnt * sizeof(double));
  return CMGO_OK;
}

/* adjoint gradient dJ/dk_i = -lam^T (dA/dk_i) u for
 * (A u)_p = h^(d-2) sum_q (k_p + k_q)/2 (u_p - u_q): node i enters the faces to
 * its neighbours q with weight 1/2, so the derivative is
 * -(1/2) h^(d-2) sum_q (u_i - u_q)(lam_i - lam_q)  (dJ/dm_i = k_i dJ/dk_i for k = exp(m)) */
int cmgo_gradient_k(const cmgo_ctx *c, const double *u, const double *lam, double *out) {
  if (!c || !c->kfield || !u || !lam || !out) return CMGO_EINVAL;
  const int d = c->P.dim, L = c->P.Lmax, N = (1 << L) + 1;
  lev g = mklev(d, L);
  const int nz = d == 3 ? N : 1;
  for (int K = 0; K < nz; K++)
    for (int J = 0; J < N; J++)
      for (int I = 0; I < N; I++) {
        const int Kn = d == 3 ? K : 1;
        const double ui = get0(u, &g, I - 1, J - 1, Kn - 1), li = get0(lam, &g, I - 1, J - 1, Kn - 1);
        volatile double acc = 0.0;
        for (int e = 0; e < 2 * d; e++) {
          const int Iq = I + NBR[e][0], Jq = J + NBR[e][1], Kq = (d == 3 ? K : 1) + NBR[e][2];
          if (Iq < 0 || Iq >= N || Jq < 0 || Jq >= N || (d == 3 && (Kq < 0 || Kq >= N))) continue;
          volatile double du = ui - get0(u, &g, Iq - 1, Jq - 1, Kq - 1);
          volatile double dl = li - get0(lam, &g, Iq - 1, Jq - 1, Kq - 1);
          volatile double pr = du * dl;
          acc = acc + pr;
        }
        volatile double t = acc * 0.5;
        t = t * ldexp(1.0, -(d - 2) * L);
        out[((int64_t)(d == 3 ? K : 0) * N + J) * N + I] = -t;
      }
  return CMGO_OK;
}

int cmgo_apply_A_diffusion(const cmgo_ctx *c, int level, const double *x, double *out) {
  if (!c || !c->kfield || level < 1 || level > c->P.Lmax) return CMGO_EINVAL;
  lev g = mklev(c->P.dim, level);
  for (int k = 0; k < g.nz; k++)
    for (int j = 0; j < g.n; j++)
      for (int i = 0; i < g.n; i++) out[idx(&g, i, j, k)] = A_at_diff64(c, x, &g, i, j, k);
  return CMGO_OK;
}

static int setst(cmgo_ctx *c, int st) {
  if (st != CMGO_OK && c->status == CMGO_OK) c->status = st;
  return st;
}

/* round-to-nearest-even right shift of a signed 128-bit integer */
static __int128 rne_shift(__int128 v, int sh) {
  if (sh <= 0) return v;
  __int128 q = v >> sh; /* floor */
  __int128 rem = v - (q << sh);
  __int128 half = (__int128)1 << (sh - 1);
  if (rem > half || (rem == half && (q & 1))) q += 1;
  return q;
}

/* f_L at node (I, J, K): nodal load h^d F(x), with F from the exact integer
 * tables rounded to the 50-bit grid (matrix-free assembly, Sec. 5.1). */
static double f_at(const cmgo_ctx *c, int L, int I, int J, int K) {
  int d = c->P.dim, stride = 1 << (c->P.Lmax - L);
  int ia[3] = {I * stride - 1, J * stride - 1, K * stride - 1};
  if (c->grhs) {  /* nodal right-hand side: f_L = h_L^d g, injected */
    const int64_t n1 = c->n1max;
    const int64_t p = d == 3 ? ((int64_t)ia[2] * n1 + ia[1]) * n1 + ia[0] : (int64_t)ia[1] * n1 + ia[0];
    return ldexp(c->grhs[p], -d * L);
  }
  __int128 F = 0;
  for (int t = 0; t < c->nterms; t++) {
    __int128 prod = 1;
    for (int a = 0; a < d; a++) prod *= (__int128)c->tab[((size_t)t * d + a) * c->n1max + ia[a]];
    F += prod;
  }
  __int128 q = rne_shift(F, c->fsh);
  return ldexp((double)(int64_t)q, c->scale_exp + c->fsh - d * L);
}

int cmgo_rhs(const cmgo_ctx *c, int L, double *out) {
  lev g = mklev(c->P.dim, L);
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < g.nz; k++)
    for (int j = 0; j < g.n; j++)
      for (int i = 0; i < g.n; i++) out[idx(&g, i, j, k)] = f_at(c, L, i + 1, j + 1, k + 1);
  return CMGO_OK;
}

/* A_1 = 2d h_1^(d-2): 4 in 2-D, 3 in 3-D (one interior node, all neighbours on
 * the boundary).  The quotient is rounded by the FP64 division; the BFP rounding
 * that follows still equals the exact RNE of the rational num/A_1, because a
 * non-dyadic quotient cannot lie within half an FP64 ulp of a W-bit tie when
 * num carries at most 53 significant bits and W <= 50. */
static double A1(int dim) { return ldexp(2.0 * dim, 2 - dim); }

/* ------------------------------------------------------------------------- */
/* Algorithm 3 steps                                                          */
/* ------------------------------------------------------------------------- */

/* The arrays of level l (and the residual array t, sized for the finest level
 * reached) are allocated when the FMG first reaches l, so that a hierarchy with
 * a large L_max can run its coarser stages alone.  Memory only: no value depends
 * on when a level was allocated. */
static int ensure_level(cmgo_ctx *c, int l) {
  if (c->w[l]) return CMGO_OK;
  lev g = mklev(c->P.dim, l);
  if (sec_alloc(&c->u[l], &g) || sec_alloc(&c->r[l], &g) || sec_alloc(&c->rc[l], &g) || sec_alloc(&c->y[l], &g))
    return CMGO_ENOMEM;
  double *w = (double *)calloc((size_t)g.np, sizeof(double));
  if (!w) return CMGO_ENOMEM;
  if (l > c->t_level) {
    double *t = (double *)calloc((size_t)g.np, sizeof(double));
    if (!t) {
      free(w);
      return CMGO_ENOMEM;
    }
    free(c->t);
    c->t = t;
    c->t_level = l;
  }
  c->w[l] = w;
  return CMGO_OK;
}

int cmgo_start(cmgo_ctx *c) {
  if (ensure_level(c, 1)) return setst(c, CMGO_ENOMEM);
  c->L = 1;
  c->inexact = 0;
  c->status = CMGO_OK;
  lev g = mklev(c->P.dim, 1);
  if (c->P.coef && !c->kfield) return setst(c, CMGO_EINVAL);
  /* coarse-grid solve; with diffusion a rounded FP64 division by the diagonal */
  double x = c->P.coef ? f_at(c, 1, 1, 1, 1) / diag1_diff64(c) : f_at(c, 1, 1, 1, 1) / A1(c->P.dim);
  return setst(c, round_dense(&g, &x, Wu(c, 1), &c->u[1]));
}

int cmgo_next_level(cmgo_ctx *c) {
  if (c->L >= c->P.Lmax) return setst(c, CMGO_EINVAL);
  if (ensure_level(c, c->L + 1)) return setst(c, CMGO_ENOMEM);
  c->L += 1;
  /* Prolongating a compact vector adds a zero section; raising L widens every
   * other section by k bits, which appends zero bits (exact, Sec. 4). */
  for (int l = 1; l < c->L; l++) c->u[l].W = Wu(c, l);
  lev g = mklev(c->P.dim, c->L);
  sec_zero(&c->u[c->L], &g, Wu(c, c->L));
  return CMGO_OK;
}

/* decode chain u^_1 = u~_1, u^_l = u~_l + P_l u^_(l-1) (eq. compact-to-standard) */
static double *decode_chain(const cmgo_ctx *c, int upto, long long *cnt) {
  double *prev = NULL;
  for (int l = 1; l <= upto; l++) {
    lev g = mklev(c->P.dim, l);
    double *cur = (double *)malloc((size_t)g.np * sizeof(double));
    if (!cur) {
      free(prev);
      return NULL;
    }
    if (l == 1) {
      cur[0] = c->u[1].v[0];
    } else {
      lev gc = mklev(c->P.dim, l - 1);
      prolong(&gc, &g, prev, cur, cnt);
      long long cc = 0;
#pragma omp parallel for reduction(+ : cc) schedule(static)
      for (int64_t p = 0; p < g.np; p++) cur[p] = xadd(c->u[l].v[p], cur[p], &cc);
      *cnt += cc;
    }
    free(prev);
    prev = cur;
  }
  return prev;
}

int cmgo_decode_solution(const cmgo_ctx *c, double *out) {
  long long cnt = 0;
  double *uh = decode_chain(c, c->L, &cnt);
  if (!uh) return CMGO_ENOMEM;
  memcpy(out, uh, (size_t)mklev(c->P.dim, c->L).np * sizeof(double));
  free(uh);
  return CMGO_OK;
}

/* Algorithm 2 (fmgResidual): decode u^_L, t_L = f_L - A_L u^_L, r_L = round(t_L);
 * with no pre-smoothing the hierarchy t_l = R_(l+1) t_(l+1), r_l = round(t_l)
 * feeds the cycle as well. */
int cmgo_residual(cmgo_ctx *c) {
  int L = c->L, d = c->P.dim;
  lev g = mklev(d, L);
  long long cnt = 0;
  double *uh = decode_chain(c, L, &cnt);
  double *Au = (double *)malloc((size_t)g.np * sizeof(double));
  if (!uh || !Au) {
    free(uh);
    free(Au);
    return setst(c, CMGO_ENOMEM);
  }
  long long cc = 0;
  if (c->P.coef) {
    /* diffusion: the outer residual in FP64, t = fl(f - A u^) with A in the
     * order of A_at_diff64 (u^ itself is exact) */
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g.nz; k++)
      for (int j = 0; j < g.n; j++)
        for (int i = 0; i < g.n; i++) {
          int64_t p = idx(&g, i, j, k);
          volatile double a = A_at_diff64(c, uh, &g, i, j, k);
          c->t[p] = f_at(c, L, i + 1, j + 1, k + 1) - a;
        }
  } else {
    apply_A(&g, uh, Au, &cnt);
#pragma omp parallel for collapse(2) reduction(+ : cc) schedule(static)
    for (int k = 0; k < g.nz; k++)
      for (int j = 0; j < g.n; j++)
        for (int i = 0; i < g.n; i++) {
          int64_t p = idx(&g, i, j, k);
          c->t[p] = xsub(f_at(c, L, i + 1, j + 1, k + 1), Au[p], &cc);
        }
  }
  cnt += cc;
  free(uh);
  free(Au);
  int st = round_dense(&g, c->t, Wr(c, L), &c->r[L]);
  if (c->P.nu1 == 0 && L > 1 && st == CMGO_OK) {
    /* Table 1 keeps t^ at (p+1)L + b1 bits in fmgResidual: every level of the
     * restriction chain rounds t_l = R_(l+1) t_(l+1) to that width (here BFP
     * blocks of that width) before r_l = round(t_l) is formed from it. */
    sec tb;
    lev gm = mklev(d, L);
    if (sec_alloc(&tb, &gm) != CMGO_OK) return setst(c, CMGO_ENOMEM);
    st = round_dense(&g, c->t, Wt(c), &tb);
    for (int l = L - 1; l >= 1 && st == CMGO_OK; l--) {
      lev gf = mklev(d, l + 1), gc = mklev(d, l);
      double *tc = (double *)malloc((size_t)gc.np * sizeof(double));
      if (!tc) {
        st = CMGO_ENOMEM;
        break;
      }
      restrict_(&gf, &gc, tb.v, tc, &cnt);
      st = round_dense(&gc, tc, Wt(c), &tb);
      if (st == CMGO_OK) st = round_dense(&gc, tb.v, Wr(c, l), &c->r[l]);
      free(tc);
    }
    free(tb.v);
    free(tb.e);
  }
  c->inexact += cnt;
  return setst(c, st);
}

/* Jacobi weight per level: M_l = c_l I with c_l = omega / (2d h_l^(d-2)). */
static double cjac(cmgo_ctx *c, int l, long long *cnt) {
  double d2 = 2.0 * c->P.dim;
  double cw = c->P.omega / d2;
  if (fma(cw, d2, -c->P.omega) != 0.0) (*cnt)++;
  return ldexp(cw, (c->P.dim - 2) * l);
}

/* colour of 0-based node (i, j, k): red (0) when (i+1)+(j+1)+(k+1) is even */
static inline int node_colour(int dim, int i, int j, int k) {
  return ((i + 1) + (j + 1) + (dim == 3 ? (k + 1) : 0)) & 1;
}

/* one weighted-Jacobi sweep y <- round(y + c (rhs - A z - A y)) on level l
 * (eq. smoother on the compact equation eq. cfas, with s = 0); z may be NULL.
 * colour >= 0 restricts the update to the nodes of that colour (the others keep
 * their value): a red half-sweep followed by a black one is one red-black
 * Gauss-Seidel sweep, since nodes of one colour couple only to the other. */

static int jacobi(cmgo_ctx *c, int l, const double *z, long long *cnt, int colour) {
  lev g = mklev(c->P.dim, l);
  double cl = cjac(c, l, cnt);
  double *Ay = (double *)malloc((size_t)g.np * sizeof(double));
  double *Az = z ? (double *)malloc((size_t)g.np * sizeof(double)) : NULL;
  double *yn = (double *)malloc((size_t)g.np * sizeof(double));
  if (!Ay || !yn || (z && !Az)) {
    free(Ay);
    free(Az);
    free(yn);
    return CMGO_ENOMEM;
  }
  apply_A(&g, c->y[l].v, Ay, cnt);
  if (z) apply_A(&g, z, Az, cnt);
  long long cc = 0;
#pragma omp parallel for reduction(+ : cc) schedule(static)
  for (int64_t p = 0; p < g.np; p++) {
    const int i = (int)(p % g.n), j = (int)((p / g.n) % g.n), k = (int)(p / ((int64_t)g.n * g.n));
    if (colour >= 0 && node_colour(g.dim, i, j, k) != colour) {  /* other colour: kept */
      yn[p] = c->y[l].v[p];
      continue;
    }
    double res = c->rc[l].v[p];
    if (z) res = xsub(res, Az[p], &cc);
    res = xsub(res, Ay[p], &cc);
    yn[p] = xadd(c->y[l].v[p], xmul(cl, res, &cc), &cc);
  }
  *cnt += cc;
  int st = round_dense(&g, yn, Wr(c, l), &c->y[l]);
  free(Ay);
  free(Az);
  free(yn);
  return st;
}

/* the binary32 and binary64 cycles: sweep, down-leg right-hand side, up-leg */
#define REAL float
#define CYC(name) name##_f32
#define TO_REAL to_f32
#include "cycle_real.inc"
#undef REAL
#undef CYC
#undef TO_REAL
#define REAL double
#define CYC(name) name##_f64
#define TO_REAL to_f64
#include "cycle_real.inc"
#undef REAL
#undef CYC
#undef TO_REAL

/* the sweep of the configured cycle arithmetic */
static int sweep_any(cmgo_ctx *c, int l, long long *cnt, int colour) {
  if (c->P.arith == 1) return jacobi_f32(c, l, NULL, cnt, colour);
  if (c->P.arith == 2) return jacobi_f64(c, l, NULL, cnt, colour);
  return jacobi(c, l, NULL, cnt, colour);
}

/* Down-leg on level l >= 2: y~_l = 0, nu1 sweeps on A y = rc_l (the coarser
 * sections are still zero, so z_l = 0), then the level-(l-1) right-hand side
 * rc_(l-1) = round(R_l (rc_l - A_l y~_l)), which equals r^_(l-1) - s^_(l-1) of
 * eq. cfas.  With nu1 = 0 it is r_(l-1) from fmgResidual (s = 0, Sec. 4). */
int cmgo_down(cmgo_ctx *c, int l) {
  if (l < 2 || l > c->L) return setst(c, CMGO_EINVAL);
  lev g = mklev(c->P.dim, l), gc = mklev(c->P.dim, l - 1);
  long long cnt = 0;
  int st = CMGO_OK;
  if (l == c->L) sec_copy(&c->rc[l], &c->r[l], &g);
  sec_zero(&c->y[l], &g, Wr(c, l));
  for (int s = 0; s < c->P.nu1 && st == CMGO_OK; s++)
    st = sweep_any(c, l, &cnt, -1);
  if (st == CMGO_OK && c->P.arith && c->P.nu1 > 0) {
    /* floating-point cycle: rc_(l-1) from d = fl(rc - A y) (cycle_real.inc) */
    st = c->P.arith == 1 ? down_rhs_f32(c, l, &cnt) : down_rhs_f64(c, l, &cnt);
  } else if (st == CMGO_OK) {
    if (c->P.nu1 > 0) {
      double *Ay = (double *)malloc((size_t)g.np * sizeof(double));
      double *dd = (double *)malloc((size_t)g.np * sizeof(double));
      double *rcc = (double *)malloc((size_t)gc.np * sizeof(double));
      if (!Ay || !dd || !rcc) {
        free(Ay);
        free(dd);
        free(rcc);
        return setst(c, CMGO_ENOMEM);
      }
      apply_A(&g, c->y[l].v, Ay, &cnt);
      long long cc = 0;
#pragma omp parallel for reduction(+ : cc) schedule(static)
      for (int64_t p = 0; p < g.np; p++) dd[p] = xsub(c->rc[l].v[p], Ay[p], &cc);
      cnt += cc;
      restrict_(&g, &gc, dd, rcc, &cnt);
      st = round_dense(&gc, rcc, Wr(c, l - 1), &c->rc[l - 1]);
      free(Ay);
      free(dd);
      free(rcc);
    } else {
      sec_copy(&c->rc[l - 1], &c->r[l - 1], &gc);
    }
  }
  c->inexact += cnt;
  return setst(c, st);
}

/* Level 1 holds a single unknown: solved exactly, y~_1 = round(rc_1 / A_1). */
int cmgo_coarse(cmgo_ctx *c) {
  lev g = mklev(c->P.dim, 1);
  if (c->L == 1) sec_copy(&c->rc[1], &c->r[1], &g);
  double x = c->P.coef ? c->rc[1].v[0] / diag1_diff64(c) : c->rc[1].v[0] / A1(c->P.dim);
  int st = round_dense(&g, &x, Wr(c, 1), &c->y[1]);
  c->w[1][0] = c->y[1].v[0];
  return setst(c, st);
}

/* Up-leg on level l >= 2 (Algorithm 1, coarse-to-fine sweep):
 * z_l = P_l (y~_(l-1) + z_(l-1)) = P_l w_(l-1), nu2 sweeps on
 * A y~_l = rc_l - A z_l, then w_l = y~_l + z_l for the next finer level. */
int cmgo_up(cmgo_ctx *c, int l) {
  if (l < 2 || l > c->L) return setst(c, CMGO_EINVAL);
  lev g = mklev(c->P.dim, l), gc = mklev(c->P.dim, l - 1);
  long long cnt = 0;
  int st = CMGO_OK;
  if (c->P.arith) { /* floating-point cycle: z = P w_(l-1), w_l = y~_l + z (cycle_real.inc) */
    st = c->P.arith == 1 ? up_f32(c, l, &cnt) : up_f64(c, l, &cnt);
    c->inexact += cnt;
    return setst(c, st);
  }
  double *z = (double *)malloc((size_t)g.np * sizeof(double));
  if (!z) return setst(c, CMGO_ENOMEM);
  prolong(&gc, &g, c->w[l - 1], z, &cnt);
  for (int s = 0; s < c->P.nu2 && st == CMGO_OK; s++) {
    if (c->P.smoother) { /* red-black Gauss-Seidel: red, then black */
      st = jacobi(c, l, z, &cnt, 0);
      if (st == CMGO_OK) st = jacobi(c, l, z, &cnt, 1);
    } else {
      st = jacobi(c, l, z, &cnt, -1);
    }
  }
  long long cc = 0;
#pragma omp parallel for reduction(+ : cc) schedule(static)
  for (int64_t p = 0; p < g.np; p++) c->w[l][p] = xadd(c->y[l].v[p], z[p], &cc);
  cnt += cc;
  free(z);
  c->inexact += cnt;
  return setst(c, st);
}

int cmgo_vcycle(cmgo_ctx *c) {
  int st = CMGO_OK;
  for (int l = c->L; l >= 2 && st == CMGO_OK; l--) st = cmgo_down(c, l);
  if (st == CMGO_OK) st = cmgo_coarse(c);
  for (int l = 2; l <= c->L && st == CMGO_OK; l++) st = cmgo_up(c, l);
  return st;
}

/* Algorithm 3, apply correction: u~_l <- round_reg(u~_l + y~_l) for every l. */
int cmgo_correct(cmgo_ctx *c) {
  int st = CMGO_OK;
  for (int l = 1; l <= c->L && st == CMGO_OK; l++) {
    lev g = mklev(c->P.dim, l);
    double *s = (double *)malloc((size_t)g.np * sizeof(double));
    if (!s) return setst(c, CMGO_ENOMEM);
    long long cc = 0;
#pragma omp parallel for reduction(+ : cc) schedule(static)
    for (int64_t p = 0; p < g.np; p++) s[p] = xadd(c->u[l].v[p], c->y[l].v[p], &cc);
    c->inexact += cc;
    st = round_dense(&g, s, Wu(c, l), &c->u[l]);
    free(s);
  }
  return setst(c, st);
}

int cmgo_ir_iteration(cmgo_ctx *c) {
  int st = cmgo_residual(c);
  if (st == CMGO_OK) st = cmgo_vcycle(c);
  if (st == CMGO_OK) st = cmgo_correct(c);
  return st;
}

int cmgo_fmg(cmgo_ctx *c) {
  int st = cmgo_start(c);
  for (int L = 2; L <= c->P.Lmax && st == CMGO_OK; L++) {
    st = cmgo_next_level(c);
    for (int it = 0; it < c->P.N && st == CMGO_OK; it++) st = cmgo_ir_iteration(c);
  }
  return st;
}

/* ------------------------------------------------------------------------- */
/* section access                                                             */
/* ------------------------------------------------------------------------- */

static const sec *pick(const cmgo_ctx *c, int which, int l) {
  switch (which) {
    case CMGO_U: return &c->u[l];
    case CMGO_R: return &c->r[l];
    case CMGO_RC: return &c->rc[l];
    case CMGO_Y: return &c->y[l];
  }
  return NULL;
}

int cmgo_get_section(const cmgo_ctx *c, int which, int level, uint32_t *words, int8_t *e,
                     double *values) {
  if (level < 1 || level > c->P.Lmax || !c->w[level]) return CMGO_EINVAL;  /* level not reached */
  const sec *s = pick(c, which, level);
  if (!s) return CMGO_EINVAL;
  lev g = mklev(c->P.dim, level);
  if (values) memcpy(values, s->v, (size_t)g.np * sizeof(double));
  if (e) memcpy(e, s->e, (size_t)g.nb);
  if (words) {
    if (s->W < 2 || s->W > 32) return CMGO_EINVAL;
    for (int k = 0; k < g.nz; k++)
      for (int j = 0; j < g.n; j++)
        for (int bx = 0; bx < g.nbx; bx++) {
          int64_t b = ((int64_t)k * g.n + j) * g.nbx + bx;
          int64_t q[32] = {0};
          int eb = s->e[b];
          for (int i = 0; i < 32 && 32 * bx + i < g.n; i++)
            q[i] = eb == -128 ? 0 : (int64_t)ldexp(s->v[idx(&g, 32 * bx + i, j, k)], s->W - 1 - eb);
          pack_block(q, s->W, words + b * s->W);
        }
  }
  return CMGO_OK;
}

int cmgo_set_section(cmgo_ctx *c, int which, int level, int W, const uint32_t *words,
                     const int8_t *e) {
  if (level < 1 || level > c->P.Lmax || W < 2 || W > 32) return CMGO_EINVAL;
  if (ensure_level(c, level)) return CMGO_ENOMEM;
  sec *s = (sec *)pick(c, which, level);
  if (!s) return CMGO_EINVAL;
  lev g = mklev(c->P.dim, level);
  int st = CMGO_OK;
  s->W = W;
  memcpy(s->e, e, (size_t)g.nb);
  for (int k = 0; k < g.nz; k++)
    for (int j = 0; j < g.n; j++)
      for (int bx = 0; bx < g.nbx; bx++) {
        int64_t b = ((int64_t)k * g.n + j) * g.nbx + bx;
        for (int i = 0; i < 32 && 32 * bx + i < g.n; i++) {
          int64_t q = unpack_code(words + b * W, W, i);
          if (q == -(int64_t)(1ull << (W - 1))) st = CMGO_ECORRUPT;
          s->v[idx(&g, 32 * bx + i, j, k)] = e[b] == -128 ? 0.0 : ldexp((double)q, e[b] - W + 1);
        }
      }
  return st;
}

int cmgo_last_t(const cmgo_ctx *c, double *out) {
  if (c->L < 1) return CMGO_EINVAL;
  memcpy(out, c->t, (size_t)mklev(c->P.dim, c->L).np * sizeof(double));
  return CMGO_OK;
}

int cmgo_last_w(const cmgo_ctx *c, int level, double *out) {
  if (level < 1 || level > c->L) return CMGO_EINVAL;
  memcpy(out, c->w[level], (size_t)mklev(c->P.dim, level).np * sizeof(double));
  return CMGO_OK;
}
